// Counter-based synthetic genomes on the device (the large and served
// workloads are generated where they are scanned).  Philox4x32-10 (Salmon,
// Moraes, Dror and Shaw, SC 2011), written from its published definition:
// ten rounds of two 32x32 -> 64-bit products (multipliers 0xD2511F53 and
// 0xCD9E8D57) mixed into the counter, the key bumped by the Weyl constants
// 0x9E3779B9 and 0xBB67AE85 between rounds.  Position P takes output P mod 4
// of the draw at counter (P div 4 low, P div 4 high, 0, 0), key (seed low,
// seed high), and maps it through its segment's integer thresholds; segments
// with a letter (N runs) write the letter; patches (planted primer sites)
// overwrite last.
#include <algorithm>

#include "ah_internal.h"

namespace ah {
namespace {

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

constexpr int kGenThreads = 256;
constexpr int kGenQuads = 16;                                        // consecutive Philox calls per thread
constexpr uint64_t kGenBlock = 4ull * kGenQuads * kGenThreads;      // 16,384 positions per block
constexpr int kGenStage = 128;                                       // segments staged in shared memory

// first segment whose end is above P, searched in [lo, hi)
__device__ __forceinline__ uint64_t seg_of(const ah_gen_segment *__restrict__ segs, uint64_t lo, uint64_t hi, uint64_t P)
{
    while (lo < hi) {
        const uint64_t mid = (lo + hi) >> 1;
        if (segs[mid].end <= P)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// Each thread draws kGenQuads consecutive quads (64 consecutive positions):
// its segment is found once and advanced as positions pass segment ends; the
// block's segments are staged in shared memory when they fit; four quads
// leave as one 16-byte store when aligned.
__global__ void __launch_bounds__(kGenThreads, 1) gen_bases_kernel(const ah_gen_segment *__restrict__ segs,
                                                                 uint64_t n_segs, uint32_t k0, uint32_t k1,
                                                                 uint64_t base0, uint64_t n, uint8_t *__restrict__ out,
                                                                 int *__restrict__ err)
{
    __shared__ uint64_t bracket[2];
    __shared__ ah_gen_segment st[kGenStage];
    const uint64_t p0 = base0 + (uint64_t)blockIdx.x * kGenBlock; // multiple of 4 (base0 is)
    const uint64_t p1 = min(base0 + n, p0 + kGenBlock);
    if (threadIdx.x == 0) {
        bracket[0] = seg_of(segs, 0, n_segs, p0);
        bracket[1] = min(n_segs, seg_of(segs, 0, n_segs, p1 - 1) + 1);
    }
    __syncthreads();
    const uint64_t s_lo = bracket[0], s_hi = bracket[1];
    if (s_lo >= n_segs || segs[s_hi - 1].end < p1) { // the segments end before this block's range
        for (uint64_t P = p0 + threadIdx.x; P < p1; P += kGenThreads)
            out[P - base0] = 'N';
        if (threadIdx.x == 0)
            atomicExch(err, kDevBounds);
        return;
    }
    const bool staged = s_hi - s_lo <= (uint64_t)kGenStage;
    if (staged)
        for (uint64_t i = threadIdx.x; i < s_hi - s_lo; i += kGenThreads)
            st[i] = segs[s_lo + i];
    __syncthreads();
    const ah_gen_segment *sg = staged ? st : segs + s_lo; // index relative to s_lo
    const uint64_t nsg = s_hi - s_lo;
    const uint64_t q0 = p0 / 4 + (uint64_t)threadIdx.x * kGenQuads;
    if (q0 * 4 >= p1)
        return;
    uint64_t s = seg_of(sg, 0, nsg, q0 * 4);
    // the current segment's fields in registers, reloaded only when a position passes its end;
    // positions counted from the thread's first one (32-bit)
    const uint64_t pbase = q0 * 4;
    auto rel_end = [&](uint64_t i) -> uint32_t { // segment end relative to pbase, saturated
        const uint64_t e = sg[i].end;
        return e <= pbase ? 0u : (e - pbase >= 0xffffffffull ? 0xffffffffu : (uint32_t)(e - pbase));
    };
    uint32_t send = rel_end(s), ta = sg[s].t_a, tc = sg[s].t_c, tg = sg[s].t_g, lt = sg[s].letter;
    uint32_t words[kGenQuads];
#pragma unroll
    for (int j = 0; j < kGenQuads; ++j) {
        const uint64_t q = q0 + j;
        const uint4 r = philox4x32_10(make_uint4((uint32_t)q, (uint32_t)(q >> 32), 0u, 0u), k0, k1);
        const uint32_t u[4] = {r.x, r.y, r.z, r.w};
        uint32_t w = 0;
#pragma unroll
        for (int x = 0; x < 4; ++x) {
            const uint32_t rp = 4u * j + x; // position - pbase
            while (rp >= send && s + 1 < nsg) {
                ++s;
                send = rel_end(s);
                ta = sg[s].t_a;
                tc = sg[s].t_c;
                tg = sg[s].t_g;
                lt = sg[s].letter;
            }
            const uint32_t v = u[x];
            const uint32_t letter = lt ? lt : (v < ta ? 'A' : (v < tc ? 'C' : (v < tg ? 'G' : 'T')));
            w |= letter << (8 * x);
        }
        words[j] = w;
    }
    const uint64_t o = q0 * 4 - base0;
    const bool full = q0 * 4 + 4 * kGenQuads <= p1;
    if (full && ((reinterpret_cast<uintptr_t>(out) + o) & 15) == 0) {
#pragma unroll
        for (int j = 0; j < kGenQuads; j += 4)
            *reinterpret_cast<uint4 *>(out + o + 4 * j) = make_uint4(words[j], words[j + 1], words[j + 2], words[j + 3]);
    } else {
#pragma unroll
        for (int j = 0; j < kGenQuads; ++j)
            for (int x = 0; x < 4; ++x) {
                const uint64_t P = (q0 + j) * 4 + x;
                if (P < p1)
                    out[P - base0] = (uint8_t)(words[j] >> (8 * x));
            }
    }
}

__global__ void gen_patch_kernel(const uint64_t *__restrict__ pos, const uint8_t *__restrict__ bytes, uint64_t np,
                                 uint64_t base0, uint64_t n, uint8_t *__restrict__ out)
{
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < np; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t p = pos[i];
        if (p >= base0 && p < base0 + n)
            out[p - base0] = bytes[i];
    }
}

} // namespace

void launch_generate_bases(const ah_gen_segment *segs, uint64_t n_segs, uint64_t seed, const uint64_t *patch_pos,
                           const uint8_t *patch_bytes, uint64_t n_patches, uint64_t base0, uint64_t n, uint8_t *out,
                           int *err, cudaStream_t s)
{
    if (n == 0)
        return;
    const uint64_t blocks = (n + kGenBlock - 1) / kGenBlock;
    if (blocks > 0x7fffffffull)
        throw Error(AH_ERR_ARG, "ah_generate_bases: range too large for one call");
    gen_bases_kernel<<<(unsigned)blocks, kGenThreads, 0, s>>>(segs, n_segs, (uint32_t)seed, (uint32_t)(seed >> 32),
                                                               base0, n, out, err);
    AH_CUDA(cudaGetLastError());
    if (n_patches) {
        const uint64_t pb = std::min<uint64_t>((n_patches + 255) / 256, 8192);
        gen_patch_kernel<<<(unsigned)pb, 256, 0, s>>>(patch_pos, patch_bytes, n_patches, base0, n, out);
        AH_CUDA(cudaGetLastError());
    }
}

} // namespace ah
