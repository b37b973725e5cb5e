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
constexpr uint64_t kGenBlock = 4096; // positions per block (4 per Philox call, 4 calls per thread)

__device__ __forceinline__ uint8_t gen_letter(const ah_gen_segment &s, uint32_t u)
{
    if (s.letter)
        return (uint8_t)s.letter;
    return u < s.t_a ? 'A' : (u < s.t_c ? 'C' : (u < s.t_g ? 'G' : 'T'));
}

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

__global__ void __launch_bounds__(kGenThreads) gen_bases_kernel(const ah_gen_segment *__restrict__ segs,
                                                                 uint64_t n_segs, uint32_t k0, uint32_t k1,
                                                                 uint64_t base0, uint64_t n, uint8_t *__restrict__ out)
{
    __shared__ uint64_t bracket[2];
    const uint64_t p0 = base0 + (uint64_t)blockIdx.x * kGenBlock; // multiple of 4 (base0 is)
    const uint64_t p1 = min(base0 + n, p0 + kGenBlock);
    if (threadIdx.x == 0) {
        bracket[0] = seg_of(segs, 0, n_segs, p0);
        bracket[1] = min(n_segs, seg_of(segs, 0, n_segs, p1 - 1) + 1);
    }
    __syncthreads();
    const uint64_t s_lo = bracket[0], s_hi = bracket[1];
    for (uint64_t q = p0 / 4 + threadIdx.x; q * 4 < p1; q += kGenThreads) {
        const uint4 r = philox4x32_10(make_uint4((uint32_t)q, (uint32_t)(q >> 32), 0u, 0u), k0, k1);
        const uint32_t u[4] = {r.x, r.y, r.z, r.w};
        uint8_t b[4];
        uint64_t s = seg_of(segs, s_lo, s_hi, q * 4);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint64_t P = q * 4 + j;
            while (s + 1 < s_hi && segs[s].end <= P)
                ++s;
            b[j] = gen_letter(segs[s], u[j]);
        }
        const uint64_t o = q * 4 - base0;
        if (q * 4 + 4 <= p1 && ((reinterpret_cast<uintptr_t>(out) + o) & 3) == 0) {
            *reinterpret_cast<uint32_t *>(out + o) = b[0] | (uint32_t)b[1] << 8 | (uint32_t)b[2] << 16 | (uint32_t)b[3] << 24;
        } else {
            for (int j = 0; j < 4 && q * 4 + j < p1; ++j)
                out[o + j] = b[j];
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
                           cudaStream_t s)
{
    if (n == 0)
        return;
    const uint64_t blocks = (n + kGenBlock - 1) / kGenBlock;
    if (blocks > 0x7fffffffull)
        throw Error(AH_ERR_ARG, "ah_generate_bases: range too large for one call");
    gen_bases_kernel<<<(unsigned)blocks, kGenThreads, 0, s>>>(segs, n_segs, (uint32_t)seed, (uint32_t)(seed >> 32),
                                                               base0, n, out);
    AH_CUDA(cudaGetLastError());
    if (n_patches) {
        const uint64_t pb = std::min<uint64_t>((n_patches + 255) / 256, 8192);
        gen_patch_kernel<<<(unsigned)pb, 256, 0, s>>>(patch_pos, patch_bytes, n_patches, base0, n, out);
        AH_CUDA(cudaGetLastError());
    }
}

} // namespace ah
