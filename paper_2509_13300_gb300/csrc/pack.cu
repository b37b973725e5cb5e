// Packer: ASCII genome -> tile-strided one-hot bitplanes (layout in ah_internal.h).
//
// One CTA packs one tile at a time.  The tile's 32 KB of ASCII are 32 rows of
// kTileW bytes (row b = flat positions t*kTileBases + b*kTileW + [0, kTileW)),
// plus the next tile's first 32 bytes ("row 32") for the extension words; a
// bulk async copy (TMA) brings them into shared memory.  Word j of plane x
// takes bit b from row b, column j, so thread i builds the four words of
// columns 4i .. 4i+3 alone, with no cross-lane traffic:
//   - per block of 4 rows it reads 4 row words (4 columns each) and
//     transposes the 4x4 bytes with PRMT, giving one register per column;
//   - base letters are told apart by bits 1 and 2 of the upper-cased byte
//     (A 00, C 01, T 10, G 11); those bits of 4 bytes are gathered into 4 bits
//     by one multiply whose partial products never overlap (no carries);
//   - a byte is a base only if it equals the letter its two bits name: the
//     expected letter comes from a 4-entry PRMT table, and an exact per-byte
//     zero test of the difference marks non-ACGT bytes (N, IUPAC, gaps, ...).
// Plane words then follow from (h, l, valid) with one LOP3 each.  About 0.2
// warp instructions per base, so the kernel is bound by HBM: 1 byte read and
// 0.516 bytes written per base.
#include "ah_internal.h"

namespace ah {
namespace {

constexpr int kRowWords = kTileW / 4; // u32 words per ASCII row in shared memory
constexpr int kPackThreads = kTileW / 4;

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void tma_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok)
                 : "r"(smem_addr(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// bounded wait: false after ~2 s instead of hanging
__device__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    if (mbar_try(bar, parity))
        return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try(bar, parity))
        if (global_ns() - t0 > 2000000000ull)
            return false;
    return true;
}

// bits 1 and 2 of the 4 bytes of u -> (l, h) as 4-bit masks; valid = byte is exactly A/C/G/T
__device__ __forceinline__ void classify4(uint32_t u, uint32_t &l4, uint32_t &h4, uint32_t &v4)
{
    const uint32_t t = (u >> 1) & 0x03030303u;                  // 2h + l per byte
    l4 = ((t & 0x01010101u) * 0x10204080u) >> 28;               // byte k bit 0 -> bit k
    h4 = (((t >> 1) & 0x01010101u) * 0x10204080u) >> 28;        // byte k bit 1 -> bit k
    const uint32_t x = t | (t >> 4);                            // nibbles t0 t1 in byte 0, t2 t3 in byte 2
    const uint32_t sel = __byte_perm(x, 0, 0x4420);             // 4 selector nibbles
    const uint32_t expect = __byte_perm(0x47544341u, 0, sel);   // "ACTG"[2h + l] per byte
    const uint32_t z = u ^ expect;
    const uint32_t nz = (((z & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | z) & 0x80808080u; // MSB set iff byte != 0
    v4 = ((nz ^ 0x80808080u) * 0x00204081u) >> 28;              // byte k MSB -> bit k
}

// Build plane words for columns 4*ci .. 4*ci+3 from rows r0 .. r0+31 of the
// staged tile and store them as words j0 .. j0+3 of the tile's planes.
__device__ __forceinline__ void pack_columns(const uint32_t *__restrict__ rows, int r0, int ci, uint32_t *__restrict__ dst,
                                             int j0)
{
    uint32_t L[4] = {0, 0, 0, 0}, H[4] = {0, 0, 0, 0}, V[4] = {0, 0, 0, 0};
#pragma unroll
    for (int rb = 0; rb < 8; ++rb) {
        const int r = r0 + 4 * rb;
        const uint32_t a = rows[(r + 0) * kRowWords + ci] & 0xDFDFDFDFu; // upper case
        const uint32_t b = rows[(r + 1) * kRowWords + ci] & 0xDFDFDFDFu;
        const uint32_t c = rows[(r + 2) * kRowWords + ci] & 0xDFDFDFDFu;
        const uint32_t d = rows[(r + 3) * kRowWords + ci] & 0xDFDFDFDFu;
        // 4x4 byte transpose: col k = bytes k of a, b, c, d
        const uint32_t t0 = __byte_perm(a, b, 0x5140), t1 = __byte_perm(a, b, 0x7362);
        const uint32_t t2 = __byte_perm(c, d, 0x5140), t3 = __byte_perm(c, d, 0x7362);
        const uint32_t col[4] = {__byte_perm(t0, t2, 0x5410), __byte_perm(t0, t2, 0x7632), __byte_perm(t1, t3, 0x5410),
                                 __byte_perm(t1, t3, 0x7632)};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            uint32_t l4, h4, v4;
            classify4(col[k], l4, h4, v4);
            L[k] |= l4 << (4 * rb);
            H[k] |= h4 << (4 * rb);
            V[k] |= v4 << (4 * rb);
        }
    }
    uint4 pa, pc, pg, pt;
    uint32_t *A = &pa.x, *C = &pc.x, *G = &pg.x, *T = &pt.x;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        A[k] = V[k] & ~H[k] & ~L[k];
        C[k] = V[k] & ~H[k] & L[k];
        T[k] = V[k] & H[k] & ~L[k];
        G[k] = V[k] & H[k] & L[k];
    }
    *reinterpret_cast<uint4 *>(dst + 0 * kTileWX + j0) = pa;
    *reinterpret_cast<uint4 *>(dst + 1 * kTileWX + j0) = pc;
    *reinterpret_cast<uint4 *>(dst + 2 * kTileWX + j0) = pg;
    *reinterpret_cast<uint4 *>(dst + 3 * kTileWX + j0) = pt;
}

__global__ void __launch_bounds__(kPackThreads) pack_kernel(const uint8_t *__restrict__ seq, uint64_t seq_base,
                                                            uint64_t seq_len, uint64_t n_bases,
                                                            uint32_t *__restrict__ planes, uint64_t t0, uint64_t t1,
                                                            int tma_ok, int *__restrict__ err)
{
    extern __shared__ __align__(128) uint32_t rows[]; // 33 rows of kTileW bytes
    __shared__ __align__(8) uint64_t bar;
    const uint64_t lim = n_bases < seq_base + seq_len ? n_bases : seq_base + seq_len;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    uint32_t phase = 0;
    for (uint64_t t = t0 + blockIdx.x; t < t1; t += gridDim.x) {
        const uint64_t p0 = t * kTileBases; // flat position of row 0, column 0
        const bool full = tma_ok && p0 >= seq_base && p0 + kTileBases + 32 <= lim;
        if (full) {
            if (threadIdx.x == 0) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(&bar)),
                             "r"((uint32_t)(kTileBases + 32))
                             : "memory");
                tma_load(rows, seq + (p0 - seq_base), (uint32_t)kTileBases, &bar);
                tma_load(rows + 32 * kRowWords, seq + (p0 + kTileBases - seq_base), 32u, &bar);
            }
            const bool ok = mbar_wait(&bar, phase);
            phase ^= 1;
            if (!__syncthreads_and(ok)) {
                if (threadIdx.x == 0)
                    atomicExch(err, kDevTimeout);
                return; // the copy never landed; nothing else is in flight
            }
        } else {
            // tail or unaligned tile: byte loads with bounds, zero past the end
            for (int w = threadIdx.x; w < 33 * kRowWords; w += blockDim.x) {
                const int r = w / kRowWords, cw = w % kRowWords;
                uint32_t v = 0;
                if (r < 32 || cw < 8) {
                    const uint64_t pos = p0 + (uint64_t)r * kTileW + 4ull * cw;
                    for (int q = 0; q < 4; ++q)
                        if (pos + q >= seq_base && pos + q < lim)
                            v |= (uint32_t)seq[pos + q - seq_base] << (8 * q);
                }
                rows[w] = v;
            }
            __syncthreads();
        }
        uint32_t *dst = planes + t * 4 * kTileWX;
        pack_columns(rows, 0, threadIdx.x, dst, 4 * threadIdx.x);
        if (threadIdx.x < kTileExt / 4) // extension words W .. W+31: rows 1 .. 32, columns 0 .. 31
            pack_columns(rows, 1, threadIdx.x, dst, kTileW + 4 * threadIdx.x);
        __syncthreads(); // the rows buffer is reused by the next tile
    }
}

// Decode the planes back to one byte per position (0 = no base, 1..4 = A C G T,
// 5 = more than one plane set, which the packer never produces).  Test aid.
__global__ void unpack_kernel(const uint32_t *__restrict__ planes, uint8_t *__restrict__ codes, uint64_t n_bases)
{
    for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n_bases;
         p += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t t = p / kTileBases, r = p % kTileBases;
        const int b = (int)(r / kTileW), j = (int)(r % kTileW);
        const uint32_t *base = planes + t * 4 * kTileWX + j;
        int n = 0, code = 0;
        for (int x = 0; x < 4; ++x)
            if ((base[x * kTileWX] >> b) & 1u) {
                ++n;
                code = x + 1;
            }
        codes[p] = (uint8_t)(n > 1 ? 5 : code);
    }
}

} // namespace

void launch_pack(const uint8_t *seq, uint64_t seq_base, uint64_t seq_len, uint64_t n_bases, uint32_t *planes,
                 uint64_t t0, uint64_t t1, int *err, cudaStream_t s)
{
    if (t1 <= t0)
        return;
    static_assert(kTileW % 128 == 0 && kTileExt == 32, "pack layout");
    const size_t smem = 33ull * kTileW; // 32 rows + the next tile's head (33 KB, under the 48 KB default)
    int dev = 0, sms = 148, per_sm = 1;
    AH_CUDA(cudaGetDevice(&dev));
    AH_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    AH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pack_kernel, kPackThreads, smem));
    uint64_t blocks = (uint64_t)sms * (uint64_t)(per_sm > 0 ? per_sm : 1);
    if (blocks > t1 - t0)
        blocks = t1 - t0;
    const int tma_ok = ((reinterpret_cast<uintptr_t>(seq) - seq_base) % 16 == 0) ? 1 : 0;
    pack_kernel<<<(unsigned)blocks, kPackThreads, smem, s>>>(seq, seq_base, seq_len, n_bases, planes, t0, t1, tma_ok,
                                                             err);
    AH_CUDA(cudaGetLastError());
}

void launch_unpack_check(const uint32_t *planes, uint64_t n_tiles, uint8_t *codes, uint64_t n_bases, cudaStream_t s)
{
    (void)n_tiles;
    if (n_bases == 0)
        return;
    uint64_t blocks = (n_bases + 255) / 256;
    if (blocks > 4096)
        blocks = 4096;
    unpack_kernel<<<(unsigned)blocks, 256, 0, s>>>(planes, codes, n_bases);
    AH_CUDA(cudaGetLastError());
}

} // namespace ah
