// Packer: ASCII genome -> tile-strided one-hot bitplanes (layout in ah_internal.h).
//
// One CTA packs one tile at a time.  The tile's 32 KB of ASCII are 32 rows of
// kTileW bytes (row b = flat positions t*kTileBases + b*kTileW + [0, kTileW)),
// plus the next tile's first 32 bytes ("row 32") for the extension words; bulk
// async copies (TMA) bring them into shared memory, two tiles staged per CTA
// so the next copy overlaps the current packing.  Word j of plane x takes bit
// b from row b, column j, so thread i builds the four words of columns
// 4i .. 4i+3 alone, with no cross-lane traffic.  Per block of 4 rows it reads
// 4 row words (4 columns each) and transposes the 4x4 bytes with PRMT, giving
// one register per column (4 rows), and then:
//   - a letter's base is read from bits 1 and 2 of its byte (A 00, C 01,
//     T 10, G 11).  Bit 2 is copied up to bit 5, and one multiply by a
//     constant whose partial products never share a bit (so no carries)
//     moves bit 1 of the 4 bytes to bits 0..3 and bit 5 to bits 4..7 of the
//     product's high word; PRMT drops that byte into the column's even- or
//     odd-block word, and two masks per plane turn these into the column's
//     32-bit bit-1 and bit-2 words;
//   - a byte is a base only if it is exactly A/C/G/T in either case.  The
//     fast test: the byte must equal, up to case, the letter its low nibble
//     names (1 A, 3 C, 4 T, 7 G; an 8-entry PRMT table).  The low nibbles of
//     two rows interleave into a selector whose byte order is that of the
//     transpose's first stage, so one PRMT and one XOR per 4 bytes give 0 or
//     0x20 for every base byte; the thread ORs them over its 128 bytes.  Only
//     when some byte fails does the thread run the exact per-byte test for its
//     columns (a per-byte zero test and a gather by multiply).
// Plane words then follow from (h, l, valid) with one LOP3 each.  The work is
// split between the logic and the multiply pipes (shifts by constants are
// multiplies by run-time powers of two) so that the kernel is bound by HBM:
// 1 byte read and 0.516 bytes written per base.
#include <algorithm>
#include <cstdlib>

#include "ah_internal.h"

namespace ah {
namespace {

constexpr int kRowWords = kTileW / 4; // u32 words per ASCII row in shared memory
constexpr int kPackThreads = kTileW / 4;
constexpr int kRows = 33;                    // 32 rows + the next tile's head
constexpr int kBufWords = kRows * kRowWords; // one staged tile

// PRMT table: byte n is the (upper-case) letter whose low nibble is n, 0xFF
// where no letter has that nibble
constexpr uint32_t kLetterLo = 0x43FF41FFu, kLetterHi = 0x47FFFF54u;
// bit 8k+1 -> bit 32+k and bit 8k+5 -> bit 36+k of the 64-bit product: byte k
// moves by 31 - 7k; every partial product lands on its own bit
constexpr uint32_t kGatherLH = (1u << 31) | (1u << 24) | (1u << 17) | (1u << 10);

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

// Exact validity of 4 bytes (one column, 4 rows): bit k set iff byte k is
// exactly one of A C G T in either case.
__device__ __forceinline__ uint32_t valid4(uint32_t raw, uint32_t sixteen, uint32_t top4)
{
    const uint32_t n = raw & 0x0F0F0F0Fu;
    const uint32_t x = n + __umulhi(n, top4);                       // nibbles n0 n1 | n2 n3 (n | n >> 4)
    const uint32_t sel = __byte_perm(x, 0, 0x4420);                 // 4 selector nibbles
    const uint32_t expect = __byte_perm(kLetterLo, kLetterHi, sel); // letter the nibble names
    const uint32_t z = (raw & 0xDFDFDFDFu) ^ expect;                // upper-cased letter vs expected
    const uint32_t s = (z & 0x7F7F7F7Fu) + 0x7F7F7F7Fu;             // byte MSB: low 7 bits non-zero
    const uint32_t valid = ~(s | z) & 0x80808080u;                  // byte MSB: z byte == 0
    return __umulhi(valid * 0x00204081u, sixteen);                  // byte k MSB -> bit k
}

// Classify 4 bytes (one column, 4 rows) and add their bits at the nibble
// given by pw (a run-time power of two) of the column's L (bit 1 of the
// letter), H (bit 2) and V (exactly one of A C G T, either case) words.
__device__ __forceinline__ void classify4(uint32_t raw, uint32_t pw, uint32_t sixteen, uint32_t top4, uint32_t &L,
                                          uint32_t &H, uint32_t &V)
{
    const uint32_t l4 = __umulhi((raw & 0x02020202u) * 0x08102040u, sixteen); // byte k bit 1 -> bit k
    const uint32_t h4 = __umulhi((raw & 0x04040404u) * 0x04081020u, sixteen); // byte k bit 2 -> bit k
    L = l4 * pw + L; // the nibbles are disjoint: add = or
    H = h4 * pw + H;
    V = valid4(raw, sixteen, top4) * pw + V;
}

// 4x4 byte transpose of rows r .. r+3 (row(q) = this thread's word of row q,
// 4 columns): col[k] = byte k of each row; t[] = the first stage, (a0 b0 a1
// b1), (a2 b2 a3 b3), (c0 d0 c1 d1), (c2 d2 c3 d3).
template <class Row>
__device__ __forceinline__ void load_block(const Row &rowf, int r, uint32_t (&row)[4], uint32_t (&t)[4],
                                           uint32_t (&col)[4])
{
#pragma unroll
    for (int q = 0; q < 4; ++q)
        row[q] = rowf(r + q);
    t[0] = __byte_perm(row[0], row[1], 0x5140);
    t[1] = __byte_perm(row[0], row[1], 0x7362);
    t[2] = __byte_perm(row[2], row[3], 0x5140);
    t[3] = __byte_perm(row[2], row[3], 0x7362);
    col[0] = __byte_perm(t[0], t[2], 0x5410);
    col[1] = __byte_perm(t[0], t[2], 0x7632);
    col[2] = __byte_perm(t[1], t[3], 0x5410);
    col[3] = __byte_perm(t[1], t[3], 0x7632);
}

// Build plane words for columns 4*ci .. 4*ci+3 from rows 0 .. 31 of the
// staged tile and store them as words 4*ci .. 4*ci+3 of the tile's planes.
// Threads of columns below kTileExt also store the extension words W + 4*ci
// .. W + 4*ci + 3: bit b of extension word W + j is the base at row b + 1,
// column j, i.e. the column's own word shifted right by one with bit 31 from
// row 32 (the next tile's first row, staged with the tile).
template <class Row>
__device__ __forceinline__ void pack_columns(const Row &rowf, int ci, uint32_t *__restrict__ dst, uint32_t one)
{
    const int j0 = 4 * ci;
    const uint32_t eight = one << 3, sixteen = one << 4, top4 = one << 28;
    // per column: byte m of ev / od = bits 1 (low nibble) and 2 (high nibble)
    // of rows 8m .. 8m+3 / 8m+4 .. 8m+7
    uint32_t ev[4] = {0, 0, 0, 0}, od[4] = {0, 0, 0, 0};
    uint32_t bad = 0; // OR of (byte ^ letter its nibble names): only 0x20 bits if all are bases
#pragma unroll
    for (int rb = 0; rb < 8; ++rb) {
        uint32_t row[4], t[4], col[4];
        load_block(rowf, 4 * rb, row, t, col);
        const uint32_t s01 = (row[0] & 0x0F0F0F0Fu) | ((row[1] * sixteen) & 0xF0F0F0F0u);
        const uint32_t s23 = (row[2] & 0x0F0F0F0Fu) | ((row[3] * sixteen) & 0xF0F0F0F0u);
        bad |= (t[0] ^ __byte_perm(kLetterLo, kLetterHi, s01)) | (t[1] ^ __byte_perm(kLetterLo, kLetterHi, s01 >> 16));
        bad |= (t[2] ^ __byte_perm(kLetterLo, kLetterHi, s23)) | (t[3] ^ __byte_perm(kLetterLo, kLetterHi, s23 >> 16));
        // byte 0 of the gathered word goes to byte rb / 2
        const uint32_t put = rb / 2 == 0 ? 0x3214u : rb / 2 == 1 ? 0x3240u : rb / 2 == 2 ? 0x3410u : 0x4210u;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t w = (col[k] & 0x02020202u) | ((col[k] * eight) & 0x20202020u);
            const uint32_t g = __umulhi(w, kGatherLH); // bits 0..3: bit 1 of rows 4rb.., bits 4..7: bit 2
            if (rb & 1)
                od[k] = __byte_perm(od[k], g, put);
            else
                ev[k] = __byte_perm(ev[k], g, put);
        }
    }
    uint32_t V[4] = {~0u, ~0u, ~0u, ~0u};
    if (bad & 0xDFDFDFDFu) { // some byte is not a base: exact per-byte test for these columns
#pragma unroll
        for (int k = 0; k < 4; ++k)
            V[k] = 0;
#pragma unroll
        for (int rb = 0; rb < 8; ++rb) {
            uint32_t row[4], t[4], col[4];
            load_block(rowf, 4 * rb, row, t, col);
            const uint32_t pw = one << (4 * rb);
#pragma unroll
            for (int k = 0; k < 4; ++k)
                V[k] = valid4(col[k], sixteen, top4) * pw + V[k];
        }
    }
    uint4 pa, pc, pg, pt;
    uint32_t *A = &pa.x, *C = &pc.x, *G = &pg.x, *T = &pt.x;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint32_t L = (ev[k] & 0x0F0F0F0Fu) | ((od[k] * sixteen) & 0xF0F0F0F0u);
        const uint32_t H = (__umulhi(ev[k], top4) & 0x0F0F0F0Fu) | (od[k] & 0xF0F0F0F0u);
        A[k] = V[k] & ~H & ~L;
        C[k] = V[k] & ~H & L;
        T[k] = V[k] & H & ~L;
        G[k] = V[k] & H & L;
    }
    *reinterpret_cast<uint4 *>(dst + 0 * kTileWX + j0) = pa;
    *reinterpret_cast<uint4 *>(dst + 1 * kTileWX + j0) = pc;
    *reinterpret_cast<uint4 *>(dst + 2 * kTileWX + j0) = pg;
    *reinterpret_cast<uint4 *>(dst + 3 * kTileWX + j0) = pt;
    if (j0 < kTileExt) {
        // row 32 of these four columns: bit k of hl / hh / hv = byte k's letter bits and validity
        uint32_t hl = 0, hh = 0, hv = 0;
        classify4(rowf(32), one, one << 4, one << 28, hl, hh, hv);
        const uint32_t ha = hv & ~hh & ~hl, hc = hv & ~hh & hl, ht = hv & hh & ~hl, hg = hv & hh & hl;
        uint4 ea, ec, eg, et;
        uint32_t *EA = &ea.x, *EC = &ec.x, *EG = &eg.x, *ET = &et.x;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            EA[k] = (A[k] >> 1) | ((ha >> k & 1u) << 31);
            EC[k] = (C[k] >> 1) | ((hc >> k & 1u) << 31);
            EG[k] = (G[k] >> 1) | ((hg >> k & 1u) << 31);
            ET[k] = (T[k] >> 1) | ((ht >> k & 1u) << 31);
        }
        *reinterpret_cast<uint4 *>(dst + 0 * kTileWX + kTileW + j0) = ea;
        *reinterpret_cast<uint4 *>(dst + 1 * kTileWX + kTileW + j0) = ec;
        *reinterpret_cast<uint4 *>(dst + 2 * kTileWX + kTileW + j0) = eg;
        *reinterpret_cast<uint4 *>(dst + 3 * kTileWX + kTileW + j0) = et;
    }
}

__global__ void __launch_bounds__(kPackThreads, 6) pack_kernel(const uint8_t *__restrict__ seq, uint64_t seq_base,
                                                            uint64_t seq_len, uint64_t n_bases,
                                                            uint32_t *__restrict__ planes, uint64_t t0, uint64_t t1,
                                                            int tma_ok, uint32_t one, int *__restrict__ err)
{
    extern __shared__ __align__(128) uint32_t smem[]; // two staged tiles
    __shared__ __align__(8) uint64_t bar[2];
    const uint64_t lim = n_bases < seq_base + seq_len ? n_bases : seq_base + seq_len;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // a tile goes through TMA when all of its bytes (and the next tile's head) are present and aligned
    auto full = [&](uint64_t t) {
        const uint64_t p0 = t * kTileBases;
        return tma_ok && p0 >= seq_base && p0 + kTileBases + 32 <= lim;
    };
    auto issue = [&](uint64_t t, int sb) {
        const uint64_t p0 = t * kTileBases;
        uint32_t *rows = smem + sb * kBufWords;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(&bar[sb])),
                     "r"((uint32_t)(kTileBases + 32))
                     : "memory");
        tma_load(rows, seq + (p0 - seq_base), (uint32_t)kTileBases, &bar[sb]);
        tma_load(rows + 32 * kRowWords, seq + (p0 + kTileBases - seq_base), 32u, &bar[sb]);
    };
    uint32_t phase0 = 0, phase1 = 0;
    const uint64_t first = t0 + blockIdx.x;
    if (threadIdx.x == 0 && first < t1 && full(first))
        issue(first, 0);
    int it = 0;
    for (uint64_t t = first; t < t1; t += gridDim.x, ++it) {
        const int sb = it & 1;
        uint32_t *rows = smem + sb * kBufWords;
        const uint64_t next = t + gridDim.x;
        // the other buffer was released by the barrier that ended the previous tile
        if (threadIdx.x == 0 && next < t1 && full(next))
            issue(next, sb ^ 1);
        const uint64_t p0 = t * kTileBases;
        if (full(t)) {
            const bool ok = mbar_wait(&bar[sb], sb ? phase1 : phase0);
            if (sb)
                phase1 ^= 1;
            else
                phase0 ^= 1;
            if (!__syncthreads_and(ok)) {
                if (threadIdx.x == 0) {
                    atomicExch(err, kDevTimeout);
                    if (next < t1 && full(next)) // bounded wait for the copy still in flight
                        mbar_wait(&bar[sb ^ 1], sb ? phase0 : phase1);
                }
                return;
            }
        } else {
            // tail or unaligned tile: byte loads with bounds, zero past the end
            for (int w = threadIdx.x; w < kBufWords; w += blockDim.x) {
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
        const int ci = threadIdx.x;
        pack_columns([&](int r) { return rows[r * kRowWords + ci]; }, ci, planes + t * 4 * kTileWX, one);
        __syncthreads(); // this buffer is refilled two tiles from now
    }
}

// ---------------------------------------------------------------------------
// Packer from 2-bit base codes (the load form whose host input is a quarter
// of ASCII's size): base p is bits 2 (p % 4) .. 2 (p % 4) + 1 of byte p / 4,
// A 0, C 1, G 2, T 3; positions listed in `gaps` (sorted, disjoint (start,
// length) pairs) and positions at or past n_bases are no base (all four
// planes 0).  One block per tile: the tile's 8 KB of codes and the next
// tile's first 8 bytes (the extension row) are loaded into shared memory with
// coalesced 16-byte loads; thread ci builds the plane words of columns
// 4 ci .. 4 ci + 3, for which row b holds exactly byte ci of the row.  Four
// rows at a time: the rows' bytes form one 32-bit word, and each column's low
// and high code bits are gathered into a nibble by one carry-free multiply.
// A tile that a gap or the end of the data touches marks its no-base
// positions in a shared bitmap first; tile_gap[t] (built at load by a merge
// walk) is the first gap that ends after tile t's start.
// ---------------------------------------------------------------------------
constexpr int kCodeRowBytes = kTileW / 4;                  // 256 bytes of codes per row
constexpr int kCodeWords = (32 * kCodeRowBytes + 16) / 4;  // the tile + the extension row (16 bytes read)
constexpr int kInvWords = (kTileBases + 32) / 32;          // no-base bitmap of the tile + extension row

// bits 0, 8, 16, 24 of v (each 0 or 1) -> bits 0..3
__device__ __forceinline__ uint32_t gather4(uint32_t v) { return (v * 0x10204080u) >> 28; }

__global__ void __launch_bounds__(kPackThreads) pack2_kernel(const uint8_t *__restrict__ codes, uint64_t base0,
                                                             uint64_t n_avail, uint64_t n_bases,
                                                             const uint64_t *__restrict__ gaps, uint64_t n_gaps,
                                                             const uint32_t *__restrict__ tile_gap,
                                                             uint32_t *__restrict__ planes, uint64_t t0, uint64_t t1)
{
    __shared__ __align__(16) uint32_t cw[kCodeWords];
    __shared__ uint32_t inv[kInvWords];
    const int ci = threadIdx.x;
    const uint64_t avail_end = base0 + n_avail < n_bases ? base0 + n_avail : n_bases; // bases present here
    for (uint64_t t = t0 + blockIdx.x; t < t1; t += gridDim.x) {
        const uint64_t p0 = t * kTileBases, pe = p0 + kTileBases + 32; // the tile and its extension row
        // codes: bytes (p0 - base0) / 4 .. + 8208 of `codes`; zero past the available bytes
        const uint64_t cb0 = (p0 - base0) / 4;
        const uint64_t bytes_avail = (avail_end > p0 ? (avail_end - p0 + 3) / 4 : 0);
        if (bytes_avail >= (uint64_t)kCodeWords * 4) {
            const uint4 *src = reinterpret_cast<const uint4 *>(codes + cb0);
            for (int w = ci; w < kCodeWords / 4; w += blockDim.x)
                reinterpret_cast<uint4 *>(cw)[w] = __ldg(src + w);
        } else {
            for (int w = ci; w < kCodeWords; w += blockDim.x) {
                uint32_t v = 0;
                for (int q = 0; q < 4; ++q)
                    if ((uint64_t)(4 * w + q) < bytes_avail)
                        v |= (uint32_t)codes[cb0 + 4 * w + q] << (8 * q);
                cw[w] = v;
            }
        }
        // no-base positions: gaps that meet [p0, pe), and everything at or past avail_end;
        // the tile's first gap ending after p0 comes from the table built at load
        const uint64_t first_gap = tile_gap[t];
        const bool marked = (first_gap < n_gaps && gaps[2 * first_gap] < pe) || avail_end < pe;
        __syncthreads();
        if (marked) {
            for (int w = ci; w < kInvWords; w += blockDim.x)
                inv[w] = 0u;
            __syncthreads();
            auto mark = [&](uint64_t a, uint64_t b) { // positions [a, b) of the tile, relative to p0
                const uint64_t w0 = a >> 5, w1 = (b - 1) >> 5;
                for (uint64_t w = w0 + ci; w <= w1; w += blockDim.x) {
                    const uint64_t x0 = a > 32 * w ? a - 32 * w : 0, x1 = b < 32 * w + 32 ? b - 32 * w : 32;
                    const uint32_t m = (x1 - x0 >= 32 ? 0xffffffffu : ((1u << (x1 - x0)) - 1u)) << x0;
                    atomicOr(&inv[w], m);
                }
            };
            for (uint64_t g = first_gap; g < n_gaps && gaps[2 * g] < pe; ++g) {
                const uint64_t e = gaps[2 * g] + gaps[2 * g + 1];
                if (e <= p0) // (only out-of-order runs end before the tile: never index with them)
                    continue;
                const uint64_t a = gaps[2 * g] > p0 ? gaps[2 * g] - p0 : 0;
                const uint64_t b = (e < pe ? e : pe) - p0;
                if (b > a)
                    mark(a, b);
            }
            if (avail_end < pe)
                mark(avail_end > p0 ? avail_end - p0 : 0, pe - p0);
        }
        __syncthreads();
        const uint8_t *cbytes = reinterpret_cast<const uint8_t *>(cw);
        uint32_t lo[4] = {0, 0, 0, 0}, hi[4] = {0, 0, 0, 0};
#pragma unroll
        for (int rb = 0; rb < 8; ++rb) {
            const uint32_t x = (uint32_t)cbytes[(4 * rb + 0) * kCodeRowBytes + ci] |
                               ((uint32_t)cbytes[(4 * rb + 1) * kCodeRowBytes + ci] << 8) |
                               ((uint32_t)cbytes[(4 * rb + 2) * kCodeRowBytes + ci] << 16) |
                               ((uint32_t)cbytes[(4 * rb + 3) * kCodeRowBytes + ci] << 24);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                lo[k] |= gather4((x >> (2 * k)) & 0x01010101u) << (4 * rb);
                hi[k] |= gather4((x >> (2 * k + 1)) & 0x01010101u) << (4 * rb);
            }
        }
        uint32_t val[4] = {0xffffffffu, 0xffffffffu, 0xffffffffu, 0xffffffffu};
        if (marked) {
#pragma unroll 4
            for (int b = 0; b < 32; ++b) {
                const uint32_t nib = (inv[b * (kTileW / 32) + (ci >> 3)] >> (4 * (ci & 7))) & 0xFu;
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    val[k] &= ~(((nib >> k) & 1u) << b);
            }
        }
        uint4 pa, pc, pg, pt;
        uint32_t *A = &pa.x, *C = &pc.x, *G = &pg.x, *T = &pt.x;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            A[k] = val[k] & ~hi[k] & ~lo[k];
            C[k] = val[k] & ~hi[k] & lo[k];
            G[k] = val[k] & hi[k] & ~lo[k];
            T[k] = val[k] & hi[k] & lo[k];
        }
        uint32_t *dst = planes + t * 4 * kTileWX;
        const int j0 = 4 * ci;
        *reinterpret_cast<uint4 *>(dst + 0 * kTileWX + j0) = pa;
        *reinterpret_cast<uint4 *>(dst + 1 * kTileWX + j0) = pc;
        *reinterpret_cast<uint4 *>(dst + 2 * kTileWX + j0) = pg;
        *reinterpret_cast<uint4 *>(dst + 3 * kTileWX + j0) = pt;
        if (j0 < kTileExt) {
            // extension words: row b + 1 of the same column, bit 31 from the next tile's head
            const uint32_t hb = cbytes[32 * kCodeRowBytes + ci];
            uint32_t hv = 0xFu;
            if (marked)
                hv = ~(inv[kTileBases / 32 + (ci >> 3)] >> (4 * (ci & 7))) & 0xFu;
            uint4 ea, ec, eg, et;
            uint32_t *EA = &ea.x, *EC = &ec.x, *EG = &eg.x, *ET = &et.x;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint32_t code = (hb >> (2 * k)) & 3u, v = (hv >> k) & 1u;
                EA[k] = (A[k] >> 1) | ((v & (code == 0)) << 31);
                EC[k] = (C[k] >> 1) | ((v & (code == 1)) << 31);
                EG[k] = (G[k] >> 1) | ((v & (code == 2)) << 31);
                ET[k] = (T[k] >> 1) | ((v & (code == 3)) << 31);
            }
            *reinterpret_cast<uint4 *>(dst + 0 * kTileWX + kTileW + j0) = ea;
            *reinterpret_cast<uint4 *>(dst + 1 * kTileWX + kTileW + j0) = ec;
            *reinterpret_cast<uint4 *>(dst + 2 * kTileWX + kTileW + j0) = eg;
            *reinterpret_cast<uint4 *>(dst + 3 * kTileWX + kTileW + j0) = et;
        }
        __syncthreads(); // the shared buffers are refilled for the next tile
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


namespace {
__global__ void copy_words_kernel(const uint32_t *__restrict__ src, uint32_t *__restrict__ dst, uint64_t n)
{
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}
} // namespace

void launch_pack2(const uint8_t *codes, uint64_t base0, uint64_t n_avail, uint64_t n_bases, const uint64_t *gaps,
                  uint64_t n_gaps, const uint32_t *tile_gap, uint32_t *planes, uint64_t t0, uint64_t t1,
                  cudaStream_t s)
{
    if (t1 <= t0)
        return;
    if (reinterpret_cast<uintptr_t>(codes) % 16 != 0 || base0 % kTileBases != 0)
        throw Error(AH_ERR_ARG, "2-bit codes must start 16-byte aligned at a tile boundary");
    static int cached_dev = -1, sms = 148;
    int dev = 0;
    AH_CUDA(cudaGetDevice(&dev));
    if (dev != cached_dev) {
        AH_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        cached_dev = dev;
    }
    const uint64_t blocks = std::min<uint64_t>(t1 - t0, (uint64_t)sms * 8);
    pack2_kernel<<<(unsigned)blocks, kPackThreads, 0, s>>>(codes, base0, n_avail, n_bases, gaps, n_gaps, tile_gap,
                                                           planes, t0, t1);
    AH_CUDA(cudaGetLastError());
}

void launch_copy_words(const uint32_t *src, uint32_t *dst, uint64_t n_words, cudaStream_t s)
{
    if (!n_words)
        return;
    const uint64_t blocks = std::min<uint64_t>((n_words + 255) / 256, 1024);
    copy_words_kernel<<<(unsigned)blocks, 256, 0, s>>>(src, dst, n_words);
    AH_CUDA(cudaGetLastError());
}

void launch_pack(const uint8_t *seq, uint64_t seq_base, uint64_t seq_len, uint64_t n_bases, uint32_t *planes,
                 uint64_t t0, uint64_t t1, int *err, cudaStream_t s)
{
    if (t1 <= t0)
        return;
    static_assert(kTileW % 128 == 0 && kTileExt == 32, "pack layout");
    const size_t smem = 2ull * kBufWords * sizeof(uint32_t); // two staged tiles (67.6 KB)
    // grid size and the shared-memory opt-in, once per device
    static int cached_dev = -1, sms = 148, per_sm = 1;
    int dev = 0;
    AH_CUDA(cudaGetDevice(&dev));
    if (dev != cached_dev) {
        AH_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        AH_CUDA(cudaFuncSetAttribute(pack_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        AH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pack_kernel, kPackThreads, smem));
        // one block per tile: blocks end as tiles are done, so kernels that run
        // beside the packing (a run's later stages) get SMs as they free up;
        // AH_PACK_BLOCKS=n keeps n persistent blocks per SM instead (profiling aid)
        const char *e = getenv("AH_PACK_BLOCKS");
        per_sm = (e && atoi(e) > 0) ? std::max(1, std::min(per_sm, atoi(e))) : (1 << 20);
        cached_dev = dev;
    }
    uint64_t blocks = (uint64_t)sms * (uint64_t)(per_sm > 0 ? per_sm : 1);
    // AH_PACK_TILES=n: n tiles per block (the second staged while the first is packed)
    static int tiles_per_block = -1;
    if (tiles_per_block < 0) {
        const char *e = getenv("AH_PACK_TILES");
        tiles_per_block = (e && atoi(e) > 0) ? atoi(e) : 1;
    }
    blocks = std::min<uint64_t>(blocks, (t1 - t0 + tiles_per_block - 1) / tiles_per_block);
    // A block that packs one tile reserves the one staging buffer it uses: six
    // blocks per SM (measured on the large workload: the packing alone at 0.97
    // of the copy peak against 0.84 with two buffers reserved, and a pass 2.4 %
    // shorter; the collection step unchanged).  AH_PACK_SMEM_KB sets the
    // reservation (profiling aid; at least one buffer).
    size_t smem_launch = blocks >= t1 - t0 ? smem / 2 : smem;
    if (const char *e = getenv("AH_PACK_SMEM_KB"))
        smem_launch = std::min(smem, std::max(blocks >= t1 - t0 ? smem / 2 : smem, (size_t)atoi(e) * 1024));
    const int tma_ok = ((reinterpret_cast<uintptr_t>(seq) - seq_base) % 16 == 0) ? 1 : 0;
    pack_kernel<<<(unsigned)blocks, kPackThreads, smem_launch, s>>>(seq, seq_base, seq_len, n_bases, planes, t0, t1,
                                                                    tma_ok, 1u, err);
    AH_CUDA(cudaGetLastError());
}

namespace {

// Contig-wise reversal of the ASCII input (decoy genomes): one block per
// stretch; consecutive threads read consecutive (descending) source bytes.
__global__ void reverse_contigs_kernel(const uint8_t *__restrict__ src, uint8_t *__restrict__ dst,
                                       const RevChunk *__restrict__ chunks)
{
    const RevChunk c = chunks[blockIdx.x];
    for (uint64_t i = threadIdx.x; i < c.len; i += blockDim.x) {
        const uint64_t k = c.start + i;
        dst[k] = src[c.mirror - k];
    }
}

} // namespace

void launch_reverse_contigs(const uint8_t *src, uint8_t *dst, const RevChunk *chunks, uint64_t n_chunks,
                            cudaStream_t s)
{
    if (n_chunks == 0)
        return;
    if (n_chunks > 0x7fffffffull)
        throw Error(AH_ERR_ARG, "reversal: too many stretches");
    reverse_contigs_kernel<<<(unsigned)n_chunks, 256, 0, s>>>(src, dst, chunks);
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
