// Packer: ASCII genome -> tile-strided one-hot bitplanes (layout in ah_internal.h).
//
// One warp builds 32 consecutive words [j, j + 32) of one tile for all four
// planes.  Lane b loads the 32 ASCII bytes at flat positions
// t * kTileBases + b * kTileW + j .. + 31 (one full 32-byte sector per lane),
// then for each byte q the warp takes four ballots over the lanes: ballot q
// of plane x is exactly word j + q of plane x (bit b = lane b's byte).  Lane
// q keeps those four words and the warp stores 4 x 128 coalesced bytes.
// HBM traffic: 1 byte read per base (+3% for the extension words) and 0.516
// bytes written per base.
#include "ah_internal.h"

namespace ah {
namespace {

constexpr int kGroupsPerTile = kTileWX / 32; // 33 word groups of 32 words

__global__ void __launch_bounds__(256) pack_kernel(const uint8_t *__restrict__ seq, uint64_t seq_base,
                                                   uint64_t seq_len, uint64_t n_bases, uint32_t *__restrict__ planes,
                                                   uint64_t t0, uint64_t t1, int vec_ok)
{
    const int lane = threadIdx.x & 31;
    const uint64_t n_groups = (t1 - t0) * kGroupsPerTile;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    const uint64_t seq_end = seq_base + seq_len; // exclusive flat end of the bytes we hold
    const uint64_t lim = n_bases < seq_end ? n_bases : seq_end;
    for (uint64_t g = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < n_groups; g += warps) {
        const uint64_t t = t0 + g / kGroupsPerTile;
        const int j = (int)(g % kGroupsPerTile) * 32;
        const uint64_t start = t * kTileBases + (uint64_t)lane * kTileW + j; // flat position of byte 0
        uint32_t w[8];
        if (vec_ok && start >= seq_base && start + 32 <= lim) {
            const uint4 *src = reinterpret_cast<const uint4 *>(seq + (start - seq_base));
            uint4 a = __ldg(src), b = __ldg(src + 1);
            w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w;
            w[4] = b.x; w[5] = b.y; w[6] = b.z; w[7] = b.w;
        } else {
#pragma unroll
            for (int q = 0; q < 8; ++q) w[q] = 0;
            for (int q = 0; q < 32; ++q) {
                uint64_t pos = start + q;
                if (pos >= seq_base && pos < lim)
                    w[q >> 2] |= (uint32_t)seq[pos - seq_base] << ((q & 3) * 8);
            }
        }
        uint32_t pa = 0, pc = 0, pg = 0, pt = 0;
#pragma unroll
        for (int q = 0; q < 32; ++q) {
            const uint32_t c = (w[q >> 2] >> ((q & 3) * 8)) & 0xDFu; // upper-case letters
            const uint32_t ba = __ballot_sync(0xffffffffu, c == 'A');
            const uint32_t bc = __ballot_sync(0xffffffffu, c == 'C');
            const uint32_t bg = __ballot_sync(0xffffffffu, c == 'G');
            const uint32_t bt = __ballot_sync(0xffffffffu, c == 'T');
            if (lane == q) {
                pa = ba; pc = bc; pg = bg; pt = bt;
            }
        }
        uint32_t *dst = planes + t * 4 * kTileWX + j + lane;
        dst[0 * kTileWX] = pa;
        dst[1 * kTileWX] = pc;
        dst[2 * kTileWX] = pg;
        dst[3 * kTileWX] = pt;
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
                 uint64_t t0, uint64_t t1, cudaStream_t s)
{
    if (t1 <= t0)
        return;
    const uint64_t n_groups = (t1 - t0) * kGroupsPerTile;
    uint64_t blocks = (n_groups + 7) / 8;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint64_t cap = (uint64_t)sms * 8;
    if (blocks > cap)
        blocks = cap;
    const int vec_ok = ((reinterpret_cast<uintptr_t>(seq) - seq_base) % 16 == 0) ? 1 : 0;
    pack_kernel<<<(unsigned)blocks, 256, 0, s>>>(seq, seq_base, seq_len, n_bases, planes, t0, t1, vec_ok);
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
