// Site keys -> canonical order -> site records.
//
// The scan appends 64-bit keys in whatever order warps finish; a radix sort
// over the key bits that carry (pair, flat position, primer, strand) gives
// the canonical order (pair, contig, pos, primer, strand), since contigs are
// laid out in load order.  The decode kernel then finds each key's contig by
// binary search over the contig offsets.
#include <cub/device/device_radix_sort.cuh>

#include "ah_internal.h"

namespace ah {
namespace {

__global__ void decode_keys_kernel(const uint64_t *__restrict__ keys, uint64_t n, int pbits,
                                   const uint64_t *__restrict__ contig_off, uint32_t n_contigs,
                                   const uint32_t *__restrict__ contig_genome, ah_site *__restrict__ out)
{
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t key = keys[i];
        const uint64_t pp = key >> 10;
        const uint64_t P = pp & ((1ull << pbits) - 1);
        const uint32_t pair = (uint32_t)(pp >> pbits);
        uint32_t lo = 0, hi = n_contigs;
        while (hi - lo > 1) {
            uint32_t mid = (lo + hi) >> 1;
            if (contig_off[mid] <= P)
                lo = mid;
            else
                hi = mid;
        }
        ah_site s;
        s.genome = contig_genome[lo];
        s.contig = lo;
        s.pos = (uint32_t)(P - contig_off[lo]);
        s.primer = (uint8_t)((key >> 9) & 1);
        s.strand = (uint8_t)((key >> 8) & 1);
        s.mm = (uint8_t)(key & 0xff);
        s.pair = (uint8_t)pair;
        out[i] = s;
    }
}

__global__ void validate_sites_kernel(const ah_site *__restrict__ sites, uint64_t n, const PairDev *__restrict__ pairs,
                                      int n_pairs, const uint64_t *__restrict__ contig_off, uint32_t n_contigs,
                                      int *__restrict__ err)
{
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const ah_site s = sites[i];
        bool ok = s.pair < n_pairs && s.primer <= 1 && s.strand <= 1 && s.contig < n_contigs;
        if (ok) {
            const uint64_t len = contig_off[s.contig + 1] - contig_off[s.contig];
            ok = (uint64_t)s.pos + (uint64_t)pairs[s.pair].L[s.primer] <= len;
        }
        if (!ok)
            atomicExch(err, kDevBounds);
    }
}

} // namespace

void launch_validate_sites(const ah_site *sites, uint64_t n, const PairDev *pairs_d, int n_pairs,
                           const uint64_t *contig_off, uint32_t n_contigs, int *err, cudaStream_t s)
{
    if (!n)
        return;
    uint64_t blocks = (n + 255) / 256;
    if (blocks > 8192)
        blocks = 8192;
    validate_sites_kernel<<<(unsigned)blocks, 256, 0, s>>>(sites, n, pairs_d, n_pairs, contig_off, n_contigs, err);
    AH_CUDA(cudaGetLastError());
}

size_t sort_keys_temp_bytes(uint64_t n, int end_bit)
{
    size_t bytes = 0;
    AH_CUDA(cub::DeviceRadixSort::SortKeys(nullptr, bytes, (const uint64_t *)nullptr, (uint64_t *)nullptr,
                                           (int64_t)n, 8, end_bit));
    return bytes;
}

void sort_keys(void *temp, size_t temp_bytes, const uint64_t *in, uint64_t *out, uint64_t n, int begin_bit,
               int end_bit, cudaStream_t s)
{
    AH_CUDA(cub::DeviceRadixSort::SortKeys(temp, temp_bytes, in, out, (int64_t)n, begin_bit, end_bit, s));
}

void launch_decode_keys(const uint64_t *keys, uint64_t n, int pbits, const uint64_t *contig_off, uint32_t n_contigs,
                        const uint32_t *contig_genome, ah_site *out, cudaStream_t s)
{
    if (!n)
        return;
    uint64_t blocks = (n + 255) / 256;
    if (blocks > 8192)
        blocks = 8192;
    decode_keys_kernel<<<(unsigned)blocks, 256, 0, s>>>(keys, n, pbits, contig_off, n_contigs, contig_genome, out);
    AH_CUDA(cudaGetLastError());
}

} // namespace ah

// ---------------------------------------------------------------------------
// Small-count fast path: one block of 1024 threads sorts up to kSmallSort
// keys held in registers (16 per thread) with a block-wide radix sort over the
// key bits in use, then writes the decoded site records directly.  A series
// of device-wide sort launches costs more than the whole job at these sizes.
// ---------------------------------------------------------------------------
#include <cub/block/block_radix_sort.cuh>

namespace ah {
namespace {

constexpr int kSortItems = 16;

// One block of THREADS threads sorts up to THREADS * 16 keys (RADIX bits per
// pass over the key bits in use) and decodes them.
template <int THREADS, int RADIX>
__global__ void __launch_bounds__(THREADS) sort_decode_small_kernel(const uint64_t *__restrict__ keys, uint32_t n,
                                                                    int end_bit, int pbits,
                                                                    const uint64_t *__restrict__ contig_off,
                                                                    uint32_t n_contigs,
                                                                    const uint32_t *__restrict__ contig_genome,
                                                                    ah_site *__restrict__ out)
{
    using Sort = cub::BlockRadixSort<uint64_t, THREADS, kSortItems, cub::NullType, RADIX>;
    extern __shared__ __align__(16) unsigned char sort_smem[]; // Sort::TempStorage (> 48 KB: dynamic)
    typename Sort::TempStorage &tmp = *reinterpret_cast<typename Sort::TempStorage *>(sort_smem);
    uint64_t k[kSortItems];
#pragma unroll
    for (int q = 0; q < kSortItems; ++q) { // blocked arrangement: thread t holds keys t*16 .. t*16+15
        const uint32_t i = threadIdx.x * kSortItems + q;
        k[q] = i < n ? keys[i] : ~0ull; // padding sorts last
    }
    Sort(tmp).Sort(k, 8, end_bit > 8 ? end_bit : 9);
    // a thread's 16 keys are consecutive in sorted order: one binary search for
    // the first, then walk forward (positions only grow within a pair)
    uint32_t lo = 0;
    uint64_t prev_pp = ~0ull;
#pragma unroll
    for (int q = 0; q < kSortItems; ++q) {
        const uint32_t i = threadIdx.x * kSortItems + q;
        if (i >= n)
            continue;
        const uint64_t key = k[q];
        const uint64_t pp = key >> 10;
        const uint64_t P = pp & ((1ull << pbits) - 1);
        if (prev_pp == ~0ull || (pp >> pbits) != (prev_pp >> pbits)) {
            lo = 0;
            uint32_t hi = n_contigs;
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (__ldg(contig_off + mid) <= P)
                    lo = mid;
                else
                    hi = mid;
            }
        } else {
            while (lo + 1 < n_contigs && __ldg(contig_off + lo + 1) <= P)
                ++lo;
        }
        prev_pp = pp;
        ah_site s;
        s.genome = contig_genome[lo];
        s.contig = lo;
        s.pos = (uint32_t)(P - contig_off[lo]);
        s.primer = (uint8_t)((key >> 9) & 1);
        s.strand = (uint8_t)((key >> 8) & 1);
        s.mm = (uint8_t)(key & 0xff);
        s.pair = (uint8_t)(pp >> pbits);
        out[i] = s;
    }
}

template <int THREADS, int RADIX>
void run_small_sort(const uint64_t *keys, uint64_t n, int end_bit, int pbits, const uint64_t *contig_off,
                    uint32_t n_contigs, const uint32_t *contig_genome, ah_site *out, cudaStream_t s)
{
    using Sort = cub::BlockRadixSort<uint64_t, THREADS, kSortItems, cub::NullType, RADIX>;
    const size_t smem = sizeof(typename Sort::TempStorage);
    static int attr_dev = -1; // one instance per template: opt in to its shared memory once per device
    int dev = 0;
    AH_CUDA(cudaGetDevice(&dev));
    if (dev != attr_dev) {
        AH_CUDA(cudaFuncSetAttribute(sort_decode_small_kernel<THREADS, RADIX>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr_dev = dev;
    }
    sort_decode_small_kernel<THREADS, RADIX><<<1, THREADS, smem, s>>>(keys, (uint32_t)n, end_bit, pbits, contig_off,
                                                                      n_contigs, contig_genome, out);
    AH_CUDA(cudaGetLastError());
}

} // namespace

bool launch_sort_decode_small(const uint64_t *keys, uint64_t n, int end_bit, int pbits, const uint64_t *contig_off,
                              uint32_t n_contigs, const uint32_t *contig_genome, ah_site *out, cudaStream_t s)
{
    if (n == 0 || n > kSmallSort)
        return false;
    static_assert(1024 * kSortItems == (int)kSmallSort, "the largest instance holds the small sort");
    if (n <= 2048)
        run_small_sort<128, 8>(keys, n, end_bit, pbits, contig_off, n_contigs, contig_genome, out, s);
    else if (n <= 4096)
        run_small_sort<256, 8>(keys, n, end_bit, pbits, contig_off, n_contigs, contig_genome, out, s);
    else if (n <= 8192)
        run_small_sort<512, 6>(keys, n, end_bit, pbits, contig_off, n_contigs, contig_genome, out, s);
    else
        run_small_sort<1024, 6>(keys, n, end_bit, pbits, contig_off, n_contigs, contig_genome, out, s);
    return true;
}

} // namespace ah
