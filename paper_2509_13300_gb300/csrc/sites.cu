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
// Small-count path: rank sort.  Site keys are distinct in their bits
// [8, end_bit) -- (pair, flat position, primer, strand) names one site -- so
// a key's place in canonical order is the number of keys below it.  A block
// of kRankWarps warps takes 32 * kRankQ keys ("queries", kRankQ per lane);
// each of its warps counts, for every query, the smaller keys in one
// kRankWarps-th of the whole key array staged in shared memory; warp 0 adds
// the partial counts, decodes its keys and writes each record at its rank.
// n^2 compares spread over the whole GPU in one launch: a few microseconds
// for thousands of sites, where a one-block radix sort or a series of
// device-wide sort launches takes tens.
// ---------------------------------------------------------------------------
namespace ah {
namespace {

constexpr int kRankWarps = 8;
constexpr int kRankQ = 2;
constexpr uint32_t kRankStageContigs = 4096; // contig offset tables up to this size are staged in shared memory

template <typename K> struct Vec16;
template <> struct Vec16<uint32_t> {
    using T = uint4;
    static constexpr int V = 4;
    __device__ static void get(const T &x, uint32_t (&e)[4]) { e[0] = x.x; e[1] = x.y; e[2] = x.z; e[3] = x.w; }
};
template <> struct Vec16<uint64_t> {
    using T = ulonglong2;
    static constexpr int V = 2;
    __device__ static void get(const T &x, uint64_t (&e)[2]) { e[0] = x.x; e[1] = x.y; }
};

// K: uint32_t when the sort bits [8, end_bit) fit in 32 bits, else uint64_t.
// Shared memory: the keys (rounded up to 16 bytes), the partial counts, and
// the contig offsets when stage_contigs.
template <typename K>
__global__ void __launch_bounds__(32 * kRankWarps)
    rank_sort_decode_kernel(const uint64_t *__restrict__ keys, uint64_t n_arg, const uint64_t *__restrict__ n_dev,
                            int pbits, const uint64_t *__restrict__ contig_off, uint32_t n_contigs,
                            bool stage_contigs, const uint32_t *__restrict__ contig_genome, ah_site *__restrict__ out,
                            uint64_t *__restrict__ n_out, uint64_t *__restrict__ redo)
{
    using VT = Vec16<K>;
    constexpr int V = VT::V;
    const uint64_t n64 = n_dev ? *n_dev : n_arg;
    if (n64 > n_arg) { // device count above the launch's size: the host redoes this step
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            *n_out = 0;
            atomicOr((unsigned long long *)redo, (unsigned long long)kRedoSites);
        }
        return;
    }
    const uint32_t n = (uint32_t)n64;
    if (n_out && blockIdx.x == 0 && threadIdx.x == 0)
        *n_out = n;
    const uint32_t q0 = blockIdx.x * 32u * kRankQ;
    if (q0 >= n)
        return;
    extern __shared__ __align__(16) unsigned char rank_smem[];
    const uint32_t nv = (n + V - 1) / V;
    K *cand = reinterpret_cast<K *>(rank_smem);
    uint32_t *part = reinterpret_cast<uint32_t *>(rank_smem + (size_t)nv * 16);
    uint64_t *coff = reinterpret_cast<uint64_t *>(rank_smem + (size_t)nv * 16 + kRankWarps * 32 * kRankQ * 4);
    // the block's own queries, full keys, loaded first so their latency overlaps the staging
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint64_t qkey[kRankQ];
#pragma unroll
    for (int j = 0; j < kRankQ; ++j) {
        const uint32_t i = q0 + lane + 32u * j;
        qkey[j] = i < n ? __ldg(keys + i) : 0;
    }
    // stage every key (sort bits only): two keys per 16-byte load, eight loads in flight per thread
    {
        const uint32_t pairs = n / 2; // keys is 16-byte aligned (a scratch allocation)
        const ulonglong2 *k2 = reinterpret_cast<const ulonglong2 *>(keys);
        for (uint32_t b = threadIdx.x; b < pairs; b += 8 * blockDim.x) {
            ulonglong2 x[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const uint32_t p = b + u * blockDim.x;
                x[u] = p < pairs ? __ldg(k2 + p) : make_ulonglong2(~0ull, ~0ull);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const uint32_t p = b + u * blockDim.x;
                if (p < pairs) {
                    cand[2 * p] = (K)(x[u].x >> 8);
                    cand[2 * p + 1] = (K)(x[u].y >> 8);
                }
            }
        }
        for (uint32_t i = 2 * pairs + threadIdx.x; i < nv * V; i += blockDim.x)
            cand[i] = i < n ? (K)(__ldg(keys + i) >> 8) : (K)~(K)0; // odd tail and padding (never below a key)
    }
    if (stage_contigs) { // n_contigs + 1 <= kRankStageContigs: at most 8 vector loads per thread, all in flight
        const uint32_t m = n_contigs + 1, m2 = m / 2;
        const ulonglong2 *c2 = reinterpret_cast<const ulonglong2 *>(contig_off); // 16-byte aligned (checked on the host)
        ulonglong2 x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const uint32_t p = threadIdx.x + u * blockDim.x;
            if (p < m2)
                x[u] = __ldg(c2 + p);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const uint32_t p = threadIdx.x + u * blockDim.x;
            if (p < m2) {
                coff[2 * p] = x[u].x;
                coff[2 * p + 1] = x[u].y;
            }
        }
        if ((m & 1) && threadIdx.x == 0)
            coff[m - 1] = __ldg(contig_off + m - 1);
    }
    __syncthreads();
    K q[kRankQ];
    uint32_t r[kRankQ];
#pragma unroll
    for (int j = 0; j < kRankQ; ++j) {
        q[j] = (K)(qkey[j] >> 8);
        r[j] = 0;
    }
    const uint32_t v0 = (uint32_t)((uint64_t)nv * w / kRankWarps);
    const uint32_t v1 = (uint32_t)((uint64_t)nv * (w + 1) / kRankWarps);
    const typename VT::T *cv = reinterpret_cast<const typename VT::T *>(cand);
#pragma unroll 4
    for (uint32_t v = v0; v < v1; ++v) {
        K e[V];
        VT::get(cv[v], e);
#pragma unroll
        for (int t = 0; t < V; ++t)
#pragma unroll
            for (int j = 0; j < kRankQ; ++j)
                r[j] += e[t] < q[j] ? 1u : 0u;
    }
#pragma unroll
    for (int j = 0; j < kRankQ; ++j)
        part[w * 32 * kRankQ + lane + 32 * j] = r[j];
    __syncthreads();
    if (w != 0)
        return;
    const uint64_t *co = stage_contigs ? coff : contig_off;
#pragma unroll
    for (int j = 0; j < kRankQ; ++j) {
        const uint32_t i = q0 + lane + 32u * j;
        if (i >= n)
            break;
        uint32_t rank = 0;
#pragma unroll
        for (int ww = 0; ww < kRankWarps; ++ww)
            rank += part[ww * 32 * kRankQ + lane + 32 * j];
        const uint64_t key = qkey[j];
        const uint64_t pp = key >> 10;
        const uint64_t P = pp & ((1ull << pbits) - 1);
        uint32_t lo = 0, hi = n_contigs;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (co[mid] <= P)
                lo = mid;
            else
                hi = mid;
        }
        ah_site s;
        s.genome = __ldg(contig_genome + lo);
        s.contig = lo;
        s.pos = (uint32_t)(P - co[lo]);
        s.primer = (uint8_t)((key >> 9) & 1);
        s.strand = (uint8_t)((key >> 8) & 1);
        s.mm = (uint8_t)(key & 0xff);
        s.pair = (uint8_t)(pp >> pbits);
        out[rank] = s;
    }
}

template <typename K>
void run_rank_sort(const uint64_t *keys, uint64_t n, const uint64_t *n_dev, int pbits, const uint64_t *contig_off,
                   uint32_t n_contigs, const uint32_t *contig_genome, ah_site *out, uint64_t *n_out, uint64_t *redo,
                   cudaStream_t s)
{
    // staging reads the offsets with 16-byte loads, 8 per thread of 256
    const bool stage = n_contigs + 1 <= kRankStageContigs && reinterpret_cast<uintptr_t>(contig_off) % 16 == 0;
    const size_t smem = (size_t)((n + Vec16<K>::V - 1) / Vec16<K>::V) * 16 + kRankWarps * 32 * kRankQ * 4 +
                        (stage ? (size_t)(n_contigs + 1) * 8 : 0);
    static int attr_dev = -1; // one instance per key type: opt in to the largest size once per device
    int dev = 0;
    AH_CUDA(cudaGetDevice(&dev));
    if (dev != attr_dev) {
        const size_t most = kSmallSort * sizeof(K) + kRankWarps * 32 * kRankQ * 4 + kRankStageContigs * 8;
        AH_CUDA(cudaFuncSetAttribute(rank_sort_decode_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)most));
        attr_dev = dev;
    }
    const unsigned blocks = (unsigned)((n + 32 * kRankQ - 1) / (32 * kRankQ));
    rank_sort_decode_kernel<K><<<blocks, 32 * kRankWarps, smem, s>>>(keys, n, n_dev, pbits, contig_off, n_contigs,
                                                                      stage, contig_genome, out, n_out, redo);
    AH_CUDA(cudaGetLastError());
}

} // namespace

void launch_rank_sort_decode(const uint64_t *keys, uint64_t n, const uint64_t *n_dev, bool key32, int pbits,
                             const uint64_t *contig_off, uint32_t n_contigs, const uint32_t *contig_genome,
                             ah_site *out, uint64_t *n_out, uint64_t *redo, cudaStream_t s)
{
    if (n == 0 || n > kSmallSort)
        throw Error(AH_ERR_ARG, "rank sort: count outside 1..16384");
    if (reinterpret_cast<uintptr_t>(keys) % 16 != 0)
        throw Error(AH_ERR_ARG, "rank sort: keys not 16-byte aligned");
    if (key32)
        run_rank_sort<uint32_t>(keys, n, n_dev, pbits, contig_off, n_contigs, contig_genome, out, n_out, redo, s);
    else
        run_rank_sort<uint64_t>(keys, n, n_dev, pbits, contig_off, n_contigs, contig_genome, out, n_out, redo, s);
}

} // namespace ah
