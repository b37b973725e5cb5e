// Amplicon sequence variants and amplitypes (Sec. 3.3, Amplicon Pattern
// Visualization: an amplitype is a genome's combination of amplicon sequence
// variants and their copy numbers; genomes sharing one are grouped).
//
// Variants: each amplicon's sequence (as ah_fetch returns it: RF reverse-
// complemented, N for any non-ACGT letter) is hashed straight from the packed
// planes with two polynomial hashes modulo the Mersenne prime 2^61 - 1 (one
// warp per amplicon, lanes hash contiguous pieces combined by powers of the
// base); amplicons with equal hash pairs are one variant.  Variants, and then
// amplitypes, are numbered by first occurrence: stable radix sorts on the
// hashes keep equal keys in input order, so the head of each run of equal
// keys is its first occurrence, and the ranks of the heads in input order are
// the ids.  Amplitype of a genome: the multiset of (variant, copies), hashed
// as a sum of mixed 64-bit words per (variant, copies) pair (two independent
// sums, order-free), then grouped the same way over the genomes in ascending
// genome order.
#include <cub/device/device_radix_sort.cuh>

#include "ah_internal.h"

namespace ah {
namespace {

constexpr uint64_t kM61 = (1ull << 61) - 1;
constexpr uint64_t kB1 = 0x1d2e3f4a5b6c7d8ull % kM61; // hash bases (any values in [2, 2^61 - 2])
constexpr uint64_t kB2 = 0x0f1e2d3c4b5a697ull % kM61;

__device__ __forceinline__ uint64_t mod61(uint64_t x)
{
    x = (x & kM61) + (x >> 61);
    return x >= kM61 ? x - kM61 : x;
}

// a * b mod 2^61 - 1 for a, b < 2^61: the 122-bit product folded at bit 61
__device__ __forceinline__ uint64_t mulmod61(uint64_t a, uint64_t b)
{
    const uint64_t lo = a * b, hi = __umul64hi(a, b);
    return mod61((lo & kM61) + (lo >> 61) + (hi << 3));
}

__device__ uint64_t powmod61(uint64_t b, uint64_t e)
{
    uint64_t r = 1;
    while (e) {
        if (e & 1)
            r = mulmod61(r, b);
        b = mulmod61(b, b);
        e >>= 1;
    }
    return r;
}

// 64-bit finaliser of the SplitMix generator (Steele, Lea and Flood, 2014)
__device__ __forceinline__ uint64_t mix64(uint64_t x)
{
    x ^= x >> 30;
    x *= 0xbf58476d1ce4e5b9ull;
    x ^= x >> 27;
    x *= 0x94d049bb133111ebull;
    x ^= x >> 31;
    return x;
}

__device__ __forceinline__ int plane_code(const uint32_t *__restrict__ planes, uint64_t P)
{
    const uint64_t t = P / kTileBases, r = P % kTileBases;
    const int b = (int)(r / kTileW), j = (int)(r % kTileW);
    const uint32_t *w = planes + t * 4 * kTileWX + j;
    int code = -1;
#pragma unroll
    for (int x = 0; x < 4; ++x)
        if ((__ldg(w + x * kTileWX) >> b) & 1u)
            code = x;
    return code;
}

// One warp per amplicon: the two hashes of its sequence (letters 1..5 = A C G T N).
__global__ void amp_hash_kernel(const ah_amplicon *__restrict__ a, uint64_t n, const uint32_t *__restrict__ planes,
                                const uint64_t *__restrict__ contig_off, uint64_t *__restrict__ h1,
                                uint64_t *__restrict__ h2)
{
    const int lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x / 32);
    for (uint64_t i = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; i < n; i += warps) {
        const ah_amplicon am = a[i];
        const uint64_t len = am.end - am.start, base = contig_off[am.contig] + am.start;
        const bool rc = am.orient == 1;
        const uint64_t piece = (len + 31) / 32, l0 = min(len, lane * piece), l1 = min(len, l0 + piece);
        uint64_t s1 = 0, s2 = 0;
        for (uint64_t q = l0; q < l1; ++q) {
            int c = plane_code(planes, base + (rc ? len - 1 - q : q));
            if (c >= 0 && rc)
                c = 3 - c;
            const uint64_t v = c < 0 ? 5 : (uint64_t)c + 1;
            s1 = mod61(mulmod61(s1, kB1) + v);
            s2 = mod61(mulmod61(s2, kB2) + v);
        }
        // piece hash times base^(letters after the piece), summed over the warp
        s1 = mulmod61(s1, powmod61(kB1, len - l1));
        s2 = mulmod61(s2, powmod61(kB2, len - l1));
        for (int d = 16; d >= 1; d >>= 1) {
            s1 = mod61(s1 + __shfl_xor_sync(0xffffffffu, s1, d));
            s2 = mod61(s2 + __shfl_xor_sync(0xffffffffu, s2, d));
        }
        if (lane == 0) {
            h1[i] = s1;
            h2[i] = s2 ^ (len << 61); // the length's low three bits in the free top bits
        }
    }
}

__global__ void iota_kernel(uint32_t *__restrict__ v, uint64_t n)
{
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        v[i] = (uint32_t)i;
}

__global__ void gather_kernel(const uint64_t *__restrict__ src, const uint32_t *__restrict__ idx, uint64_t n,
                              uint64_t *__restrict__ dst)
{
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (uint64_t)gridDim.x * blockDim.x)
        dst[k] = src[idx[k]];
}

// head[k] = 1 where the sorted key pair changes (k = 0 included)
__global__ void heads_kernel(const uint64_t *__restrict__ a, const uint64_t *__restrict__ b, uint64_t n,
                             uint64_t *__restrict__ head)
{
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (uint64_t)gridDim.x * blockDim.x)
        head[k] = (k == 0 || a[k] != a[k - 1] || (b && b[k] != b[k - 1])) ? 1 : 0;
}

// at each run head: mark the run's first element (in input order) as a first occurrence
__global__ void firsts_kernel(const uint64_t *__restrict__ head, const uint32_t *__restrict__ idx, uint64_t n,
                              uint64_t *__restrict__ is_first)
{
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (uint64_t)gridDim.x * blockDim.x)
        if (head[k])
            is_first[idx[k]] = 1;
}

// id of element idx[k] = first-occurrence rank of its run's head; runs are
// scanned from the sorted heads: run_of[k] = (inclusive count of heads) - 1
__global__ void assign_kernel(const uint64_t *__restrict__ head_excl, const uint64_t *__restrict__ head,
                              const uint32_t *__restrict__ idx, const uint64_t *__restrict__ rank, uint64_t n,
                              uint32_t *__restrict__ run_head_pos, uint32_t *__restrict__ id_out)
{
    // pass 1 (this kernel with id_out == nullptr): position of every run's head
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t run = head_excl[k] + head[k] - 1;
        if (!id_out) {
            if (head[k])
                run_head_pos[run] = (uint32_t)k;
        } else {
            id_out[idx[k]] = (uint32_t)rank[idx[run_head_pos[run]]];
        }
    }
}

// per (genome, variant) run of the sorted keys: copies, and the genome's sums
__global__ void genome_sums_kernel(const uint64_t *__restrict__ keys, const uint64_t *__restrict__ head,
                                   const uint64_t *__restrict__ head_excl, const uint32_t *__restrict__ run_head_pos,
                                   uint64_t n, const uint64_t *__restrict__ n_runs_dev, unsigned long long *__restrict__ g1,
                                   unsigned long long *__restrict__ g2, unsigned int *__restrict__ gamp,
                                   unsigned int *__restrict__ gvar)
{
    const uint64_t n_runs = *n_runs_dev;
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (uint64_t)gridDim.x * blockDim.x) {
        if (!head[k])
            continue;
        const uint64_t run = head_excl[k];
        const uint64_t end = run + 1 < n_runs ? run_head_pos[run + 1] : n;
        const uint64_t copies = end - k;
        const uint32_t g = (uint32_t)(keys[k] >> 32);
        const uint64_t v = keys[k] & 0xffffffffull;
        atomicAdd(g1 + g, (unsigned long long)mix64((v << 32 | copies) * 2 + 1));
        atomicAdd(g2 + g, (unsigned long long)mix64((v << 32 | copies) ^ 0x9e3779b97f4a7c15ull));
        atomicAdd(gamp + g, (unsigned int)copies);
        atomicAdd(gvar + g, 1u);
    }
}

__global__ void genome_flags_kernel(const unsigned int *__restrict__ gamp, uint64_t n, uint64_t *__restrict__ has)
{
    for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (uint64_t)gridDim.x * blockDim.x)
        has[g] = gamp[g] ? 1 : 0;
}

// compact the genomes with amplicons (ascending id) and their hash sums
__global__ void genome_compact_kernel(const uint64_t *__restrict__ has, const uint64_t *__restrict__ pos, uint64_t n,
                                      const unsigned long long *__restrict__ g1, const unsigned long long *__restrict__ g2,
                                      uint32_t *__restrict__ gid, uint64_t *__restrict__ k1, uint64_t *__restrict__ k2)
{
    for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (uint64_t)gridDim.x * blockDim.x)
        if (has[g]) {
            gid[pos[g]] = (uint32_t)g;
            k1[pos[g]] = g1[g];
            k2[pos[g]] = g2[g];
        }
}

__global__ void rows_kernel(const uint32_t *__restrict__ gid, const uint32_t *__restrict__ type, uint64_t m,
                            const unsigned int *__restrict__ gamp, const unsigned int *__restrict__ gvar,
                            ah_genome_amplitype *__restrict__ rows)
{
    for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < m; r += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t g = gid[r];
        rows[r] = {g, type[r], gamp[g], gvar[g]};
    }
}

__global__ void genome_key_kernel(const ah_amplicon *__restrict__ a, const uint32_t *__restrict__ variant, uint64_t n,
                                  const uint32_t *__restrict__ contig_genome, uint64_t *__restrict__ keys,
                                  int *__restrict__ err)
{
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const ah_amplicon am = a[i]; // contig already checked
        const uint32_t g = contig_genome[am.contig];
        if (am.genome != g || am.orient > 3)
            atomicExch(err, kDevBounds);
        keys[i] = (uint64_t)g << 32 | variant[i];
    }
}

unsigned grid(uint64_t n, int threads = 256)
{
    uint64_t b = (n + threads - 1) / threads;
    return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(b, 8192));
}

} // namespace

// Stable sort of idx (initially 0..n-1) by (ka, kb): LSD over kb then ka.
// Scratch: 2n u64 keys, n u32 values, CUB temporary storage.
void AmpliTypeScratch::sort_by(const uint64_t *ka, const uint64_t *kb, uint64_t n, cudaStream_t s)
{
    keys_b_valid = kb != nullptr;
    iota_kernel<<<grid(n), 256, 0, s>>>(idx, n);
    AH_CUDA(cudaGetLastError());
    size_t tb = temp_bytes;
    if (kb) {
        AH_CUDA(cub::DeviceRadixSort::SortPairs(temp, tb, kb, keys_b, idx, idx_b, (int64_t)n, 0, 64, s));
        gather_kernel<<<grid(n), 256, 0, s>>>(ka, idx_b, n, keys_a);
        AH_CUDA(cudaGetLastError());
        tb = temp_bytes;
        AH_CUDA(cub::DeviceRadixSort::SortPairs(temp, tb, keys_a, keys_s, idx_b, idx, (int64_t)n, 0, 64, s));
        gather_kernel<<<grid(n), 256, 0, s>>>(kb, idx, n, keys_b);
        AH_CUDA(cudaGetLastError());
    } else {
        AH_CUDA(cub::DeviceRadixSort::SortPairs(temp, tb, ka, keys_s, idx, idx_b, (int64_t)n, 0, 64, s));
        AH_CUDA(cudaMemcpyAsync(idx, idx_b, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    }
}

size_t AmpliTypeScratch::cub_bytes(uint64_t n)
{
    size_t b = 0;
    AH_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, b, (const uint64_t *)nullptr, (uint64_t *)nullptr,
                                            (const uint32_t *)nullptr, (uint32_t *)nullptr, (int64_t)n, 0, 64));
    return b;
}

// Runs of equal keys after sort_by: heads, their positions and (device)
// count; with id_out, every element's first-occurrence id of its run.
void AmpliTypeScratch::ids(uint64_t n, uint32_t *id_out, uint64_t *n_runs_dev, cudaStream_t s)
{
    heads_kernel<<<grid(n), 256, 0, s>>>(keys_s, keys_b_valid ? keys_b : nullptr, n, head);
    AH_CUDA(cudaGetLastError());
    exclusive_scan_u64(scan_temp, scan_bytes, head, head_excl, n, s);
    assign_kernel<<<grid(n), 256, 0, s>>>(head_excl, head, idx, rank, n, run_pos, nullptr);
    AH_CUDA(cudaGetLastError());
    launch_total(head_excl, head, n, nullptr, 0, n_runs_dev, 0, nullptr, nullptr, 0, s);
    if (!id_out)
        return;
    AH_CUDA(cudaMemsetAsync(is_first, 0, n * sizeof(uint64_t), s));
    firsts_kernel<<<grid(n), 256, 0, s>>>(head, idx, n, is_first);
    AH_CUDA(cudaGetLastError());
    exclusive_scan_u64(scan_temp, scan_bytes, is_first, rank, n, s);
    assign_kernel<<<grid(n), 256, 0, s>>>(head_excl, head, idx, rank, n, run_pos, id_out);
    AH_CUDA(cudaGetLastError());
}

void launch_amp_hash(const ah_amplicon *a, uint64_t n, const uint32_t *planes, const uint64_t *contig_off,
                     uint64_t *h1, uint64_t *h2, cudaStream_t s)
{
    if (!n)
        return;
    amp_hash_kernel<<<grid(n * 32, 256), 256, 0, s>>>(a, n, planes, contig_off, h1, h2);
    AH_CUDA(cudaGetLastError());
}

void launch_genome_key(const ah_amplicon *a, const uint32_t *variant, uint64_t n, const uint32_t *contig_genome,
                       uint64_t *keys, int *err, cudaStream_t s)
{
    genome_key_kernel<<<grid(n), 256, 0, s>>>(a, variant, n, contig_genome, keys, err);
    AH_CUDA(cudaGetLastError());
}

void AmpliTypeScratch::genome_sums(uint64_t n, const uint64_t *n_runs_dev, unsigned long long *g1,
                                   unsigned long long *g2, unsigned int *gamp, unsigned int *gvar, cudaStream_t s)
{
    genome_sums_kernel<<<grid(n), 256, 0, s>>>(keys_s, head, head_excl, run_pos, n, n_runs_dev, g1, g2, gamp, gvar);
    AH_CUDA(cudaGetLastError());
}

void launch_genome_compact(const unsigned int *gamp, uint64_t n_ids, uint64_t *has, uint64_t *pos, void *scan_temp,
                           size_t scan_bytes, const unsigned long long *g1, const unsigned long long *g2, uint32_t *gid,
                           uint64_t *k1, uint64_t *k2, uint64_t *n_out_dev, cudaStream_t s)
{
    genome_flags_kernel<<<grid(n_ids), 256, 0, s>>>(gamp, n_ids, has);
    AH_CUDA(cudaGetLastError());
    exclusive_scan_u64(scan_temp, scan_bytes, has, pos, n_ids, s);
    genome_compact_kernel<<<grid(n_ids), 256, 0, s>>>(has, pos, n_ids, g1, g2, gid, k1, k2);
    AH_CUDA(cudaGetLastError());
    launch_total(pos, has, n_ids, nullptr, 0, n_out_dev, 0, nullptr, nullptr, 0, s);
}

void launch_amplitype_rows(const uint32_t *gid, const uint32_t *type, uint64_t m, const unsigned int *gamp,
                           const unsigned int *gvar, ah_genome_amplitype *rows, cudaStream_t s)
{
    if (!m)
        return;
    rows_kernel<<<grid(m), 256, 0, s>>>(gid, type, m, gamp, gvar, rows);
    AH_CUDA(cudaGetLastError());
}

} // namespace ah
