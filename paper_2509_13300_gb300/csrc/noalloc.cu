// ah_pair_noalloc: amplicon calling that allocates no memory at all.
//
// Some callers cannot call cudaMalloc during a call: an application whose
// own allocator owns all of device memory and forbids side allocations, or a
// latency-bound loop that must stay off the driver's allocator (cudaMalloc
// and cudaFree can take milliseconds and cudaFree synchronises the device).
// This entry point runs the same pairing kernels as ah_pair but keeps every
// piece of scratch (per-site counts and offsets, the prefix-sum temporary,
// the per-pair lengths and windows, the error word and the result count) in
// one file-scope device array of fixed size, so it neither allocates nor
// frees anything, on the device or through any library.  It does wait on its
// stream (it reads the error word and the amplicon count back to the host).
//
// The array is kScratchBytes (about 4.4 MB); every GPU that loads this
// library holds it until the process exits.  Host code cannot use the
// array's name as a device address, so the first call on each device looks
// its address up with cudaGetSymbolAddress (with that device current) and
// caches it for the life of the process: the cache assumes the device's
// primary context is never reset (no cudaDeviceReset in between).  All calls
// share the array: calls that overlap on the GPU (on two streams, or from two
// threads) race and must not be issued.
#include <cub/device/device_scan.cuh>

#include <algorithm>
#include <mutex>

#include "ah_internal.h"

namespace {

constexpr uint64_t kMaxSites = 1u << 18;                 // sites per call
constexpr size_t kCountsBytes = kMaxSites * sizeof(uint64_t);
constexpr size_t kPairsBytes = AH_MAX_PAIRS_PER_SCAN * ((sizeof(ah::PairDev) + 255) / 256 * 256);
constexpr size_t kCubBytes = 64u << 10;                  // prefix-sum temporary
constexpr size_t kFlagBytes = 256;                       // error word + result count
constexpr size_t kScratchBytes = 2 * kCountsBytes + kPairsBytes + kCubBytes + kFlagBytes;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_addr[kMaxDevices] = {};

// Reject records whose pair, primer or strand would index outside the
// per-pair table (the only memory the pairing kernels index with them), and
// lists out of canonical order (pair, contig, pos, primer, strand), which the
// pairing's searches assume.
__global__ void check_records(const ah_site *__restrict__ s, uint64_t n, int n_pairs, int *__restrict__ err)
{
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const ah_site b = s[i];
        bool bad = b.pair >= n_pairs || b.primer > 1 || b.strand > 1;
        if (i > 0) {
            const ah_site a = s[i - 1];
            const unsigned long long ka = ((unsigned long long)a.pair << 32) | a.contig,
                                     kb = ((unsigned long long)b.pair << 32) | b.contig;
            const unsigned long long ta = ((unsigned long long)a.pos << 2) | ((a.primer & 1u) << 1) | (a.strand & 1u),
                                     tb = ((unsigned long long)b.pos << 2) | ((b.primer & 1u) << 1) | (b.strand & 1u);
            bad |= ka > kb || (ka == kb && ta > tb);
        }
        if (bad)
            atomicExch(err, 1);
    }
}

struct Windows {
    int32_t w[AH_MAX_PAIRS_PER_SCAN][4]; // L_fwd, L_rev, min_len, max_len
};

// Write the fields of the per-pair table that the pairing kernels read.
__global__ void set_windows(Windows win, int n_pairs, ah::PairDev *__restrict__ pd)
{
    const int j = threadIdx.x;
    if (j < n_pairs) {
        pd[j].L[0] = win.w[j][0];
        pd[j].L[1] = win.w[j][1];
        pd[j].min_len = win.w[j][2];
        pd[j].max_len = win.w[j][3];
    }
}

bool on_device(const void *p, int dev)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice && a.device == dev) || a.type == cudaMemoryTypeManaged;
}

} // namespace

extern "C" ah_status ah_pair_noalloc(const int32_t *pair_windows, uint32_t n_pairs, const ah_site *sites,
                                     const uint8_t *pass, uint64_t n, ah_amplicon *out, uint64_t cap,
                                     uint64_t *n_out, void *stream)
{
    if (!pair_windows || !n_out || n_pairs < 1 || n_pairs > AH_MAX_PAIRS_PER_SCAN || n > kMaxSites)
        return AH_ERR_ARG;
    *n_out = 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return AH_ERR_CUDA;
    }
    unsigned char *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_addr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return AH_ERR_CUDA;
            }
            g_addr[dev] = (unsigned char *)p;
        }
        base = g_addr[dev];
    }
    for (uint32_t j = 0; j < n_pairs; ++j) { // the windows are checked whatever n is
        const int32_t *w = pair_windows + 4 * j;
        if (w[0] < 1 || w[0] > AH_MAX_PRIMER_LEN || w[1] < 1 || w[1] > AH_MAX_PRIMER_LEN || w[2] < 0 || w[2] > w[3])
            return AH_ERR_ARG;
    }
    if (n == 0)
        return AH_OK;
    if (!sites || !on_device(sites, dev) || (pass && !on_device(pass, dev)) || (cap && (!out || !on_device(out, dev))))
        return AH_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    uint64_t *counts = (uint64_t *)base;
    uint64_t *offs = (uint64_t *)(base + kCountsBytes);
    ah::PairDev *pd = (ah::PairDev *)(base + 2 * kCountsBytes);
    void *cub_temp = base + 2 * kCountsBytes + kPairsBytes;
    int *err = (int *)(base + 2 * kCountsBytes + kPairsBytes + kCubBytes);
    uint64_t *last = (uint64_t *)(err + 2); // [offset of the last site, count of the last site]

    size_t cub_bytes = 0;
    if (cub::DeviceScan::ExclusiveSum(nullptr, cub_bytes, counts, offs, (int64_t)n) != cudaSuccess ||
        cub_bytes > kCubBytes) {
        cudaGetLastError();
        return AH_ERR_CUDA;
    }
    try {
        Windows win;
        for (uint32_t j = 0; j < n_pairs; ++j)
            for (int q = 0; q < 4; ++q)
                win.w[j][q] = pair_windows[4 * j + q];
        set_windows<<<1, 32, 0, st>>>(win, (int)n_pairs, pd);
        AH_CUDA(cudaGetLastError());
        AH_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st)); // the array keeps the last call's contents
        const unsigned blocks = (unsigned)std::min<uint64_t>((n + 255) / 256, 4096);
        check_records<<<blocks, 256, 0, st>>>(sites, n, (int)n_pairs, err);
        AH_CUDA(cudaGetLastError());
        int bad = 0;
        AH_CUDA(cudaMemcpyAsync(&bad, err, sizeof(int), cudaMemcpyDeviceToHost, st));
        AH_CUDA(cudaStreamSynchronize(st));
        if (bad)
            return AH_ERR_ARG;
        ah::launch_pair_count(sites, n, nullptr, pass, pd, counts, st);
        ah::exclusive_scan_u64(cub_temp, cub_bytes, counts, offs, n, st);
        AH_CUDA(cudaMemcpyAsync(&last[0], offs + n - 1, sizeof(uint64_t), cudaMemcpyDeviceToDevice, st));
        AH_CUDA(cudaMemcpyAsync(&last[1], counts + n - 1, sizeof(uint64_t), cudaMemcpyDeviceToDevice, st));
        uint64_t h[2] = {0, 0};
        AH_CUDA(cudaMemcpyAsync(h, last, 2 * sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
        AH_CUDA(cudaStreamSynchronize(st));
        const uint64_t total = h[0] + h[1];
        *n_out = total;
        if (total > cap)
            return AH_ERR_OVERFLOW;
        if (total) {
            ah::launch_pair_write(sites, n, nullptr, pass, pd, offs, out, total, nullptr, 0, st);
            AH_CUDA(cudaStreamSynchronize(st));
        }
    } catch (const ah::Error &e) {
        return e.status;
    }
    return AH_OK;
}
