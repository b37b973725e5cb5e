// Issue rates of the integer pipes that bound the scan (its roofline
// denominator): LOP3 (the logic pipe) and IADD3 lane-operations per clock per
// SM, measured with the SM's own cycle counter, so the figure does not depend
// on the clock the GPU runs at.  One block of 1024 threads per SM; each thread
// runs eight independent dependency chains (enough to cover the pipes'
// latency), and the block's cycle span between two barriers gives the rate.
#include <algorithm>
#include <vector>

#include "ah_internal.h"

namespace {

constexpr int kRateThreads = 1024;
constexpr int kRateIters = 4096;

template <int OP> __global__ void __launch_bounds__(kRateThreads) rate_kernel(uint32_t seed, uint32_t *sink,
                                                                             unsigned long long *cycles)
{
    uint32_t v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j)
        v[j] = seed * (threadIdx.x + 1) + j;
    const uint32_t a = seed ^ 0x9e3779b9u, b = seed + 0x7f4a7c15u;
    __syncthreads();
    const long long t0 = clock64();
#pragma unroll 4
    for (int it = 0; it < kRateIters; ++it) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (OP == 0)
                asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(v[j]) : "r"(a), "r"(b));
            else
                asm volatile("add.u32 %0, %0, %1;" : "+r"(v[j]) : "r"(a));
        }
    }
    __syncthreads();
    const long long t1 = clock64();
    uint32_t x = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j)
        x ^= v[j];
    if (x == 0x12345678u) // keeps the chains alive
        sink[threadIdx.x] = x;
    if (threadIdx.x == 0)
        cycles[blockIdx.x] = (unsigned long long)(t1 - t0);
}

} // namespace

// lanes[0]: LOP3 lane-operations per clock per SM; lanes[1]: the same for
// 32-bit integer adds.  Runs on the current device (a measurement aid; not
// in the public header).  Returns 0 on success.
extern "C" int ah_debug_pipe_rates(double *lanes)
{
    if (!lanes)
        return 1;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 2;
    uint32_t *sink = nullptr;
    unsigned long long *cyc = nullptr;
    if (cudaMalloc(&sink, kRateThreads * sizeof(uint32_t)) != cudaSuccess)
        return 3;
    if (cudaMalloc(&cyc, sms * sizeof(unsigned long long)) != cudaSuccess) {
        cudaFree(sink);
        return 3;
    }
    std::vector<unsigned long long> h(sms);
    int rc = 0;
    for (int op = 0; op < 2 && rc == 0; ++op) {
        double best = 0;
        for (int rep = 0; rep < 3 && rc == 0; ++rep) {
            if (op == 0)
                rate_kernel<0><<<sms, kRateThreads>>>(0x1234u + rep, sink, cyc);
            else
                rate_kernel<1><<<sms, kRateThreads>>>(0x1234u + rep, sink, cyc);
            if (cudaDeviceSynchronize() != cudaSuccess ||
                cudaMemcpy(h.data(), cyc, sms * sizeof(unsigned long long), cudaMemcpyDeviceToHost) != cudaSuccess) {
                rc = 4;
                break;
            }
            std::sort(h.begin(), h.end());
            const double ops = (double)kRateThreads * kRateIters * 8;
            best = std::max(best, ops / (double)h[h.size() / 2]); // the median SM's span
        }
        lanes[op] = best;
    }
    cudaGetLastError();
    cudaFree(sink);
    cudaFree(cyc);
    return rc;
}
