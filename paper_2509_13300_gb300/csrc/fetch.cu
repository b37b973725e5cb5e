// Amplicon sequences (Sec. 2.1, Visualization: the main output is a FASTA of
// amplicon sequences).  Decoded from the packed planes: upper case, 'N' for
// any position with no base plane set; RF amplicons reverse-complemented so
// they read from the forward primer.  One block per amplicon.
#include "ah_internal.h"

namespace ah {
namespace {

__global__ void fetch_len_kernel(const ah_amplicon *__restrict__ a, uint64_t n_arg, const uint64_t *__restrict__ n_dev,
                                 const uint64_t *__restrict__ contig_off, uint32_t n_contigs,
                                 uint64_t *__restrict__ len, int *__restrict__ err)
{
    const uint64_t n = dev_count(n_arg, n_dev);
    if (n_dev && blockIdx.x == 0 && threadIdx.x == 0)
        len[n] = 0; // closing entry of the offsets scan
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const ah_amplicon am = a[i];
        bool ok = am.contig < n_contigs && am.start <= am.end;
        if (ok)
            ok = (uint64_t)am.end <= contig_off[am.contig + 1] - contig_off[am.contig];
        if (!ok)
            atomicExch(err, kDevBounds);
        len[i] = ok ? (uint64_t)(am.end - am.start) : 0;
    }
}

// One block per amplicon: consecutive threads decode consecutive positions,
// which sit in consecutive words of a plane row, so the loads coalesce.
__global__ void __launch_bounds__(256) fetch_kernel(const ah_amplicon *__restrict__ a, uint64_t n_arg,
                                                    const uint64_t *__restrict__ n_dev,
                                                    const uint64_t *__restrict__ offsets,
                                                    const uint32_t *__restrict__ planes,
                                                    const uint64_t *__restrict__ contig_off, char *__restrict__ out,
                                                    const uint64_t *__restrict__ skip, uint64_t skip_bit)
{
    if (skip && (*skip & skip_bit))
        return;
    const uint64_t n = dev_count(n_arg, n_dev);
    for (uint64_t i = blockIdx.x; i < n; i += gridDim.x) {
        const uint64_t len = offsets[i + 1] - offsets[i];
        if (len == 0)
            continue;
        const ah_amplicon am = a[i];
        const uint64_t base = contig_off[am.contig] + am.start;
        const bool rc = am.orient == 1;
        char *o = out + offsets[i];
        for (uint64_t q = threadIdx.x; q < len; q += blockDim.x) {
            const uint64_t P = base + (rc ? len - 1 - q : q);
            const uint64_t t = P / kTileBases, r = P % kTileBases;
            const int b = (int)(r / kTileW), j = (int)(r % kTileW);
            const uint32_t *w = planes + t * 4 * kTileWX + j;
            int code = -1;
#pragma unroll
            for (int x = 0; x < 4; ++x)
                if ((__ldg(w + x * kTileWX) >> b) & 1u)
                    code = x;
            if (code >= 0 && rc)
                code = 3 - code;
            o[q] = code < 0 ? 'N' : "ACGT"[code];
        }
    }
}

} // namespace

void launch_fetch_lengths(const ah_amplicon *a, uint64_t n, const uint64_t *n_dev, const uint64_t *contig_off,
                          uint32_t n_contigs, uint64_t *len, int *err, cudaStream_t s)
{
    if (!n)
        return;
    uint64_t blocks = (n + 255) / 256;
    if (blocks > 1024)
        blocks = 1024;
    fetch_len_kernel<<<(unsigned)blocks, 256, 0, s>>>(a, n, n_dev, contig_off, n_contigs, len, err);
    AH_CUDA(cudaGetLastError());
}

void launch_fetch(const ah_amplicon *a, uint64_t n, const uint64_t *n_dev, const uint64_t *offsets,
                  const uint32_t *planes, const uint64_t *contig_off, char *out, const uint64_t *skip,
                  uint64_t skip_bit, cudaStream_t s)
{
    if (!n)
        return;
    // blocks loop over amplicons; a device-count launch is sized for its largest
    // count, so keep the grid to a few blocks per SM
    const uint64_t most = n_dev ? 2048 : 8192;
    const uint64_t blocks = n < most ? n : most;
    fetch_kernel<<<(unsigned)blocks, 256, 0, s>>>(a, n, n_dev, offsets, planes, contig_off, out, skip, skip_bit);
    AH_CUDA(cudaGetLastError());
}

} // namespace ah
