// Amplicon calling (Sec. 2.1): pair '+' sites with '-' sites of the same pair
// and contig inside the length window, labelled FR/RF/FF/RR (Sec. 2.1,
// Amplicon analysis, item 1).
//
// Sites arrive in canonical order, so all sites at one (pair, contig, pos)
// are adjacent (at most F+, F-, R+, R-).  One thread owns each "start group"
// -- the '+' sites at one position (F+ and/or R+) -- and walks the sorted
// sites after it whose position can close an amplicon: right sites t with
// t >= s and t + L_Y - s in [min_len, max_len].  A count pass, an exclusive
// scan and a write pass place every group's amplicons at fixed offsets; the
// write pass merges the up-to-four (left primer, right primer) streams of its
// group by (end, orient), each of which is already sorted by end, so the
// output comes out in canonical order with no global sort.
#include <cub/device/device_scan.cuh>

#include "ah_internal.h"

namespace ah {
namespace {

__device__ __forceinline__ bool same_group(const ah_site &a, const ah_site &b)
{
    return a.pair == b.pair && a.contig == b.contig && a.pos == b.pos;
}

__device__ __forceinline__ bool site_less(const ah_site &m, uint32_t pair, uint32_t contig, uint64_t t)
{
    return (m.pair < pair) || (m.pair == pair && (m.contig < contig || (m.contig == contig && m.pos < t)));
}

// First index in [lo, n) whose (pair, contig, pos) >= (pair, contig, t), by
// galloping from lo: probes lo, lo+1, lo+3, lo+7, ... then a binary search in
// the last gap.  Candidates usually sit right after the group, so this takes
// one or two dependent loads where a plain binary search over all sites takes
// log2(n).
__device__ uint64_t lower_bound_pos(const ah_site *__restrict__ s, uint64_t lo, uint64_t n, uint32_t pair,
                                    uint32_t contig, uint64_t t)
{
    uint64_t step = 1, hi = lo;
    while (hi < n && site_less(s[hi], pair, contig, t)) {
        lo = hi + 1;
        hi = lo + step - 1;
        step <<= 1;
    }
    if (hi > n)
        hi = n;
    while (lo < hi) { // s[lo-1] is less (or lo is the start), s[hi] is not (or hi == n)
        const uint64_t mid = (lo + hi) >> 1;
        if (site_less(s[mid], pair, contig, t))
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

struct Group {
    int nl;          // number of passing left sites (0..2)
    uint64_t li[2];  // their indices
    int lx[2];       // their primers
    uint64_t first;  // first candidate index
    uint64_t tmax;   // last candidate position
    bool valid;
};

__device__ Group make_group(const ah_site *__restrict__ s, uint64_t n, const uint8_t *__restrict__ pass,
                            const PairDev *__restrict__ pairs, uint64_t a)
{
    Group g;
    g.valid = false;
    g.nl = 0;
    // the site and its three neighbours either side, as one batch of independent loads
    ah_site nb[7];
#pragma unroll
    for (int d = -3; d <= 3; ++d) {
        const int64_t idx = (int64_t)a + d;
        if (idx >= 0 && (uint64_t)idx < n)
            nb[d + 3] = s[idx];
        else
            nb[d + 3].pair = 0xff; // no site: never in a group
    }
    const ah_site sa = nb[3];
    if (sa.strand != 0)
        return g;
    uint64_t g0 = a; // first site of this (pair, contig, pos) group
#pragma unroll
    for (int d = 1; d <= 3; ++d) {
        const ah_site &p = nb[3 - d];
        if (p.pair == 0xff || !same_group(p, sa))
            break;
        if (p.strand == 0)
            return g; // an earlier '+' site leads this group
        g0 = a - d;
    }
#pragma unroll
    for (int d = 0; d <= 3; ++d) {
        const ah_site &q = nb[3 + d];
        if (q.pair == 0xff || !same_group(q, sa))
            break;
        if (q.strand == 0 && (!pass || pass[a + d])) {
            g.li[g.nl] = a + d;
            g.lx[g.nl] = q.primer;
            ++g.nl;
        }
    }
    if (g.nl == 0)
        return g;
    const PairDev &pd = pairs[sa.pair];
    const int Lmin = min(pd.L[0], pd.L[1]), Lmax = max(pd.L[0], pd.L[1]);
    const int64_t lo = max((int64_t)0, (int64_t)pd.min_len - Lmax);
    const int64_t hi = (int64_t)pd.max_len - Lmin;
    if (hi < lo)
        return g;
    g.first = lower_bound_pos(s, g0, n, sa.pair, sa.contig, (uint64_t)sa.pos + (uint64_t)lo);
    g.tmax = (uint64_t)sa.pos + (uint64_t)hi;
    g.valid = true;
    return g;
}

__device__ __forceinline__ bool in_window(const PairDev &pd, uint32_t s_pos, const ah_site &r, uint32_t *end)
{
    const int64_t e = (int64_t)r.pos + pd.L[r.primer];
    const int64_t len = e - (int64_t)s_pos;
    *end = (uint32_t)e;
    return r.pos >= s_pos && len >= pd.min_len && len <= pd.max_len;
}

__global__ void pair_count_kernel(const ah_site *__restrict__ s, uint64_t n_arg, const uint64_t *__restrict__ n_dev,
                                  const uint8_t *__restrict__ pass, const PairDev *__restrict__ pairs,
                                  uint64_t *__restrict__ counts)
{
    const uint64_t n = dev_count(n_arg, n_dev);
    for (uint64_t a = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; a < n; a += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t cnt = 0;
        const Group g = make_group(s, n, pass, pairs, a);
        if (g.valid) {
            const ah_site sa = s[a];
            const PairDev &pd = pairs[sa.pair];
            for (uint64_t b = g.first; b < n; ++b) {
                const ah_site r = s[b];
                if (r.pair != sa.pair || r.contig != sa.contig || r.pos > g.tmax)
                    break;
                if (r.strand != 1 || (pass && !pass[b]))
                    continue;
                uint32_t end;
                if (in_window(pd, sa.pos, r, &end))
                    cnt += g.nl;
            }
        }
        counts[a] = cnt;
    }
}

__device__ __forceinline__ int orient_of(int x, int y) { return (x == 0 && y == 1) ? 0 : (x == 1 && y == 0) ? 1 : (x == 0 ? 2 : 3); }

__global__ void pair_write_kernel(const ah_site *__restrict__ s, uint64_t n_arg, const uint64_t *__restrict__ n_dev,
                                  const uint8_t *__restrict__ pass, const PairDev *__restrict__ pairs,
                                  const uint64_t *__restrict__ offsets, ah_amplicon *__restrict__ out, uint64_t cap,
                                  const uint64_t *__restrict__ skip, uint64_t skip_bit)
{
    if (skip && (*skip & skip_bit))
        return;
    const uint64_t n = dev_count(n_arg, n_dev);
    for (uint64_t a = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; a < n; a += (uint64_t)gridDim.x * blockDim.x) {
        const Group g = make_group(s, n, pass, pairs, a);
        if (!g.valid)
            continue;
        const ah_site sa = s[a];
        const PairDev &pd = pairs[sa.pair];
        // streams: (left index li, right primer y); cursor = next candidate index
        uint64_t cur[4];
        const int ns = g.nl * 2;
        auto advance = [&](int st, uint64_t from) -> uint64_t {
            const int y = st & 1;
            for (uint64_t b = from; b < n; ++b) {
                const ah_site r = s[b];
                if (r.pair != sa.pair || r.contig != sa.contig || r.pos > g.tmax)
                    return n;
                if (r.strand != 1 || r.primer != y || (pass && !pass[b]))
                    continue;
                uint32_t end;
                if (in_window(pd, sa.pos, r, &end))
                    return b;
            }
            return n;
        };
        for (int st = 0; st < ns; ++st)
            cur[st] = advance(st, g.first);
        uint64_t o = offsets[a];
        for (;;) {
            int best = -1;
            uint32_t bend = 0;
            int bor = 0;
            for (int st = 0; st < ns; ++st) {
                if (cur[st] >= n)
                    continue;
                const ah_site r = s[cur[st]];
                const uint32_t end = r.pos + pd.L[r.primer];
                const int orr = orient_of(g.lx[st >> 1], r.primer);
                if (best < 0 || end < bend || (end == bend && orr < bor)) {
                    best = st;
                    bend = end;
                    bor = orr;
                }
            }
            if (best < 0)
                break;
            if (o < cap) {
                ah_amplicon am;
                am.genome = sa.genome;
                am.contig = sa.contig;
                am.start = sa.pos;
                am.end = bend;
                am.left = (uint32_t)g.li[best >> 1];
                am.right = (uint32_t)cur[best];
                am.orient = (uint8_t)bor;
                am.pair = sa.pair;
                am.pad0 = am.pad1 = 0;
                out[o] = am;
            }
            ++o;
            cur[best] = advance(best, cur[best] + 1);
        }
    }
}

__global__ void total_kernel(const uint64_t *__restrict__ offs, const uint64_t *__restrict__ counts, uint64_t n_arg,
                             const uint64_t *__restrict__ n_dev, uint64_t add, uint64_t *__restrict__ out,
                             uint64_t cap, uint64_t *__restrict__ eff, uint64_t *__restrict__ redo, uint64_t redo_bit)
{
    const uint64_t n = n_dev ? min(*n_dev + add, n_arg) : n_arg;
    const uint64_t t = n ? offs[n - 1] + counts[n - 1] : 0;
    *out = t;
    if (eff) {
        *eff = t <= cap ? t : 0;
        if (t > cap)
            atomicOr((unsigned long long *)redo, (unsigned long long)redo_bit);
    }
}

// One-block exclusive scan of m u64 values (m = n, or min(*n_dev + add, n)),
// 4096 at a time: coalesced loads (four per thread in flight) staged through
// shared memory, each thread scans four consecutive values, warp shuffles and
// one shared pass scan the 1024 thread sums, and the results leave through
// shared memory as coalesced stores.  With tot it also writes the sum of all
// m values; with eff, *eff = that sum if it is at most cap, else 0 with
// redo_bit set in *redo.
__global__ void __launch_bounds__(1024) scan_small_kernel(const uint64_t *__restrict__ in, uint64_t *__restrict__ out,
                                                          uint32_t n_arg, const uint64_t *__restrict__ n_dev,
                                                          uint64_t add, uint64_t *__restrict__ tot, uint64_t cap,
                                                          uint64_t *__restrict__ eff, uint64_t *__restrict__ redo,
                                                          uint64_t redo_bit)
{
    __shared__ uint64_t buf[4096];
    __shared__ uint64_t wsum[32];
    const uint32_t n = n_dev ? (uint32_t)min(*n_dev + add, (uint64_t)n_arg) : n_arg;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint64_t carry = 0;
    for (uint32_t base = 0; base < n; base += 4096) {
        uint64_t v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint32_t i = base + tid + 1024u * u;
            v[u] = i < n ? in[i] : 0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            buf[tid + 1024 * u] = v[u];
        __syncthreads();
        const uint64_t x0 = buf[4 * tid], x1 = buf[4 * tid + 1], x2 = buf[4 * tid + 2], x3 = buf[4 * tid + 3];
        const uint64_t sum = x0 + x1 + x2 + x3;
        uint64_t incl = sum;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint64_t y = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d)
                incl += y;
        }
        if (lane == 31)
            wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            uint64_t w = wsum[lane];
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint64_t y = __shfl_up_sync(0xffffffffu, w, d);
                if (lane >= d)
                    w += y;
            }
            wsum[lane] = w;
        }
        __syncthreads();
        const uint64_t ex = carry + (warp ? wsum[warp - 1] : 0) + incl - sum;
        buf[4 * tid] = ex;
        buf[4 * tid + 1] = ex + x0;
        buf[4 * tid + 2] = ex + x0 + x1;
        buf[4 * tid + 3] = ex + x0 + x1 + x2;
        carry += wsum[31];
        __syncthreads();
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint32_t i = base + tid + 1024u * u;
            if (i < n)
                out[i] = buf[tid + 1024 * u];
        }
        __syncthreads(); // buf and wsum are rewritten by the next chunk
    }
    if (tid == 0 && tot) {
        *tot = carry;
        if (eff) {
            *eff = carry <= cap ? carry : 0;
            if (carry > cap)
                atomicOr((unsigned long long *)redo, (unsigned long long)redo_bit);
        }
    }
}

unsigned grid_for(uint64_t n, int threads)
{
    uint64_t b = (n + threads - 1) / threads;
    if (b > 16384)
        b = 16384;
    if (b == 0)
        b = 1;
    return (unsigned)b;
}

} // namespace

void launch_pair_count(const ah_site *sites, uint64_t n, const uint64_t *n_dev, const uint8_t *pass,
                       const PairDev *pairs_d, uint64_t *counts, cudaStream_t s)
{
    if (!n)
        return;
    pair_count_kernel<<<grid_for(n, 128), 128, 0, s>>>(sites, n, n_dev, pass, pairs_d, counts);
    AH_CUDA(cudaGetLastError());
}

void launch_total(const uint64_t *offs, const uint64_t *counts, uint64_t n, const uint64_t *n_dev, uint64_t add,
                  uint64_t *out, uint64_t cap, uint64_t *eff, uint64_t *redo, uint64_t redo_bit, cudaStream_t s)
{
    total_kernel<<<1, 1, 0, s>>>(offs, counts, n, n_dev, add, out, cap, eff, redo, redo_bit);
    AH_CUDA(cudaGetLastError());
}

size_t scan_u64_temp_bytes(uint64_t n)
{
    size_t bytes = 0;
    AH_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, bytes, (const uint64_t *)nullptr, (uint64_t *)nullptr, (int64_t)n));
    return bytes;
}

void exclusive_scan_u64(void *temp, size_t temp_bytes, const uint64_t *in, uint64_t *out, uint64_t n, cudaStream_t s)
{
    if (n == 0)
        return;
    if (n <= kSmallScan) {
        scan_small_kernel<<<1, 1024, 0, s>>>(in, out, (uint32_t)n, nullptr, 0, nullptr, 0, nullptr, nullptr, 0);
        AH_CUDA(cudaGetLastError());
        return;
    }
    AH_CUDA(cub::DeviceScan::ExclusiveSum(temp, temp_bytes, in, out, (int64_t)n, s));
}

void exclusive_scan_u64_dev(const uint64_t *in, uint64_t *out, uint64_t n, const uint64_t *n_dev, uint64_t add,
                            uint64_t *tot, uint64_t cap, uint64_t *eff, uint64_t *redo, uint64_t redo_bit,
                            cudaStream_t s)
{
    if (n == 0 || n > kSmallScan)
        throw Error(AH_ERR_ARG, "device-count scan: size outside 1..65536");
    scan_small_kernel<<<1, 1024, 0, s>>>(in, out, (uint32_t)n, n_dev, add, tot, cap, eff, redo, redo_bit);
    AH_CUDA(cudaGetLastError());
}

int scan_u64_launches(uint64_t n) { return n == 0 ? 0 : n <= kSmallScan ? 1 : 2; }

void launch_pair_write(const ah_site *sites, uint64_t n, const uint64_t *n_dev, const uint8_t *pass,
                       const PairDev *pairs_d, const uint64_t *offsets, ah_amplicon *out, uint64_t cap,
                       const uint64_t *skip, uint64_t skip_bit, cudaStream_t s)
{
    if (!n)
        return;
    pair_write_kernel<<<grid_for(n, 128), 128, 0, s>>>(sites, n, n_dev, pass, pairs_d, offsets, out, cap, skip,
                                                       skip_bit);
    AH_CUDA(cudaGetLastError());
}

} // namespace ah
