// Melting temperature of each site (Sec. 2.1, Melting temperature filtering):
// the maximum over every oligonucleotide of the degenerate primer of the
// two-state nearest-neighbour Tm against the template at the site,
//     Tm(o) = 1000 dH(o) / (dS(o) + C) - 273.15 (+ shift for salt methods 1-4),
// C = R ln(x) (+ 0.368 (L - 1) ln[Na_eq] for salt method 5).
//
// The paper evaluates every oligo separately.  Here the maximum is found
// exactly without enumeration: dH and dS are sums over adjacent primer
// positions, so for a trial value lam the minimum over oligos of
// F(o) = 1000 dH(o) - lam (dS(o) + C) is a 4-state shortest path along the
// primer (choice = base at each position, restricted to its IUPAC set), and
// Dinkelbach's iteration lam <- ratio(argmin F) climbs to the maximum ratio in
// a few rounds, provided dS(o) + C < 0 for every oligo (checked first with a
// max-path pass; otherwise the kernel enumerates the oligos).  One thread per
// site, fp32; when a pass flag is requested and the fp32 Tm is within 0.05 deg C
// of tm_min the site is recomputed in fp64 so the decision equals the fp64 one.
#include <cmath>

#include "ah_internal.h"

namespace ah {
namespace {

constexpr double kR = 1.987; // cal / (K mol)

template <class T> struct Tab {
    const T *sdH, *sdS, *tdH, *tdS;
};

__device__ __forceinline__ Tab<float> tab_of(const PairDev &p, float)
{
    return {p.stack_dH, p.stack_dS, p.term_dH, p.term_dS};
}
__device__ __forceinline__ Tab<double> tab_of(const PairDev &p, double)
{
    return {p.stack_dH_d, p.stack_dS_d, p.term_dH_d, p.term_dS_d};
}

// Max Tm ratio (Kelvin) over oligos with o_i in mask[i], template bases bt[i]
// opposite o_i.  Returns NaN if it cannot decide (never with sane tables).
template <class T>
__device__ T max_ratio(const PairDev &pd, const uint8_t *mask, const int *bt, int L, T cst, int *used_enum)
{
    const Tab<T> tb = tab_of(pd, T(0));
    const T INF = (T)INFINITY;
    // 1. the largest denominator over oligos: max path of dS
    T smax[4];
    for (int x = 0; x < 4; ++x)
        smax[x] = (mask[0] >> x & 1) ? tb.tdS[x * 4 + bt[0]] : -INF;
    for (int i = 1; i < L; ++i) {
        T nx[4];
        for (int y = 0; y < 4; ++y) {
            nx[y] = -INF;
            if (!(mask[i] >> y & 1))
                continue;
            for (int x = 0; x < 4; ++x) {
                T v = smax[x] + tb.sdS[((x * 4 + y) * 4 + bt[i - 1]) * 4 + bt[i]];
                nx[y] = v > nx[y] ? v : nx[y];
            }
        }
        for (int y = 0; y < 4; ++y)
            smax[y] = nx[y];
    }
    T dmax = -INF;
    for (int x = 0; x < 4; ++x) {
        T v = smax[x] + tb.tdS[x * 4 + bt[L - 1]];
        dmax = v > dmax ? v : dmax;
    }
    if (dmax + cst < (T)0) {
        // 2. Dinkelbach iteration on lam
        T lam = 0;
        for (int it = 0; it < 64; ++it) {
            T c[4], h[4], s[4];
            for (int x = 0; x < 4; ++x) {
                if (mask[0] >> x & 1) {
                    h[x] = tb.tdH[x * 4 + bt[0]];
                    s[x] = tb.tdS[x * 4 + bt[0]];
                    c[x] = (T)1000 * h[x] - lam * s[x];
                } else {
                    c[x] = INF;
                    h[x] = s[x] = 0;
                }
            }
            for (int i = 1; i < L; ++i) {
                T nc[4], nh[4], ns[4];
                for (int y = 0; y < 4; ++y) {
                    nc[y] = INF;
                    nh[y] = ns[y] = 0;
                    if (!(mask[i] >> y & 1))
                        continue;
                    for (int x = 0; x < 4; ++x) {
                        if (!(c[x] < INF))
                            continue;
                        const int idx = ((x * 4 + y) * 4 + bt[i - 1]) * 4 + bt[i];
                        const T dh = tb.sdH[idx], ds = tb.sdS[idx];
                        const T v = c[x] + (T)1000 * dh - lam * ds;
                        if (v < nc[y]) {
                            nc[y] = v;
                            nh[y] = h[x] + dh;
                            ns[y] = s[x] + ds;
                        }
                    }
                }
                for (int y = 0; y < 4; ++y) {
                    c[y] = nc[y];
                    h[y] = nh[y];
                    s[y] = ns[y];
                }
            }
            T best = INF, bh = 0, bs = 0;
            for (int x = 0; x < 4; ++x) {
                if (!(c[x] < INF))
                    continue;
                const T th = tb.tdH[x * 4 + bt[L - 1]], ts = tb.tdS[x * 4 + bt[L - 1]];
                const T v = c[x] + (T)1000 * th - lam * ts;
                if (v < best) {
                    best = v;
                    bh = h[x] + th;
                    bs = s[x] + ts;
                }
            }
            const T r = (T)1000 * bh / (bs + cst);
            if (it > 0 && !(r > lam))
                return lam;
            lam = r;
        }
        return lam;
    }
    // 3. fallback: enumerate every oligo
    *used_enum = 1;
    int dig[AH_MAX_PRIMER_LEN];
    for (int i = 0; i < L; ++i) {
        dig[i] = 0;
        while (!(mask[i] >> dig[i] & 1))
            ++dig[i];
    }
    T best = -INF;
    for (int guard = 0; guard < 20000; ++guard) {
        T H = tb.tdH[dig[0] * 4 + bt[0]] + tb.tdH[dig[L - 1] * 4 + bt[L - 1]];
        T S = tb.tdS[dig[0] * 4 + bt[0]] + tb.tdS[dig[L - 1] * 4 + bt[L - 1]];
        for (int i = 1; i < L; ++i) {
            const int idx = ((dig[i - 1] * 4 + dig[i]) * 4 + bt[i - 1]) * 4 + bt[i];
            H += tb.sdH[idx];
            S += tb.sdS[idx];
        }
        const T r = (T)1000 * H / (S + cst);
        best = r > best ? r : best;
        int i = L - 1;
        for (; i >= 0; --i) {
            do {
                ++dig[i];
            } while (dig[i] < 4 && !(mask[i] >> dig[i] & 1));
            if (dig[i] < 4)
                break;
            dig[i] = 0;
            while (!(mask[i] >> dig[i] & 1))
                ++dig[i];
        }
        if (i < 0)
            break;
    }
    return best;
}

__device__ __forceinline__ int base_at(const uint32_t *__restrict__ planes, uint64_t P)
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

__global__ void __launch_bounds__(128) tm_kernel(const ah_site *__restrict__ sites, uint64_t n,
                                                 const PairDev *__restrict__ pairs, int n_pairs,
                                                 const uint32_t *__restrict__ planes,
                                                 const uint64_t *__restrict__ contig_off, float *__restrict__ tm_out,
                                                 uint8_t *__restrict__ pass_out, int *__restrict__ err)
{
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const ah_site s = sites[i];
        if (s.pair >= n_pairs || s.primer > 1 || s.strand > 1) {
            atomicExch(err, kDevBounds);
            tm_out[i] = NAN;
            if (pass_out)
                pass_out[i] = 0;
            continue;
        }
        const PairDev &pd = pairs[s.pair];
        const int L = pd.L[s.primer];
        const uint8_t *mask = pd.mask[s.primer];
        const uint64_t P = contig_off[s.contig] + s.pos;
        int bt[AH_MAX_PRIMER_LEN];
        bool bad = false;
        for (int q = 0; q < L; ++q) {
            const int c = base_at(planes, P + (s.strand == 0 ? q : L - 1 - q));
            if (c < 0)
                bad = true;
            bt[q] = (s.strand == 0) ? 3 - c : c; // template base opposite primer position q
        }
        float tm = NAN;
        uint8_t pass = 0;
        if (!bad) {
            int used_enum = 0;
            const float cst = (float)(pd.sconst + pd.salt_dS_per_stack * (L - 1));
            tm = max_ratio<float>(pd, mask, bt, L, cst, &used_enum) - 273.15f + (float)pd.tm_shift;
            if (pass_out) {
                if (fabsf(tm - pd.tm_min_f) < 0.05f) {
                    const double cst_d = pd.sconst + pd.salt_dS_per_stack * (L - 1);
                    const double tm_d = max_ratio<double>(pd, mask, bt, L, cst_d, &used_enum) - 273.15 + pd.tm_shift;
                    pass = tm_d >= pd.tm_min;
                } else {
                    pass = tm >= pd.tm_min_f;
                }
            }
        }
        tm_out[i] = tm;
        if (pass_out)
            pass_out[i] = pass;
    }
}

} // namespace

void launch_tm(const ah_site *sites, uint64_t n, const PairDev *pairs_d, int n_pairs, const uint32_t *planes,
               const uint64_t *contig_off, float *tm_out, uint8_t *pass_out, int *err, cudaStream_t s)
{
    if (!n)
        return;
    uint64_t blocks = (n + 127) / 128;
    if (blocks > 65535)
        blocks = 65535;
    tm_kernel<<<(unsigned)blocks, 128, 0, s>>>(sites, n, pairs_d, n_pairs, planes, contig_off, tm_out, pass_out, err);
    AH_CUDA(cudaGetLastError());
}

} // namespace ah
