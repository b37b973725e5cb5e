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
// max-path pass; otherwise the oligos are enumerated).  Four lanes per site,
// fp32; when a pass flag is requested and the fp32 Tm is within 0.01 deg C of
// tm_min, the decision is taken in fp64 (one DP at the threshold), so it
// equals the fp64 decision.
#include <cmath>

#include "ah_internal.h"

namespace ah {
namespace {

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

// Four lanes per site: lane y of a group holds the DP state "oligo base at
// the current position = y".  Each step takes the four predecessor costs by
// shuffles, keeps the best predecessor (2 bits per position, so the argmin
// oligo is recovered by a backtrack across the group's lanes) and the
// oligo's dH, dS are then summed by the four lanes together.  Eight sites per
// warp; the rare enumeration fallback and the fp64 recompute near tm_min run
// on lane 0 of the group with the single-thread routine above.
constexpr int kTmWarps = 4;

template <class F> __device__ __forceinline__ float group_reduce(float v, F op)
{
    v = op(v, __shfl_xor_sync(0xffffffffu, v, 1));
    v = op(v, __shfl_xor_sync(0xffffffffu, v, 2));
    return v;
}

__global__ void __launch_bounds__(32 * kTmWarps) tm_kernel(const ah_site *__restrict__ sites, uint64_t n,
                                                           const PairDev *__restrict__ pairs, int n_pairs,
                                                           const uint32_t *__restrict__ planes,
                                                           const uint64_t *__restrict__ contig_off,
                                                           float *__restrict__ tm_out, uint8_t *__restrict__ pass_out,
                                                           int *__restrict__ err)
{
    __shared__ int8_t bts[kTmWarps][8][AH_MAX_PRIMER_LEN];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, y = lane & 3, g0 = lane & ~3;
    int8_t *bt = bts[warp][g];
    const float INF = INFINITY;
    const uint64_t groups = (uint64_t)gridDim.x * kTmWarps * 8;
    for (uint64_t base = ((uint64_t)blockIdx.x * kTmWarps + warp) * 8; base < n; base += groups) {
        const uint64_t i = base + g;
        const bool live = i < n;
        ah_site s{};
        if (live)
            s = sites[i];
        bool bad_rec = live && (s.pair >= n_pairs || s.primer > 1 || s.strand > 1);
        if (bad_rec && y == 0)
            atomicExch(err, kDevBounds);
        const bool act = live && !bad_rec;
        const PairDev &pd = pairs[act ? s.pair : 0];
        const int L = act ? pd.L[s.primer] : 2;
        const uint8_t *mask = pd.mask[act ? s.primer : 0];
        // template base opposite each primer position (-1: not a base)
        // every entry the DP reads is written (0..3), also for groups without a live site
        bool bad = false;
        if (act) {
            const uint64_t P = contig_off[s.contig] + s.pos;
            for (int q = y; q < L; q += 4) {
                const int c = base_at(planes, P + (s.strand == 0 ? q : L - 1 - q));
                bad |= c < 0;
                bt[q] = (int8_t)(c < 0 ? 0 : (s.strand == 0 ? 3 - c : c));
            }
        } else {
            for (int q = y; q < L; q += 4)
                bt[q] = 0;
        }
        __syncwarp();
        bad = __shfl_sync(0xffffffffu, (int)bad, g0) | __shfl_sync(0xffffffffu, (int)bad, g0 + 1) |
              __shfl_sync(0xffffffffu, (int)bad, g0 + 2) | __shfl_sync(0xffffffffu, (int)bad, g0 + 3);
        const bool run = act && !bad;
        const float cst = act ? (float)(pd.sconst + pd.salt_dS_per_stack * (L - 1)) : -1.f;
        // Shuffles need all 32 lanes, but the groups' primer lengths differ: every
        // position loop runs to the warp's longest primer Lw and each group only
        // reads tables and updates its state while q < L (bt[q] is written for q < L).
        int Lw = L;
        for (int d = 16; d >= 1; d >>= 1)
            Lw = max(Lw, __shfl_xor_sync(0xffffffffu, Lw, d));
        // largest denominator over oligos (max-path of dS)
        float sm = (run && (mask[0] >> y & 1)) ? pd.term_dS[y * 4 + bt[0]] : -INF;
        for (int q = 1; q < Lw; ++q) {
            const bool in = q < L;
            float best = -INF;
            for (int x = 0; x < 4; ++x) {
                const float cx = __shfl_sync(0xffffffffu, sm, g0 + x);
                if (in) {
                    const float v = cx + pd.stack_dS[((x * 4 + y) * 4 + bt[q - 1]) * 4 + bt[q]];
                    best = v > best ? v : best;
                }
            }
            if (in)
                sm = (mask[q] >> y & 1) ? best : -INF;
        }
        float dm = sm + ((mask[L - 1] >> y & 1) ? pd.term_dS[y * 4 + bt[L - 1]] : 0.f);
        dm = group_reduce(dm, [](float a, float b) { return a > b ? a : b; });
        const bool dink = run && dm + cst < 0.f;
        float lam = 0.f;
        for (int it = 0; it < 64; ++it) {
            // min over oligos of 1000 dH - lam dS, with the best predecessor of every position
            float c = (dink && (mask[0] >> y & 1)) ? 1000.f * pd.term_dH[y * 4 + bt[0]] - lam * pd.term_dS[y * 4 + bt[0]]
                                                    : INF;
            uint64_t pred = 0;
            for (int q = 1; q < Lw; ++q) {
                const bool in = q < L;
                float best = INF;
                int arg = 0;
                for (int x = 0; x < 4; ++x) {
                    const float cx = __shfl_sync(0xffffffffu, c, g0 + x);
                    if (in) {
                        const int idx = ((x * 4 + y) * 4 + bt[q - 1]) * 4 + bt[q];
                        const float v = cx + 1000.f * pd.stack_dH[idx] - lam * pd.stack_dS[idx];
                        if (v < best) {
                            best = v;
                            arg = x;
                        }
                    }
                }
                if (in) {
                    c = (mask[q] >> y & 1) ? best : INF;
                    pred |= (uint64_t)arg << (2 * q);
                }
            }
            float fin = c + 1000.f * pd.term_dH[y * 4 + bt[L - 1]] - lam * pd.term_dS[y * 4 + bt[L - 1]];
            if (!(c < INF))
                fin = INF;
            // argmin over the group's four end states (ties: lowest base)
            float fmin = group_reduce(fin, [](float a, float b) { return a < b ? a : b; });
            const unsigned hit = __ballot_sync(0xffffffffu, fin == fmin) >> g0 & 0xFu;
            int cur = hit ? __ffs(hit) - 1 : 0;
            // backtrack the oligo: o[L-1] = cur, o[q-1] = pred of lane o[q] at position q
            uint64_t olig = (uint64_t)cur << (2 * (L - 1));
            for (int q = Lw - 1; q >= 1; --q) {
                const uint64_t pp = __shfl_sync(0xffffffffu, pred, g0 + cur);
                if (q < L) {
                    cur = (int)(pp >> (2 * q) & 3u);
                    olig |= (uint64_t)cur << (2 * (q - 1));
                }
            }
            // its dH and dS, split over the four lanes
            float H = 0.f, S = 0.f;
            for (int q = 1 + y; q < L; q += 4) {
                const int a = (int)(olig >> (2 * (q - 1)) & 3u), b2 = (int)(olig >> (2 * q) & 3u);
                const int idx = ((a * 4 + b2) * 4 + bt[q - 1]) * 4 + bt[q];
                H += pd.stack_dH[idx];
                S += pd.stack_dS[idx];
            }
            H = group_reduce(H, [](float a, float b) { return a + b; });
            S = group_reduce(S, [](float a, float b) { return a + b; });
            const int o0 = (int)(olig & 3u), oL = (int)(olig >> (2 * (L - 1)) & 3u);
            H += pd.term_dH[o0 * 4 + bt[0]] + pd.term_dH[oL * 4 + bt[L - 1]];
            S += pd.term_dS[o0 * 4 + bt[0]] + pd.term_dS[oL * 4 + bt[L - 1]];
            const float r = 1000.f * H / (S + cst);
            // warp-uniform loop: stop when no group still improves
            const bool more = dink && (it == 0 || r > lam);
            if (more)
                lam = r;
            if (!__any_sync(0xffffffffu, more))
                break;
        }
        // Pass flags: the fp32 maximum decides unless it lies within 0.01 deg C of
        // tm_min (fp32 error here is ~1e-4 deg C).  Those sites are decided in
        // fp64 by one DP at lam = T = tm_min + 273.15 - shift: max Tm >= tm_min
        // iff the minimum over oligos of 1000 dH - T (dS + C) is <= 0.
        const float tm32 = lam - 273.15f + (act ? (float)pd.tm_shift : 0.f);
        const bool need = pass_out && dink && fabsf(tm32 - pd.tm_min_f) < 0.01f;
        bool pass64 = false;
        if (__any_sync(0xffffffffu, need)) {
            const double T = act ? pd.tm_min + 273.15 - pd.tm_shift : 0.0;
            const double DINF = INFINITY;
            double cd = (need && (mask[0] >> y & 1)) ? 1000.0 * pd.term_dH_d[y * 4 + bt[0]] - T * pd.term_dS_d[y * 4 + bt[0]]
                                                      : DINF;
            for (int q = 1; q < Lw; ++q) {
                const bool in = q < L;
                double best = DINF;
                for (int x = 0; x < 4; ++x) {
                    const double cx = __shfl_sync(0xffffffffu, cd, g0 + x);
                    if (in) {
                        const int idx = ((x * 4 + y) * 4 + bt[q - 1]) * 4 + bt[q];
                        const double v = cx + 1000.0 * pd.stack_dH_d[idx] - T * pd.stack_dS_d[idx];
                        best = v < best ? v : best;
                    }
                }
                if (in)
                    cd = (mask[q] >> y & 1) ? best : DINF;
            }
            double fin = cd + 1000.0 * pd.term_dH_d[y * 4 + bt[L - 1]] - T * pd.term_dS_d[y * 4 + bt[L - 1]];
            if (!(cd < DINF))
                fin = DINF;
            fin = fmin(fin, __shfl_xor_sync(0xffffffffu, fin, 1));
            fin = fmin(fin, __shfl_xor_sync(0xffffffffu, fin, 2));
            const double cst_d = act ? pd.sconst + pd.salt_dS_per_stack * (L - 1) : 0.0;
            pass64 = fin - T * cst_d <= 0.0;
        }
        if (y == 0 && act) {
            float tm = NAN;
            uint8_t pass = 0;
            if (!bad) {
                if (dink) {
                    tm = tm32;
                    pass = need ? (uint8_t)pass64 : (uint8_t)(tm >= pd.tm_min_f);
                } else {
                    // tables under which some duplex entropy is >= -C: enumerate the oligos
                    int bti[AH_MAX_PRIMER_LEN];
                    for (int q = 0; q < L; ++q)
                        bti[q] = bt[q];
                    int used_enum = 0;
                    tm = max_ratio<float>(pd, mask, bti, L, cst, &used_enum) - 273.15f + (float)pd.tm_shift;
                    if (pass_out) {
                        if (fabsf(tm - pd.tm_min_f) < 0.01f) {
                            const double cst_d = pd.sconst + pd.salt_dS_per_stack * (L - 1);
                            const double tm_d =
                                max_ratio<double>(pd, mask, bti, L, cst_d, &used_enum) - 273.15 + pd.tm_shift;
                            pass = tm_d >= pd.tm_min;
                        } else {
                            pass = tm >= pd.tm_min_f;
                        }
                    }
                }
            }
            tm_out[i] = tm;
            if (pass_out)
                pass_out[i] = pass;
        } else if (y == 0 && bad_rec) {
            tm_out[i] = NAN;
            if (pass_out)
                pass_out[i] = 0;
        }
        __syncwarp();
    }
}

} // namespace

void launch_tm(const ah_site *sites, uint64_t n, const PairDev *pairs_d, int n_pairs, const uint32_t *planes,
               const uint64_t *contig_off, float *tm_out, uint8_t *pass_out, int *err, cudaStream_t s)
{
    if (!n)
        return;
    const uint64_t per_block = 8ull * kTmWarps; // sites per block per pass
    uint64_t blocks = (n + per_block - 1) / per_block;
    if (blocks > 65535)
        blocks = 65535;
    tm_kernel<<<(unsigned)blocks, 32 * kTmWarps, 0, s>>>(sites, n, pairs_d, n_pairs, planes, contig_off, tm_out,
                                                         pass_out, err);
    AH_CUDA(cudaGetLastError());
}

} // namespace ah
