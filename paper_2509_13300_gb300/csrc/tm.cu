// Melting temperature of each site (Sec. 2.1, Melting temperature filtering):
// the maximum over every oligonucleotide of the degenerate primer of the
// two-state nearest-neighbour Tm against the template at the site,
//     Tm(o) = 1000 dH(o) / (dS(o) + C) - 273.15 (+ shift for salt methods 1-4),
// C = R ln(x), and salt method 5 adds 0.368 (L - 1) ln[Na_eq] to dS.
//
// The paper evaluates every oligo separately.  Here the maximum is found
// without enumeration: dH and dS are sums over adjacent primer positions, so
// for a trial value lam the minimum over oligos of F(o) = 1000 dH(o) -
// lam (dS(o) + C) is a 4-state shortest path along the primer (the state is
// the oligo's base at a position, restricted to its IUPAC set; only the
// degenerate positions and the two ends need a step, the fixed stretches
// between them being folded into per-site 4x4 tables), and
// Dinkelbach's iteration lam <- ratio(argmin F) climbs to the maximum ratio in
// a few rounds, provided dS(o) + C < 0 for every oligo (checked first with a
// max-path pass).  Four lanes per site (one DP state each), fp32.
//
// Sites whose fp32 maximum lies within 0.01 deg C of tm_min (fp32 error here
// is ~1e-3 deg C at most) get an exact decision instead: Tm(o) >= tm_min iff
// F(o) = 1000 dH(o) - thr (dS(o) + C) <= 0 at thr = tm_min in kelvin (the
// entropy side is negative), so one more shortest-path pass, in fp64 at
// lam = thr, gives the sign of the minimum of F over all oligos.  Its fp64
// error is ~1e-10 cal; a minimum within 1e-6 cal of zero (a ratio within
// ~1e-9 K of the threshold), and every site under a table where some duplex
// entropy reaches -C, is evaluated the reference way: every oligo, in fp64,
// with the same operation order as the definition and no fused multiply-adds,
// a whole block sharing one site's oligos (tm_exact_kernel).  Either way the
// pass flag is the exact fp64 decision.
#include <algorithm>
#include <cmath>

#include <cstdlib>

#include "ah_internal.h"

namespace ah {
namespace {

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

constexpr int kTmWarps = 4; // 128 threads: also the block size of exact_site

template <class F> __device__ __forceinline__ float group_reduce(float v, F op)
{
    v = op(v, __shfl_xor_sync(0xffffffffu, v, 1));
    v = op(v, __shfl_xor_sync(0xffffffffu, v, 2));
    return v;
}

// fp64 Tm of oligo `olig` (2-bit codes) against template bases bt, in the
// operation order of the definition: stacks 0..L-2, then the 5' and the 3'
// initiation terms, then the salt entropy, then the ratio; _rn intrinsics so
// nothing is contracted.
__device__ double exact_tm(const PairDev &pd, const int8_t *bt, int L, uint64_t olig)
{
    double H = 0.0, S = 0.0;
    for (int q = 0; q + 1 < L; ++q) {
        const int a = (int)(olig >> (2 * q) & 3u), b = (int)(olig >> (2 * (q + 1)) & 3u);
        const int idx = ((a * 4 + b) * 4 + bt[q]) * 4 + bt[q + 1];
        H = __dadd_rn(H, pd.stack_dH_d[idx]);
        S = __dadd_rn(S, pd.stack_dS_d[idx]);
    }
    const int o0 = (int)(olig & 3u), oL = (int)(olig >> (2 * (L - 1)) & 3u);
    H = __dadd_rn(H, pd.term_dH_d[o0 * 4 + bt[0]]);
    S = __dadd_rn(S, pd.term_dS_d[o0 * 4 + bt[0]]);
    H = __dadd_rn(H, pd.term_dH_d[oL * 4 + bt[L - 1]]);
    S = __dadd_rn(S, pd.term_dS_d[oL * 4 + bt[L - 1]]);
    if (pd.saltcorr == 5)
        S = __dadd_rn(S, __dmul_rn(__dmul_rn(0.368, (double)(L - 1)), pd.log_na));
    double tm = __dsub_rn(__ddiv_rn(__dmul_rn(1000.0, H), __dadd_rn(S, pd.sconst)), 273.15);
    if (pd.saltcorr == 1)
        tm = __dadd_rn(tm, pd.tm_shift);
    return tm;
}

// Oligo number o (0 <= o < degeneracy <= 10000) of a primer with position sets
// qm -> its bases, 2 bits per position (mixed radix over the positions' sets).
__device__ uint64_t oligo_number(const uint8_t *qm, int L, int o)
{
    uint64_t olig = 0;
    int rem = o;
    for (int q = L - 1; q >= 0; --q) {
        const int nqb = __popc(qm[q]);
        int d; // rem % nqb, rem /= nqb for nqb in 1..4 (rem < 10000)
        if (nqb == 1) {
            d = 0;
        } else if (nqb == 2) {
            d = rem & 1;
            rem >>= 1;
        } else if (nqb == 4) {
            d = rem & 3;
            rem >>= 2;
        } else {
            const int q3 = (rem * 43691) >> 17; // rem / 3, exact for rem < 2^16
            d = rem - 3 * q3;
            rem = q3;
        }
        int base_q = 0;
        for (int x = 0; x < 4; ++x)
            if (qm[q] >> x & 1) {
                if (d == 0) {
                    base_q = x;
                    break;
                }
                --d;
            }
        olig |= (uint64_t)base_q << (2 * q);
    }
    return olig;
}

// One queued site with a whole block of kExactThreads: every oligo in fp64
// with the definition's operation order (exact_tm), block-wide maximum, then
// the Tm and the pass flag.  bt and wmax are the block's shared scratch.
constexpr int kExactThreads = 128; // fp64-bound: a block of 128 already keeps the SM's fp64 units busy

__device__ void exact_site(const ah_site *__restrict__ sites, const PairDev *__restrict__ pairs,
                           const uint32_t *__restrict__ planes, const uint64_t *__restrict__ contig_off, uint32_t i,
                           float *__restrict__ tm_out, uint8_t *__restrict__ pass_out, int8_t *bt, double *wmax)
{
    const ah_site s = sites[i];
    const PairDev &pd = pairs[s.pair];
    const int L = pd.L[s.primer];
    const uint8_t *qm = pd.mask[s.primer];
    const uint64_t P = contig_off[s.contig] + s.pos;
    for (int q = threadIdx.x; q < L; q += blockDim.x) {
        const int c = base_at(planes, P + (s.strand == 0 ? q : L - 1 - q));
        bt[q] = (int8_t)(s.strand == 0 ? 3 - c : c); // queued sites have only A/C/G/T
    }
    __syncthreads();
    int deg = 1;
    for (int q = 0; q < L; ++q)
        deg *= __popc(qm[q]);
    double best = -INFINITY;
    for (int o = threadIdx.x; o < deg; o += blockDim.x) {
        const double t = exact_tm(pd, bt, L, oligo_number(qm, L, o));
        best = t > best ? t : best;
    }
    for (int d = 16; d >= 1; d >>= 1) {
        const double o2 = __shfl_xor_sync(0xffffffffu, best, d);
        best = o2 > best ? o2 : best;
    }
    if ((threadIdx.x & 31) == 0)
        wmax[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = wmax[0];
        for (int w = 1; w < kExactThreads / 32; ++w)
            m = wmax[w] > m ? wmax[w] : m;
        float tm = (float)m;
        if (pass_out) {
            const bool pass = m >= pd.tm_min;
            pass_out[i] = pass;
            if (!pass && tm >= pd.tm_min_f) // rounding to fp32 may reach the threshold: stay below it
                tm = nextafterf(pd.tm_min_f, -INFINITY);
        }
        tm_out[i] = tm;
    }
    __syncthreads(); // bt and wmax are reused by the next queued site
}

// Queued sites, one block per site (tables under which many sites may queue).
// The queue length is read on the device.
__global__ void __launch_bounds__(kExactThreads) tm_exact_kernel(const ah_site *__restrict__ sites,
                                                                 const PairDev *__restrict__ pairs,
                                                                 const uint32_t *__restrict__ planes,
                                                                 const uint64_t *__restrict__ contig_off,
                                                                 const uint32_t *__restrict__ queue,
                                                                 const uint32_t *__restrict__ queue_n,
                                                                 float *__restrict__ tm_out,
                                                                 uint8_t *__restrict__ pass_out)
{
    __shared__ int8_t bt[AH_MAX_PRIMER_LEN];
    __shared__ double wmax[kExactThreads / 32];
    const uint32_t nq = *queue_n;
    for (uint32_t e = blockIdx.x; e < nq; e += gridDim.x)
        exact_site(sites, pairs, planes, contig_off, queue[e], tm_out, pass_out, bt, wmax);
}

// Per-pair constants of the fp32 path, staged in shared memory by every
// block (the shortest-path steps read them in dependent chains).
struct TmPairS {
    float2 st[256]; // (dH, dS) of each stack
    float2 tm[16];  // (dH, dS) of each terminal pair
    uint8_t mask[2][AH_MAX_PRIMER_LEN];
    uint8_t key[2][AH_MAX_PRIMER_LEN];
    int L[2], nkey[2];
};
static_assert(sizeof(TmPairS) % 16 == 0, "TmPairS keeps 16-byte alignment");

// The weights 1000 dH - thr dS of every table entry at the pair's threshold
// thr, for the near-threshold sign test: computed in fp64 from the fp64
// table, then held as fixed point (units of 2^-30 cal/mol, int64) so that
// every path sum is exact; staged for up to kTmStageD pairs.
struct TmPairD {
    long long st[256];
    long long tm[16];
};
constexpr double kFix = 1073741824.0; // 2^30: fixed-point scale of the sign test
// |each weight's rounding| <= 2^-31 cal/mol, so a path of <= 32 terms is within
// 2e-8 of its exact value; decisions use a margin of 1e-6 cal/mol (file comment)
constexpr long long kFixMargin = 1074; // 1e-6 * 2^30
constexpr int kSweepMax = 64;          // thresholds per sweep (one bit each)

__device__ __forceinline__ long long fix_weight(double dH, double dS, double thr)
{
    return __double2ll_rn((1000.0 * dH - thr * dS) * kFix);
}
constexpr int kTmStageD = 4;

// Four lanes per site: lane y of a group holds the DP state "oligo base at
// the current key position = y".  Each step takes the four predecessor costs
// by shuffles and keeps the best predecessor (2 bits per key), so the argmin
// oligo is recovered by a backtrack across the group's lanes; its dH, dS are
// then summed by the four lanes together.  Eight sites per warp.
__global__ void __launch_bounds__(32 * kTmWarps) tm_kernel(const ah_site *__restrict__ sites, uint64_t n_arg,
                                                           const uint64_t *__restrict__ n_dev,
                                                           const PairDev *__restrict__ pairs, int n_pairs,
                                                           const uint32_t *__restrict__ planes,
                                                           const uint64_t *__restrict__ contig_off,
                                                           float *__restrict__ tm_out, uint8_t *__restrict__ pass_out,
                                                           uint32_t *__restrict__ queue, uint32_t *__restrict__ queue_n,
                                                           int seg_max, int last_block_exact, int *__restrict__ err,
                                                           const uint32_t *__restrict__ idx_list)
{
    static_assert(32 * kTmWarps == kExactThreads, "the last block evaluates queued sites with exact_site");
    __shared__ int8_t bts[kTmWarps][8][AH_MAX_PRIMER_LEN];
    // dynamic: [n_pairs] TmPairS, [n_pairs <= kTmStageD ? n_pairs : 0] TmPairD,
    // then [kTmWarps * 8 sites][seg_max][16] segment tables
    extern __shared__ __align__(16) unsigned char tm_smem[];
    TmPairS *ps = reinterpret_cast<TmPairS *>(tm_smem);
    const int nd = n_pairs <= kTmStageD ? n_pairs : 0;
    TmPairD *pdd = reinterpret_cast<TmPairD *>(tm_smem + (size_t)n_pairs * sizeof(TmPairS));
    float2 *seg_smem =
        reinterpret_cast<float2 *>(tm_smem + (size_t)n_pairs * sizeof(TmPairS) + (size_t)nd * sizeof(TmPairD));
    // a block with no site of the list skips the tables (it still counts itself below)
    const bool has_work = (uint64_t)blockIdx.x * kTmWarps * 8 < dev_count(n_arg, n_dev);
    for (int j = 0; has_work && j < n_pairs; ++j) {
        const PairDev &P = pairs[j];
        for (int t = threadIdx.x; t < 256; t += blockDim.x)
            ps[j].st[t] = make_float2(P.stack_dH[t], P.stack_dS[t]);
        if (threadIdx.x < 16)
            ps[j].tm[threadIdx.x] = make_float2(P.term_dH[threadIdx.x], P.term_dS[threadIdx.x]);
        if (threadIdx.x < 2 * AH_MAX_PRIMER_LEN) {
            (&ps[j].mask[0][0])[threadIdx.x] = (&P.mask[0][0])[threadIdx.x];
            (&ps[j].key[0][0])[threadIdx.x] = (&P.key[0][0])[threadIdx.x];
        }
        if (threadIdx.x < 2) {
            ps[j].L[threadIdx.x] = P.L[threadIdx.x];
            ps[j].nkey[threadIdx.x] = P.nkey[threadIdx.x];
        }
        if (j < nd) {
            for (int t = threadIdx.x; t < 256; t += blockDim.x)
                pdd[j].st[t] = fix_weight(P.stack_dH_d[t], P.stack_dS_d[t], P.thr);
            if (threadIdx.x < 16)
                pdd[j].tm[threadIdx.x] = fix_weight(P.term_dH_d[threadIdx.x], P.term_dS_d[threadIdx.x], P.thr);
        }
    }
    __syncthreads();
    const uint64_t n = dev_count(n_arg, n_dev);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, y = lane & 3, g0 = lane & ~3;
    int8_t *bt = bts[warp][g];
    const float INF = INFINITY;
    const uint64_t groups = (uint64_t)gridDim.x * kTmWarps * 8;
    for (uint64_t base = ((uint64_t)blockIdx.x * kTmWarps + warp) * 8; base < n; base += groups) {
        const bool live = base + g < n;
        // with idx_list, the sites taken are sites[idx_list[0 .. n)]
        const uint64_t i = live && idx_list ? (uint64_t)idx_list[base + g] : base + g;
        ah_site s{};
        if (live)
            s = sites[i];
        const bool bad_rec = live && (s.pair >= n_pairs || s.primer > 1 || s.strand > 1);
        if (bad_rec && y == 0)
            atomicExch(err, kDevBounds);
        const bool act = live && !bad_rec;
        const PairDev &pd = pairs[act ? s.pair : 0];
        const TmPairS &sp = ps[act ? s.pair : 0];
        const int L = act ? sp.L[s.primer] : 2;
        const uint8_t *mask = sp.mask[act ? s.primer : 0];
        // template base opposite each primer position; every entry the DP reads
        // is written (0..3), also for groups without a live site.  All of a lane's
        // plane words are requested before any is used (one memory latency).
        bool bad = false;
        if (act) {
            const uint64_t P = contig_off[s.contig] + s.pos;
            uint32_t w[8][4];
            int bitpos[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int q = min(y + 4 * j, L - 1); // past the primer: a repeat of its last position, unused
                const uint64_t Pq = P + (s.strand == 0 ? q : L - 1 - q);
                const uint64_t t = Pq / kTileBases, r = Pq % kTileBases;
                bitpos[j] = (int)(r / kTileW);
                const uint32_t *wp = planes + t * 4 * kTileWX + (r % kTileW);
#pragma unroll
                for (int x = 0; x < 4; ++x)
                    w[j][x] = __ldg(wp + x * kTileWX);
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int q = y + 4 * j;
                if (q < L) {
                    int c = -1;
#pragma unroll
                    for (int x = 0; x < 4; ++x)
                        if ((w[j][x] >> bitpos[j]) & 1u)
                            c = x;
                    bad |= c < 0;
                    bt[q] = (int8_t)(c < 0 ? 0 : (s.strand == 0 ? 3 - c : c));
                }
            }
        } else {
            for (int q = y; q < L; q += 4)
                bt[q] = 0;
        }
        __syncwarp();
        bad = __shfl_sync(0xffffffffu, (int)bad, g0) | __shfl_sync(0xffffffffu, (int)bad, g0 + 1) |
              __shfl_sync(0xffffffffu, (int)bad, g0 + 2) | __shfl_sync(0xffffffffu, (int)bad, g0 + 3);
        const bool run = act && !bad;
        const float cst =
            act ? (float)(pd.sconst + (pd.saltcorr == 5 ? 0.368 * (double)(L - 1) * pd.log_na : 0.0)) : -1.f;
        // Steps at key positions only (primer positions 0 and L-1 and every
        // degenerate one): between two keys the oligo bases are fixed, so all
        // stacks from key i to key i+1 form a 4x4 table of (dH, dS) sums
        // indexed by the bases at the two keys, E[i][a * 4 + b].  Lane y fills
        // column y of the site's tables once; every pass below reads them.
        const int m = act ? sp.nkey[s.primer] - 1 : 0; // segments
        const uint8_t *key = sp.key[act ? s.primer : 0];
        float2 *E = seg_smem + (size_t)(warp * 8 + g) * seg_max * 16;
        if (run) {
            for (int si = 0; si < m; ++si) {
                const int k0 = key[si], k1 = key[si + 1];
                if (k1 == k0 + 1) {
                    for (int x = 0; x < 4; ++x) {
                        E[si * 16 + x * 4 + y] = sp.st[((x * 4 + y) * 4 + bt[k0]) * 4 + bt[k1]];
                    }
                } else {
                    float cH = 0.f, cS = 0.f; // stacks between two fixed bases
                    for (int q = k0 + 2; q < k1; ++q) {
                        const int a0 = __ffs(mask[q - 1]) - 1, b0 = __ffs(mask[q]) - 1;
                        const float2 e = sp.st[((a0 * 4 + b0) * 4 + bt[q - 1]) * 4 + bt[q]];
                        cH += e.x;
                        cS += e.y;
                    }
                    const int fa = __ffs(mask[k0 + 1]) - 1, fb = __ffs(mask[k1 - 1]) - 1;
                    const float2 eq = sp.st[((fb * 4 + y) * 4 + bt[k1 - 1]) * 4 + bt[k1]]; // into key k1, base y
                    const float qH = eq.x + cH, qS = eq.y + cS;
                    for (int x = 0; x < 4; ++x) {
                        const float2 ep = sp.st[((x * 4 + fa) * 4 + bt[k0]) * 4 + bt[k0 + 1]]; // out of key k0, base x
                        E[si * 16 + x * 4 + y] = make_float2(ep.x + qH, ep.y + qS);
                    }
                }
            }
        }
        __syncwarp();
        // bit i: base y is allowed at key i; this lane's terminal terms at both ends
        uint32_t amask = 0;
        float2 t0 = make_float2(0.f, 0.f), tL = make_float2(0.f, 0.f);
        if (run) {
            for (int si = 0; si <= m; ++si)
                amask |= (uint32_t)(mask[key[si]] >> y & 1) << si;
            t0 = sp.tm[y * 4 + bt[0]];
            tL = sp.tm[y * 4 + bt[L - 1]];
        }
        // Shuffles need all 32 lanes, but the groups' segment counts differ: every
        // segment loop runs to the warp's largest count mw and each group only
        // updates its state while si < m.
        int mw = run ? m : 0;
        for (int d = 16; d >= 1; d >>= 1)
            mw = max(mw, __shfl_xor_sync(0xffffffffu, mw, d));
        // largest denominator over oligos (max-path of dS)
        float sm = (amask & 1u) ? t0.y : -INF;
        for (int si = 0; si < mw; ++si) {
            const bool in = run && si < m;
            float best = -INF;
#pragma unroll
            for (int x = 0; x < 4; ++x) {
                const float cx = __shfl_sync(0xffffffffu, sm, g0 + x);
                if (in) {
                    const float v = cx + E[si * 16 + x * 4 + y].y;
                    best = v > best ? v : best;
                }
            }
            if (in)
                sm = (amask >> (si + 1) & 1u) ? best : -INF;
        }
        float dm = sm + ((amask >> m & 1u) ? tL.y : 0.f);
        dm = group_reduce(dm, [](float a, float b) { return a > b ? a : b; });
        const bool dink = run && dm + cst < 0.f;
        float lam = 0.f;
        for (int it = 0; it < 64; ++it) {
            // min over oligos of 1000 dH - lam dS, with the best predecessor at every key
            float c = (dink && (amask & 1u)) ? 1000.f * t0.x - lam * t0.y : INF;
            uint64_t pred = 0;
            for (int si = 0; si < mw; ++si) {
                const bool in = dink && si < m;
                float best = INF;
                int arg = 0;
#pragma unroll
                for (int x = 0; x < 4; ++x) {
                    const float cx = __shfl_sync(0xffffffffu, c, g0 + x);
                    if (in) {
                        const float2 e = E[si * 16 + x * 4 + y];
                        const float v = cx + fmaf(-lam, e.y, 1000.f * e.x);
                        if (v < best) {
                            best = v;
                            arg = x;
                        }
                    }
                }
                if (in) {
                    c = (amask >> (si + 1) & 1u) ? best : INF;
                    pred |= (uint64_t)arg << (2 * si);
                }
            }
            float fin = dink ? c + 1000.f * tL.x - lam * tL.y : INF;
            if (!(c < INF))
                fin = INF;
            // argmin over the group's four end states (ties: lowest base)
            const float fmin = group_reduce(fin, [](float a, float b) { return a < b ? a : b; });
            const unsigned hit = __ballot_sync(0xffffffffu, fin == fmin) >> g0 & 0xFu;
            int cur = hit ? __ffs(hit) - 1 : 0;
            // backtrack the bases at the keys: ks[i] = base at key i (2 bits each)
            uint64_t ks = (uint64_t)cur << (2 * m);
            for (int si = mw - 1; si >= 0; --si) {
                const uint64_t pp = __shfl_sync(0xffffffffu, pred, g0 + cur);
                if (si < m) {
                    cur = (int)(pp >> (2 * si) & 3u);
                    ks |= (uint64_t)cur << (2 * si);
                }
            }
            // its dH and dS: the segment tables, split over the four lanes
            float H = 0.f, S = 0.f;
            if (dink)
                for (int si = y; si < m; si += 4) {
                    const int a0 = (int)(ks >> (2 * si) & 3u), b0 = (int)(ks >> (2 * (si + 1)) & 3u);
                    const float2 e = E[si * 16 + a0 * 4 + b0];
                    H += e.x;
                    S += e.y;
                }
            H = group_reduce(H, [](float a, float b) { return a + b; });
            S = group_reduce(S, [](float a, float b) { return a + b; });
            // terminal terms of the chosen end bases: held by the lanes of those bases
            const int o0 = (int)(ks & 3u), oL = (int)(ks >> (2 * m) & 3u);
            H += __shfl_sync(0xffffffffu, t0.x, g0 + o0) + __shfl_sync(0xffffffffu, tL.x, g0 + oL);
            S += __shfl_sync(0xffffffffu, t0.y, g0 + o0) + __shfl_sync(0xffffffffu, tL.y, g0 + oL);
            const float r = 1000.f * H / (S + cst);
            // Warp-uniform loop: stop when no group still improves by more than
            // 1e-4 K.  In fp32 two oligos of nearly equal ratio could otherwise
            // trade places by one ulp for many rounds; 1e-4 K is far below the
            // 0.01 deg C tolerance, and sites near tm_min are decided exactly below.
            const bool more = dink && (it == 0 || r > lam + 1e-4f);
            if (more)
                lam = r;
            if (!__any_sync(0xffffffffu, more))
                break;
        }
        const float tm32 = lam - 273.15f + (act ? (float)pd.tm_shift : 0.f);
        // near the threshold: the sign of min F at lam = thr, in fp64 (file comment)
        const bool near = dink && pass_out && fabsf(tm32 - pd.tm_min_f) < 0.01f;
        int decided = -1; // 1 pass, 0 fail, -1 undecided
        if (__any_sync(0xffffffffu, near)) {
            // Same key segments, exact fixed-point weights at lam = thr.  First every
            // weight W[i][x] of this lane's column (independent work, written over the
            // fp32 tables, no longer needed), then the dependent chain over the segments.
            const long long LINF = 0x2000000000000000ll; // above any path sum, no overflow when added to
            long long *W = reinterpret_cast<long long *>(E); // W[si * 16 + x * 4 + y], 8 bytes per float2 slot
            const bool staged = act && s.pair < nd;
            const TmPairD &sd = pdd[staged ? s.pair : 0];
            auto stW = [&](int idx) {
                return staged ? sd.st[idx] : fix_weight(pd.stack_dH_d[idx], pd.stack_dS_d[idx], pd.thr);
            };
            auto tmW = [&](int idx) {
                return staged ? sd.tm[idx] : fix_weight(pd.term_dH_d[idx], pd.term_dS_d[idx], pd.thr);
            };
            __syncwarp();
            if (near) {
                for (int si = 0; si < m; ++si) {
                    const int k0 = key[si], k1 = key[si + 1];
                    if (k1 == k0 + 1) {
                        for (int x = 0; x < 4; ++x)
                            W[si * 16 + x * 4 + y] = stW(((x * 4 + y) * 4 + bt[k0]) * 4 + bt[k1]);
                    } else {
                        long long cw = 0; // the fixed stretch and the step into key k1 with base y
                        for (int q = k0 + 2; q < k1; ++q) {
                            const int a0 = __ffs(mask[q - 1]) - 1, b0 = __ffs(mask[q]) - 1;
                            cw += stW(((a0 * 4 + b0) * 4 + bt[q - 1]) * 4 + bt[q]);
                        }
                        const int fa = __ffs(mask[k0 + 1]) - 1, fb = __ffs(mask[k1 - 1]) - 1;
                        cw += stW(((fb * 4 + y) * 4 + bt[k1 - 1]) * 4 + bt[k1]);
                        for (int x = 0; x < 4; ++x)
                            W[si * 16 + x * 4 + y] = stW(((x * 4 + fa) * 4 + bt[k0]) * 4 + bt[k0 + 1]) + cw;
                    }
                }
            }
            __syncwarp();
            long long cd = (near && (amask & 1u)) ? tmW(y * 4 + bt[0]) : LINF;
            for (int si = 0; si < mw; ++si) {
                const bool in = near && si < m;
                long long best = LINF;
#pragma unroll
                for (int x = 0; x < 4; ++x) {
                    const long long cx = __shfl_sync(0xffffffffu, cd, g0 + x);
                    if (in) {
                        const long long v = cx + W[si * 16 + x * 4 + y];
                        best = v < best ? v : best;
                    }
                }
                if (in)
                    cd = (amask >> (si + 1) & 1u) ? best : LINF;
            }
            long long fin = cd < LINF ? cd + tmW(y * 4 + bt[L - 1]) : LINF;
            long long o1 = __shfl_xor_sync(0xffffffffu, fin, 1);
            fin = o1 < fin ? o1 : fin;
            o1 = __shfl_xor_sync(0xffffffffu, fin, 2);
            fin = o1 < fin ? o1 : fin;
            if (near) {
                // min F = min path sum - thr (C + salt entropy)
                const double Cp = pd.sconst + (pd.saltcorr == 5 ? 0.368 * (double)(L - 1) * pd.log_na : 0.0);
                const long long F = fin - __double2ll_rn(pd.thr * Cp * kFix);
                decided = F < -kFixMargin ? 1 : (F > kFixMargin ? 0 : -1);
            }
        }
        // sites decided the reference way (see the file comment) go to a queue, worked
        // off below by the last block or by tm_exact_kernel, a whole block per site
        const bool exact = run && (!dink || (near && decided < 0));
        if (exact && y == 0)
            queue[atomicAdd(queue_n, 1u)] = (uint32_t)i;
        if (y == 0 && act) {
            float tm = NAN;
            uint8_t pass = 0;
            if (!bad) {
                tm = tm32; // replaced by the exact evaluation for queued sites
                pass = tm32 >= pd.tm_min_f;
                if (decided >= 0) { // the exact decision; the fp32 value (within 1e-3) made consistent with it
                    pass = (uint8_t)decided;
                    if (decided && tm < pd.tm_min_f)
                        tm = pd.tm_min_f;
                    if (!decided && tm >= pd.tm_min_f)
                        tm = nextafterf(pd.tm_min_f, -INFINITY);
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
    // Tables under which only the rare ambiguous sites queue: the last block to
    // finish evaluates them (no second launch).  queue_n[1] counts finished blocks.
    if (last_block_exact) {
        __shared__ int is_last;
        __threadfence(); // this block's queue entries and results before its count
        __syncthreads();
        if (threadIdx.x == 0)
            is_last = atomicAdd(queue_n + 1, 1u) == gridDim.x - 1;
        __syncthreads();
        if (is_last) {
            __threadfence();
            const uint32_t nq = *(volatile const uint32_t *)queue_n;
            double *wmax = reinterpret_cast<double *>(seg_smem); // the segment tables are free now
            int8_t *bt0 = &bts[0][0][0];
            for (uint32_t e = 0; e < nq; ++e)
                exact_site(sites, pairs, planes, contig_off, queue[e], tm_out, pass_out, bt0, wmax);
        }
    }
}

// ---------------------------------------------------------------------------
// Thread-per-site Tm (the path taken when every pair has few_exact).  The same
// maximum as tm_kernel -- Dinkelbach iteration on the key-position shortest
// path, fp32 -- but one thread carries all four states of one site: each
// state keeps its path cost and the path's dH and dS sums, so the argmin
// oligo's terms come out of the forward pass without a backtrack.  Between
// two keys that are not adjacent the segment's table is separable (the stack
// out of key k0 depends only on the base at k0, the stack into key k1 only on
// the base at k1, the fixed stretch between them on neither), so one argmin
// over the four predecessors serves all four successors.  A warp gathers its
// 32 sites' windows together: per site, four coalesced 32-word loads (one per
// plane) and four ballots give the window's bases as 32-bit columns.  Sites
// whose maximum lies within 0.01 deg C of tm_min are deferred to tm_kernel
// (which decides them exactly); everything else is written here.
// ---------------------------------------------------------------------------
constexpr int kFastThreads = 128;

// Per pair in shared memory: stacks as (1000 dH, dS) indexed [template bases
// (t0, t1)][oligo bases (o0, o1)], so the 16 entries of one template pair are
// contiguous; terminal pairs [oligo base][template base]; per primer its keys,
// masks, length and C + salt entropy.
struct TmFastPair {
    float2 st[256];
    float2 tm[16];
    uint8_t mask[2][AH_MAX_PRIMER_LEN];
    uint8_t key[2][AH_MAX_PRIMER_LEN];
    int L[2], nkey[2];
    float cst[2];
    float tm_min_f, tm_shift_f;
};
static_assert(sizeof(TmFastPair) % 8 == 0, "TmFastPair keeps 8-byte alignment");

__global__ void __launch_bounds__(kFastThreads) tm_fast_kernel(const ah_site *__restrict__ sites, uint64_t n_arg,
                                                               const uint64_t *__restrict__ n_dev,
                                                               const PairDev *__restrict__ pairs, int n_pairs,
                                                               const uint32_t *__restrict__ planes,
                                                               const uint64_t *__restrict__ contig_off,
                                                               float *__restrict__ tm_out,
                                                               uint8_t *__restrict__ pass_out,
                                                               uint32_t *__restrict__ defer,
                                                               unsigned long long *__restrict__ defer_n,
                                                               int *__restrict__ err)
{
    extern __shared__ __align__(16) unsigned char fast_smem[];
    TmFastPair *fp = reinterpret_cast<TmFastPair *>(fast_smem);
    const uint64_t n = dev_count(n_arg, n_dev);
    if ((uint64_t)blockIdx.x * blockDim.x >= n)
        return; // the whole block: no site for it
    for (int j = 0; j < n_pairs; ++j) {
        const PairDev &P = pairs[j];
        for (int t = threadIdx.x; t < 256; t += blockDim.x) {
            const int o0 = t >> 6, o1 = (t >> 4) & 3, t0 = (t >> 2) & 3, t1 = t & 3; // PairDev index order
            fp[j].st[((t0 * 4 + t1) * 4 + o0) * 4 + o1] = make_float2(1000.f * P.stack_dH[t], P.stack_dS[t]);
        }
        if (threadIdx.x < 16)
            fp[j].tm[threadIdx.x] = make_float2(1000.f * P.term_dH[threadIdx.x], P.term_dS[threadIdx.x]);
        if (threadIdx.x < 2 * AH_MAX_PRIMER_LEN) {
            (&fp[j].mask[0][0])[threadIdx.x] = (&P.mask[0][0])[threadIdx.x];
            (&fp[j].key[0][0])[threadIdx.x] = (&P.key[0][0])[threadIdx.x];
        }
        if (threadIdx.x < 2) {
            const int x = threadIdx.x;
            fp[j].L[x] = P.L[x];
            fp[j].nkey[x] = P.nkey[x];
            fp[j].cst[x] = (float)(P.sconst + (P.saltcorr == 5 ? 0.368 * (double)(P.L[x] - 1) * P.log_na : 0.0));
        }
        if (threadIdx.x == 0) {
            fp[j].tm_min_f = P.tm_min_f;
            fp[j].tm_shift_f = (float)P.tm_shift;
        }
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const float INF = INFINITY;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    // whole warps take 32 consecutive sites, so the window gather below is uniform
    for (uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); i0 < n; i0 += stride) {
        const uint64_t i = i0 + lane;
        const bool live = i < n;
        ah_site s{};
        if (live)
            s = sites[i];
        const bool bad_rec = live && (s.pair >= n_pairs || s.primer > 1 || s.strand > 1);
        if (bad_rec)
            atomicExch(err, kDevBounds);
        const bool act = live && !bad_rec;
        const TmFastPair &sp = fp[act ? s.pair : 0];
        const int pr = act ? s.primer : 0;
        const int L = sp.L[pr];
        // window of the site: tile word offset and bit row of its first position
        uint64_t wofs = 0;
        int brow = 0;
        if (act) {
            const uint64_t P = contig_off[s.contig] + s.pos;
            const uint64_t t = P / kTileBases, r = P % kTileBases;
            brow = (int)(r / kTileW);
            wofs = t * 4 * kTileWX + (r % kTileW);
        }
        // columns of the window's bases (bit q = base at position P + q is A / C / G / T),
        // eight sites at a time: their 32 loads are all in flight before the ballots
        uint32_t cA = 0, cC = 0, cG = 0, cT = 0;
        const uint32_t actm = __ballot_sync(0xffffffffu, act);
        for (int k0 = 0; k0 < 32; k0 += 8) {
            if (!((actm >> k0) & 0xffu))
                continue;
            uint32_t wv[8][4];
            int bk[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const uint64_t wk = __shfl_sync(0xffffffffu, wofs, k0 + j);
                bk[j] = __shfl_sync(0xffffffffu, brow, k0 + j);
                const int Lk = __shfl_sync(0xffffffffu, L, k0 + j);
                // the window's L positions only (the sectors past them are not read)
                const bool on = ((actm >> (k0 + j)) & 1u) && lane < Lk;
                const uint32_t *w = planes + wk + lane; // position P_k + lane (the tile's extension covers 32 more)
#pragma unroll
                for (int x = 0; x < 4; ++x)
                    wv[j][x] = on ? __ldg(w + x * kTileWX) : 0u;
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const uint32_t a = __ballot_sync(0xffffffffu, (wv[j][0] >> bk[j]) & 1u);
                const uint32_t c = __ballot_sync(0xffffffffu, (wv[j][1] >> bk[j]) & 1u);
                const uint32_t g = __ballot_sync(0xffffffffu, (wv[j][2] >> bk[j]) & 1u);
                const uint32_t tt = __ballot_sync(0xffffffffu, (wv[j][3] >> bk[j]) & 1u);
                if (lane == k0 + j) {
                    cA = a;
                    cC = c;
                    cG = g;
                    cT = tt;
                }
            }
        }
        if (!act) {
            if (bad_rec) {
                tm_out[i] = NAN;
                if (pass_out)
                    pass_out[i] = 0;
            }
            continue;
        }
        const uint32_t lm = L >= 32 ? 0xffffffffu : ((1u << L) - 1u);
        const bool bad = (~(cA | cC | cG | cT) & lm) != 0u; // a letter other than A, C, G, T
        // template base opposite primer position q, 2 bits as (hi << 1) | lo with
        // A 0, C 1, G 2, T 3: '+' the complement of the window base at q, '-' the
        // window base at L - 1 - q
        uint32_t blo, bhi;
        if (s.strand == 0) {
            blo = ~(cC | cT) & lm;
            bhi = ~(cG | cT) & lm;
        } else {
            blo = __brev(cC | cT) >> (32 - L);
            bhi = __brev(cG | cT) >> (32 - L);
        }
        if (bad) {
            tm_out[i] = NAN;
            if (pass_out)
                pass_out[i] = 0;
            continue;
        }
        auto bt = [&](int q) { return (int)(((blo >> q) & 1u) | (((bhi >> q) & 1u) << 1)); };
        const uint8_t *key = sp.key[pr];
        const uint8_t *mask = sp.mask[pr];
        const int nk = sp.nkey[pr];
        const int b0 = bt(0), bL = bt(L - 1);
        const float cst = sp.cst[pr];
        // What does not depend on lam, once per site.  The fixed stretches
        // between keys that are not adjacent are the same for every oligo: they
        // add one constant to every path, move no argmin, and join H and S at
        // the end.  The start is an achieved ratio, that of one oligo: at each
        // position the base pairing with the template where the mask allows it,
        // else the mask's first base.  Each pass then either confirms the ratio
        // (no oligo beats it by more than 1e-4 K) or moves to a better one.
        float SH = 0.f, SE = 0.f;
        for (int si = 0; si + 1 < nk; ++si) {
            const int k0 = key[si], k1 = key[si + 1];
            for (int q = k0 + 2; q < k1; ++q) {
                const float2 v2 =
                    sp.st[(bt(q - 1) * 4 + bt(q)) * 16 + (__ffs(mask[q - 1]) - 1) * 4 + (__ffs(mask[q]) - 1)];
                SH += v2.x;
                SE += v2.y;
            }
        }
        float lam;
        {
            auto pick = [&](int q) {
                const int pairing = 3 - bt(q);
                return ((mask[q] >> pairing) & 1) ? pairing : __ffs(mask[q]) - 1;
            };
            int o0 = pick(0);
            float2 t = sp.tm[o0 * 4 + b0];
            float H0 = t.x, S0 = t.y;
            for (int q = 1; q < L; ++q) {
                const int o1 = pick(q);
                const float2 v2 = sp.st[(bt(q - 1) * 4 + bt(q)) * 16 + o0 * 4 + o1];
                H0 += v2.x;
                S0 += v2.y;
                o0 = o1;
            }
            t = sp.tm[o0 * 4 + bL];
            lam = (H0 + t.x) / (S0 + t.y + cst);
        }
        for (int it = 0; it < 64; ++it) {
            // forward pass at lam: per state y (oligo base at the current key) the
            // cheapest path cost 1000 dH - lam dS and that path's 1000 dH and dS
            // (fixed stretches left out)
            float c[4], h[4], e[4];
#pragma unroll
            for (int y = 0; y < 4; ++y) {
                const float2 t = sp.tm[y * 4 + b0];
                const bool ok = (mask[0] >> y) & 1;
                c[y] = ok ? fmaf(-lam, t.y, t.x) : INF;
                h[y] = t.x;
                e[y] = t.y;
            }
            for (int si = 0; si + 1 < nk; ++si) {
                const int k0 = key[si], k1 = key[si + 1];
                const int m1 = mask[k1];
                float nc[4], nh[4], ne[4];
                if (k1 == k0 + 1) {
                    const float2 *E = &sp.st[(bt(k0) * 4 + bt(k1)) * 16]; // E[o0 * 4 + o1]
#pragma unroll
                    for (int y = 0; y < 4; ++y) {
                        float best = INF, bh = 0.f, be = 0.f;
#pragma unroll
                        for (int x = 0; x < 4; ++x) {
                            const float2 v2 = E[x * 4 + y];
                            const float v = c[x] + fmaf(-lam, v2.y, v2.x);
                            if (v < best) {
                                best = v;
                                bh = h[x] + v2.x;
                                be = e[x] + v2.y;
                            }
                        }
                        const bool ok = (m1 >> y) & 1;
                        nc[y] = ok ? best : INF;
                        nh[y] = bh;
                        ne[y] = be;
                    }
                } else {
                    // the stack out of k0 into the fixed base after it: one argmin over
                    // the bases at k0, shared by every y; then the stack into k1
                    const int fa = __ffs(mask[k0 + 1]) - 1, fb = __ffs(mask[k1 - 1]) - 1;
                    const float2 *EA = &sp.st[(bt(k0) * 4 + bt(k0 + 1)) * 16 + fa]; // EA[o0 * 4]
                    float best = INF, bh = 0.f, be = 0.f;
#pragma unroll
                    for (int x = 0; x < 4; ++x) {
                        const float2 v2 = EA[x * 4];
                        const float v = c[x] + fmaf(-lam, v2.y, v2.x);
                        if (v < best) {
                            best = v;
                            bh = h[x] + v2.x;
                            be = e[x] + v2.y;
                        }
                    }
                    const float2 *EB = &sp.st[(bt(k1 - 1) * 4 + bt(k1)) * 16 + fb * 4]; // EB[o1]
#pragma unroll
                    for (int y = 0; y < 4; ++y) {
                        const float2 v2 = EB[y];
                        const bool ok = ((m1 >> y) & 1) && best < INF;
                        nc[y] = ok ? best + fmaf(-lam, v2.y, v2.x) : INF;
                        nh[y] = bh + v2.x;
                        ne[y] = be + v2.y;
                    }
                }
#pragma unroll
                for (int y = 0; y < 4; ++y) {
                    c[y] = nc[y];
                    h[y] = nh[y];
                    e[y] = ne[y];
                }
            }
            // the 3' terminal pair, then the argmin end state (ties: the lowest base)
            float best = INF, H = 0.f, S = 0.f;
#pragma unroll
            for (int y = 0; y < 4; ++y) {
                const float2 t = sp.tm[y * 4 + bL];
                const float v = c[y] < INF ? c[y] + fmaf(-lam, t.y, t.x) : INF;
                if (v < best) {
                    best = v;
                    H = h[y] + t.x;
                    S = e[y] + t.y;
                }
            }
            const float r = (H + SH) / (S + SE + cst);
            // stop when the ratio no longer improves by more than 1e-4 K (as tm_kernel)
            if (!(r > lam + 1e-4f))
                break;
            lam = r;
        }
        const float tm32 = lam - 273.15f + sp.tm_shift_f;
        if (pass_out && fabsf(tm32 - sp.tm_min_f) < 0.01f) {
            defer[atomicAdd(defer_n, 1ull)] = (uint32_t)i; // decided exactly by tm_kernel
            continue;
        }
        tm_out[i] = tm32;
        if (pass_out)
            pass_out[i] = tm32 >= sp.tm_min_f;
    }
}

// ---------------------------------------------------------------------------
// Tm-threshold sweep (Sec. 3.3, Annealing Temperature Optimization: amplicon
// counts, genomes amplified and off-target patterns as the threshold moves).
// Per site a bit per threshold (passes or not, decided as the fp64 definition
// decides: the fp32 maximum where it is 0.01 deg C or more from the threshold,
// else the exact fixed-point sign test of the file comment, else every oligo
// in fp64), then per amplicon the AND of its two sites' bits.
// ---------------------------------------------------------------------------

// W[(pair * n_thr + j) * 272 + e]: fixed-point weight of table entry e (256
// stacks, then 16 terminal pairs) at threshold j, in the pair's ratio units
__global__ void sweep_weights_kernel(const PairDev *__restrict__ pairs, int n_pairs, const double *__restrict__ thr_c,
                                     int n_thr, long long *__restrict__ W)
{
    const int total = n_pairs * n_thr * 272;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int e = i % 272, pj = i / 272, j = pj % n_thr, p = pj / n_thr;
        const PairDev &pd = pairs[p];
        const double thr = thr_c[j] + 273.15 - pd.tm_shift;
        W[i] = e < 256 ? fix_weight(pd.stack_dH_d[e], pd.stack_dS_d[e], thr)
                       : fix_weight(pd.term_dH_d[e - 256], pd.term_dS_d[e - 256], thr);
    }
}

// One thread per site: bit j of pass_mask[i] = site i passes threshold j.
__global__ void sweep_pass_kernel(const ah_site *__restrict__ sites, uint64_t n, const PairDev *__restrict__ pairs,
                                  const uint32_t *__restrict__ planes, const uint64_t *__restrict__ contig_off,
                                  const float *__restrict__ tm, const double *__restrict__ thr_c, int n_thr,
                                  const long long *__restrict__ W, int few_exact, uint64_t *__restrict__ pass_mask)
{
    const long long LINF = 0x2000000000000000ll;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const ah_site s = sites[i];
        const float t = tm[i];
        const PairDev &pd = pairs[s.pair];
        const int L = pd.L[s.primer];
        const uint8_t *qm = pd.mask[s.primer];
        int8_t bt[AH_MAX_PRIMER_LEN];
        bool have_bt = false;
        uint64_t m = 0;
        for (int j = 0; j < n_thr; ++j) {
            const double T = thr_c[j];
            bool pass;
            if (isnan(t)) {
                pass = false; // a template with a non-ACGT letter fails every threshold
            } else if (fabs((double)t - T) >= 0.01) {
                pass = (double)t >= T;
            } else {
                if (!have_bt) {
                    const uint64_t P = contig_off[s.contig] + s.pos;
                    for (int q = 0; q < L; ++q) {
                        const int c = base_at(planes, P + (s.strand == 0 ? q : L - 1 - q));
                        bt[q] = (int8_t)(s.strand == 0 ? 3 - c : c); // finite Tm: only A/C/G/T
                    }
                    have_bt = true;
                }
                int dec = -1;
                if (few_exact) { // sign of min over oligos of F at this threshold, exactly
                    const long long *Wp = W + ((size_t)s.pair * n_thr + j) * 272;
                    long long c[4];
                    for (int y = 0; y < 4; ++y)
                        c[y] = (qm[0] >> y & 1) ? Wp[256 + y * 4 + bt[0]] : LINF;
                    for (int q = 1; q < L; ++q) {
                        long long nc[4];
                        for (int y = 0; y < 4; ++y) {
                            long long best = LINF;
                            if (qm[q] >> y & 1)
                                for (int x = 0; x < 4; ++x)
                                    if (c[x] < LINF) {
                                        const long long v = c[x] + Wp[((x * 4 + y) * 4 + bt[q - 1]) * 4 + bt[q]];
                                        best = v < best ? v : best;
                                    }
                            nc[y] = best;
                        }
                        for (int y = 0; y < 4; ++y)
                            c[y] = nc[y];
                    }
                    long long fin = LINF;
                    for (int y = 0; y < 4; ++y)
                        if (c[y] < LINF) {
                            const long long v = c[y] + Wp[256 + y * 4 + bt[L - 1]];
                            fin = v < fin ? v : fin;
                        }
                    const double thr = T + 273.15 - pd.tm_shift;
                    const double Cp = pd.sconst + (pd.saltcorr == 5 ? 0.368 * (double)(L - 1) * pd.log_na : 0.0);
                    const long long F = fin - __double2ll_rn(thr * Cp * kFix);
                    dec = F < -kFixMargin ? 1 : (F > kFixMargin ? 0 : -1);
                }
                if (dec < 0) { // every oligo, in the definition's fp64 order
                    int deg = 1;
                    for (int q = 0; q < L; ++q)
                        deg *= __popc(qm[q]);
                    double best = -INFINITY;
                    for (int o = 0; o < deg; ++o) {
                        const double v = exact_tm(pd, bt, L, oligo_number(qm, L, o));
                        best = v > best ? v : best;
                    }
                    dec = best >= T ? 1 : 0;
                }
                pass = dec == 1;
            }
            if (pass)
                m |= 1ull << j;
        }
        pass_mask[i] = m;
    }
}

// Per amplicon: the thresholds both of its sites pass; counts per threshold
// (all, FF or RR) and, per genome, the thresholds at which it is amplified.
__global__ void sweep_count_kernel(const ah_amplicon *__restrict__ a, uint64_t na, uint64_t n_sites,
                                   const uint64_t *__restrict__ pass_mask, uint32_t max_genome, int n_thr,
                                   unsigned long long *__restrict__ amps, unsigned long long *__restrict__ ffrr,
                                   unsigned long long *__restrict__ gmask, int *__restrict__ err)
{
    __shared__ unsigned long long sa[kSweepMax], sf[kSweepMax];
    for (int j = threadIdx.x; j < kSweepMax; j += blockDim.x)
        sa[j] = sf[j] = 0;
    __syncthreads();
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < na; i += (uint64_t)gridDim.x * blockDim.x) {
        const ah_amplicon am = a[i];
        if (am.left >= n_sites || am.right >= n_sites || am.genome > max_genome || am.orient > 3) {
            atomicExch(err, kDevBounds);
            continue;
        }
        uint64_t m = pass_mask[am.left] & pass_mask[am.right];
        if (m)
            atomicOr(gmask + am.genome, (unsigned long long)m);
        while (m) {
            const int j = __ffsll((long long)m) - 1;
            m &= m - 1;
            atomicAdd(&sa[j], 1ull);
            if (am.orient >= 2)
                atomicAdd(&sf[j], 1ull);
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < n_thr; j += blockDim.x) {
        if (sa[j])
            atomicAdd(amps + j, sa[j]);
        if (sf[j])
            atomicAdd(ffrr + j, sf[j]);
    }
}

__global__ void sweep_genomes_kernel(const unsigned long long *__restrict__ gmask, uint64_t n_words, int n_thr,
                                     unsigned long long *__restrict__ gcount)
{
    __shared__ unsigned long long sg[kSweepMax];
    for (int j = threadIdx.x; j < kSweepMax; j += blockDim.x)
        sg[j] = 0;
    __syncthreads();
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_words; i += (uint64_t)gridDim.x * blockDim.x) {
        unsigned long long m = gmask[i];
        while (m) {
            const int j = __ffsll((long long)m) - 1;
            m &= m - 1;
            atomicAdd(&sg[j], 1ull);
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < n_thr; j += blockDim.x)
        if (sg[j])
            atomicAdd(gcount + j, sg[j]);
}

} // namespace

void launch_tm(const ah_site *sites, uint64_t n, const uint64_t *n_dev, const PairDev *pairs_d, int n_pairs,
               const uint32_t *planes, const uint64_t *contig_off, float *tm_out, uint8_t *pass_out, uint32_t *queue,
               uint32_t *queue_n, int seg_max, bool few_exact, int *err, cudaStream_t s)
{
    if (!n)
        return;
    if (seg_max < 1 || seg_max > AH_MAX_PRIMER_LEN - 1)
        throw Error(AH_ERR_ARG, "Tm: segment count outside 1..31");
    static int cached_dev = -1, sms = 148, fast_bps = 1, tm_bps = 1;
    int dev = 0;
    AH_CUDA(cudaGetDevice(&dev));
    const size_t smem = (size_t)n_pairs * sizeof(TmPairS) + (size_t)(n_pairs <= kTmStageD ? n_pairs : 0) * sizeof(TmPairD) +
                        (size_t)kTmWarps * 8 * seg_max * 16 * sizeof(float2);
    const size_t fast_smem = (size_t)n_pairs * sizeof(TmFastPair);
    if (dev != cached_dev) {
        AH_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        const int most = AH_MAX_PAIRS_PER_SCAN * (int)sizeof(TmPairS) + kTmStageD * (int)sizeof(TmPairD) +
                         kTmWarps * 8 * (AH_MAX_PRIMER_LEN - 1) * 16 * (int)sizeof(float2);
        AH_CUDA(cudaFuncSetAttribute(tm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, most));
        const int most_fast = AH_MAX_PAIRS_PER_SCAN * (int)sizeof(TmFastPair);
        AH_CUDA(cudaFuncSetAttribute(tm_fast_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, most_fast));
        AH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fast_bps, tm_fast_kernel, kFastThreads, most_fast));
        AH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&tm_bps, tm_kernel, 32 * kTmWarps, most));
        fast_bps = std::max(1, fast_bps);
        tm_bps = std::max(1, tm_bps);
        // AH_TM_FAST_BLOCKS=n: at most n blocks of the thread-per-site kernel per SM (profiling aid)
        if (const char *e = getenv("AH_TM_FAST_BLOCKS"))
            if (atoi(e) > 0)
                fast_bps = std::min(fast_bps, atoi(e));
        cached_dev = dev;
    }
    // queue length, finished blocks, deferred sites
    AH_CUDA(cudaMemsetAsync(queue_n, 0, 2 * sizeof(uint64_t), s));
    // Few sites (a latency-bound launch): the four-lane kernel alone finishes first
    // (measured on GB300 for 6,253 sites: 33 us, against 36 + 27 us for the two
    // kernels below); many sites: one thread per site (3.5x the four-lane rate on
    // 3.2 M sites).
    constexpr uint64_t kFastMinSites = 32768;
    if (few_exact && n >= kFastMinSites) {
        // every site in one thread; those near tm_min go to the four-lane kernel below
        uint32_t *defer = queue + n;
        unsigned long long *defer_n = reinterpret_cast<unsigned long long *>(queue_n) + 1;
        const uint64_t fb = std::min<uint64_t>((n + kFastThreads - 1) / kFastThreads, (uint64_t)sms * fast_bps);
        tm_fast_kernel<<<(unsigned)fb, kFastThreads, fast_smem, s>>>(sites, n, n_dev, pairs_d, n_pairs, planes,
                                                                      contig_off, tm_out, pass_out, defer, defer_n,
                                                                      err);
        AH_CUDA(cudaGetLastError());
        // deferred sites (few; their count stays on the device): a persistent grid
        const uint64_t tb = std::min<uint64_t>((n + 8 * kTmWarps - 1) / (8 * kTmWarps), (uint64_t)sms * tm_bps);
        tm_kernel<<<(unsigned)tb, 32 * kTmWarps, smem, s>>>(sites, n, reinterpret_cast<const uint64_t *>(defer_n),
                                                            pairs_d, n_pairs, planes, contig_off, tm_out, pass_out,
                                                            queue, queue_n, seg_max, 1, err, defer);
        AH_CUDA(cudaGetLastError());
        return;
    }
    const uint64_t per_block = 8ull * kTmWarps; // sites per block per pass
    uint64_t blocks = (n + per_block - 1) / per_block;
    if (blocks > 65535)
        blocks = 65535;
    tm_kernel<<<(unsigned)blocks, 32 * kTmWarps, smem, s>>>(sites, n, n_dev, pairs_d, n_pairs, planes, contig_off,
                                                            tm_out, pass_out, queue, queue_n, seg_max,
                                                            few_exact ? 1 : 0, err, nullptr);
    AH_CUDA(cudaGetLastError());
    if (few_exact)
        return;
    tm_exact_kernel<<<(unsigned)sms, kExactThreads, 0, s>>>(sites, pairs_d, planes, contig_off, queue, queue_n,
                                                              tm_out, pass_out);
    AH_CUDA(cudaGetLastError());
}

// Sweep: counts[0..n_thr) amplicons, [64..64+n_thr) FF/RR, [128..128+n_thr)
// genomes; counts and gmask (max_genome + 1 words) zeroed here.
void launch_tm_sweep(const ah_site *sites, uint64_t n_sites, const ah_amplicon *amps, uint64_t n_amps,
                     const PairDev *pairs_d, int n_pairs, const uint32_t *planes, const uint64_t *contig_off,
                     const float *tm, const double *thr_d, int n_thr, long long *W, bool few_exact,
                     uint64_t *pass_mask, unsigned long long *gmask, uint32_t max_genome, unsigned long long *counts,
                     int *err, cudaStream_t s)
{
    if (n_thr < 1 || n_thr > kSweepMax)
        throw Error(AH_ERR_ARG, "sweep: 1..64 thresholds");
    AH_CUDA(cudaMemsetAsync(counts, 0, 3 * kSweepMax * sizeof(unsigned long long), s));
    AH_CUDA(cudaMemsetAsync(gmask, 0, ((uint64_t)max_genome + 1) * sizeof(unsigned long long), s));
    sweep_weights_kernel<<<(n_pairs * n_thr * 272 + 255) / 256, 256, 0, s>>>(pairs_d, n_pairs, thr_d, n_thr, W);
    AH_CUDA(cudaGetLastError());
    if (n_sites) {
        const uint64_t blocks = std::min<uint64_t>((n_sites + 127) / 128, 8192);
        sweep_pass_kernel<<<(unsigned)blocks, 128, 0, s>>>(sites, n_sites, pairs_d, planes, contig_off, tm, thr_d,
                                                           n_thr, W, few_exact ? 1 : 0, pass_mask);
        AH_CUDA(cudaGetLastError());
    }
    if (n_amps) {
        const uint64_t blocks = std::min<uint64_t>((n_amps + 255) / 256, 4096);
        sweep_count_kernel<<<(unsigned)blocks, 256, 0, s>>>(amps, n_amps, n_sites, pass_mask, max_genome, n_thr,
                                                            counts, counts + kSweepMax, gmask, err);
        AH_CUDA(cudaGetLastError());
    }
    const uint64_t words = (uint64_t)max_genome + 1;
    const uint64_t blocks = std::min<uint64_t>((words + 255) / 256, 1024);
    sweep_genomes_kernel<<<(unsigned)blocks, 256, 0, s>>>(gmask, words, n_thr, counts + 2 * kSweepMax);
    AH_CUDA(cudaGetLastError());
}

} // namespace ah
