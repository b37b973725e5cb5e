// Profile-HMM homology scores of amplicons (Sec. 2.1, Amplicon analysis,
// item 2: a profile HMM trained on amplicons whose primers match exactly
// scores every predicted amplicon).
//
// Profile (built on the host, build_profile): the most frequent training
// sequence is the reference (first occurrence on ties); every training
// sequence is aligned to it globally with unit costs (equal A/C/G/T letters
// cost 0, any other pair 1, a gap 1), the traceback preferring a diagonal
// step, then a step that consumes a letter of the sequence (an insertion
// after the current column), then a step that consumes a column (a
// deletion); the state path of each alignment (B = M_0, M_j, I_j, D_j, E)
// gives transition counts from every state to the next column's M (E after
// column m), to I_j and to the next column's D, and letter counts for each
// match column; probabilities are counts + 1 normalised over the allowed
// moves (and over A/C/G/T); insert states emit the background.  Scores are
// bits against the uniform background: log2(p / (1/4)) for match emissions
// (0 for an unknown letter), 0 for insert emissions, log2 p for moves.
//
// Scores (hmm_score_kernel): the glocal Viterbi log-odds score of each
// amplicon's sequence (as ah_fetch returns it) against the profile, fp32, or
// the glocal Forward score: the same recurrence with the maximum of the
// predecessors replaced by log2(2^a + 2^b) (the log-sum semiring).
// Two kernels compute the same recurrence.
//
// hmm_wave_kernel (the Forward scores' default): one warp per amplicon, no
// block barriers.  The
// profile's columns are cut into stripes of 32 * K; within a stripe lane l
// owns K consecutive columns with their 13 scores in registers and, at step
// s, computes row i = s - l (an anti-diagonal wavefront): M and I of its
// columns from its own previous row, the delete chain along its K columns.
// The left neighbour's last column arrives by one shuffle per state (its row
// i from the previous step; its row i - 1 is kept from the step before).
// Lane 0 takes column (stripe start - 1) from the previous stripe, whose
// lane 31 wrote it per row to a per-warp boundary buffer in global memory;
// the warp loads it 32 rows at a time (one row per lane, two blocks ahead of
// use) and hands row i to lane 0 by shuffle at step i (row i is overwritten
// at step i + 31, after its block was loaded).  A stripe
// costs len + 32 steps, so the wavefront's fill and drain are 31 steps per
// stripe.
//
// hmm_score_kernel (the Viterbi scores' default; AH_HMM_KERNEL=rows or =wave
// forces one kernel for both scores): a block scores a group of amplicons
// of similar length in lockstep, rows = sequence letters: each thread owns K
// consecutive profile columns with their 13 scores in registers; M and I of a
// row depend only on the previous row (the left neighbour's values come by
// shuffle, or through shared memory across warps); the delete chain
// D_j = max(E_j, D_{j-1} + t_DD) is a block-wide scan in the (max, +)
// semiring over (t_DD, E_j) pairs (for the Forward score, in (log-sum, +)).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "ah_internal.h"
#include "hmm.h"

namespace ah {
namespace {

int letter_code(char c)
{
    switch (c) {
    case 'A': case 'a': return 0;
    case 'C': case 'c': return 1;
    case 'G': case 'g': return 2;
    case 'T': case 't': return 3;
    default: return 4;
    }
}

enum { kM = 0, kI = 1, kD = 2 };

} // namespace

void build_profile(const char *seqs, const uint64_t *off, uint64_t n, HmmProfile &p)
{
    // the reference: most frequent sequence, first occurrence on ties (by hashing)
    std::map<std::string, std::pair<uint64_t, uint64_t>> freq; // sequence -> (count, first index)
    for (uint64_t q = 0; q < n; ++q) {
        std::string s(seqs + off[q], seqs + off[q + 1]);
        auto it = freq.find(s);
        if (it == freq.end())
            freq.emplace(std::move(s), std::make_pair(1ull, q));
        else
            ++it->second.first;
    }
    uint64_t best_q = 0, best_n = 0;
    for (const auto &kv : freq)
        if (kv.second.first > best_n || (kv.second.first == best_n && kv.second.second < best_q)) {
            best_n = kv.second.first;
            best_q = kv.second.second;
        }
    const char *R = seqs + off[best_q];
    const int64_t m = (int64_t)(off[best_q + 1] - off[best_q]);
    p.m = (int)m;
    p.reference = best_q;
    std::vector<double> ct((size_t)(m + 1) * 9, 0.0), ce((size_t)(m + 1) * 4, 0.0);
    std::vector<int> rc(m);
    for (int64_t j = 0; j < m; ++j)
        rc[j] = letter_code(R[j]);
    std::vector<uint32_t> dist; // (len + 1) x (m + 1) alignment costs
    std::vector<uint8_t> moves;
    for (uint64_t q = 0; q < n; ++q) {
        const char *S = seqs + off[q];
        const int64_t ls = (int64_t)(off[q + 1] - off[q]);
        const int64_t W = m + 1;
        dist.assign((size_t)(ls + 1) * W, 0);
        for (int64_t j = 0; j <= m; ++j)
            dist[j] = (uint32_t)j;
        for (int64_t i = 1; i <= ls; ++i) {
            const int si = letter_code(S[i - 1]);
            uint32_t *row = &dist[i * W];
            const uint32_t *up = &dist[(i - 1) * W];
            row[0] = (uint32_t)i;
            for (int64_t j = 1; j <= m; ++j) {
                const uint32_t sub = up[j - 1] + ((si < 4 && si == rc[j - 1]) ? 0u : 1u);
                row[j] = std::min(sub, std::min(up[j], row[j - 1]) + 1u);
            }
        }
        moves.clear();
        int64_t i = ls, j = m;
        while (i > 0 || j > 0) {
            const uint32_t here = dist[i * W + j];
            if (i > 0 && j > 0) {
                const int si = letter_code(S[i - 1]);
                const uint32_t sub = dist[(i - 1) * W + j - 1] + ((si < 4 && si == rc[j - 1]) ? 0u : 1u);
                if (here == sub) {
                    moves.push_back(kM);
                    --i;
                    --j;
                    continue;
                }
            }
            if (i > 0 && here == dist[(i - 1) * W + j] + 1u) {
                moves.push_back(kI);
                --i;
            } else {
                moves.push_back(kD);
                --j;
            }
        }
        int from = kM; // B = M_0
        int64_t col = 0, pos = 0;
        for (auto it = moves.rbegin(); it != moves.rend(); ++it) {
            const int to = *it;
            ct[(size_t)col * 9 + from * 3 + to] += 1.0;
            if (to == kM) {
                ++col;
                const int l = letter_code(S[pos]);
                if (l < 4)
                    ce[(size_t)col * 4 + l] += 1.0;
                ++pos;
            } else if (to == kI) {
                ++pos;
            } else {
                ++col;
            }
            from = to;
        }
        ct[(size_t)col * 9 + from * 3 + kM] += 1.0; // to E
    }
    p.t.assign((size_t)(m + 1) * 9, -INFINITY);
    p.e.assign((size_t)(m + 1) * 4, 0.0f);
    for (int64_t j = 0; j <= m; ++j) {
        for (int x = 0; x < 3; ++x) {
            if (j == 0 && x == kD)
                continue; // D_0 does not exist
            const bool has_d = j < m;
            double tot = 0.0;
            for (int y = 0; y < 3; ++y)
                if (y != kD || has_d)
                    tot += ct[(size_t)j * 9 + x * 3 + y] + 1.0;
            for (int y = 0; y < 3; ++y)
                if (y != kD || has_d)
                    p.t[(size_t)j * 9 + x * 3 + y] = (float)std::log2((ct[(size_t)j * 9 + x * 3 + y] + 1.0) / tot);
        }
        if (j > 0) {
            const double tot = ce[j * 4] + ce[j * 4 + 1] + ce[j * 4 + 2] + ce[j * 4 + 3] + 4.0;
            for (int l = 0; l < 4; ++l)
                p.e[(size_t)j * 4 + l] = (float)std::log2((ce[(size_t)j * 4 + l] + 1.0) / tot * 4.0);
        }
    }
}

namespace {

constexpr int kHmmThreads = 512;
constexpr float kNeg = -INFINITY;

// The semiring's "sum" of two log2 scores: Viterbi takes the larger, Forward
// log2(2^a + 2^b) (exp2f and the __log2f intrinsic of CUDA's math library).
struct MaxSum {
    __device__ static __forceinline__ float add(float a, float b) { return fmaxf(a, b); }
};
struct LogSum {
    __device__ static __forceinline__ float add(float a, float b)
    {
        const float hi = fmaxf(a, b), lo = fminf(a, b);
        if (lo == kNeg) // also both -inf
            return hi;
        return hi + __log2f(1.0f + exp2f(lo - hi)); // 1 + 2^d in [1, 2]: absolute error ~2^-22
    }
};

// Letter codes of amplicon `am` (as fetched: RF reverse-complemented) into seq.
__device__ void decode_letters(const ah_amplicon &am, const uint32_t *__restrict__ planes,
                               const uint64_t *__restrict__ contig_off, uint8_t *seq, int len)
{
    const uint64_t base = contig_off[am.contig] + am.start;
    const bool rc = am.orient == 1;
    for (int q = threadIdx.x; q < len; q += blockDim.x) {
        const uint64_t P = base + (rc ? (uint64_t)(len - 1 - q) : (uint64_t)q);
        const uint64_t t = P / kTileBases, r = P % kTileBases;
        const int b = (int)(r / kTileW), j = (int)(r % kTileW);
        const uint32_t *w = planes + t * 4 * kTileWX + j;
        int code = 4;
#pragma unroll
        for (int x = 0; x < 4; ++x)
            if ((__ldg(w + x * kTileWX) >> b) & 1u)
                code = x;
        if (code < 4 && rc)
            code = 3 - code;
        seq[q] = (uint8_t)code;
    }
}

// A amplicons per block, in lockstep over rows (the host groups amplicons of
// similar length): the barriers of a row serve A rows of work.  The delete
// chain's (max, +) pairs share their t_DD part across the A amplicons.
template <class Op, int K, int A, int NT>
__global__ void __launch_bounds__(NT) hmm_score_kernel(const ah_amplicon *__restrict__ amps,
                                                                  const uint32_t *__restrict__ order, uint64_t n_amps,
                                                                  const uint32_t *__restrict__ planes,
                                                                  const uint64_t *__restrict__ contig_off,
                                                                  uint32_t n_contigs, const float *__restrict__ t,
                                                                  const float *__restrict__ e, int m, int max_len,
                                                                  float *__restrict__ score_out, int *__restrict__ err)
{
    extern __shared__ uint8_t seq[];                    // A x max_len letter codes
    __shared__ float edge_prev[A][3][NT / 32]; // M, I, D of each warp's last column, previous row
    __shared__ float edge_cur[A][2][NT / 32];  // M, I of each warp's last column, current row
    __shared__ float wtot_a[NT / 32], wtot_b[A][NT / 32];
    __shared__ float wpre_a[NT / 32], wpre_b[A][NT / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int c0 = threadIdx.x * K;
    // this thread's columns: scores of the moves into M_j (from j-1), into D_j
    // (from j-1) and into I_j (from j), and M_j's emissions
    float toM[K][3], toD[K][3], toI[K][3], em[K][4];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int j = c0 + k;
#pragma unroll
        for (int x = 0; x < 3; ++x) {
            toM[k][x] = (j >= 1 && j <= m) ? t[(j - 1) * 9 + x * 3 + 0] : kNeg;
            toD[k][x] = (j >= 1 && j <= m) ? t[(j - 1) * 9 + x * 3 + 2] : kNeg;
            toI[k][x] = (j <= m) ? t[j * 9 + x * 3 + 1] : kNeg;
        }
#pragma unroll
        for (int l = 0; l < 4; ++l)
            em[k][l] = (j >= 1 && j <= m) ? e[j * 4 + l] : 0.0f;
    }
    // the delete chain's t_DD prefix of this thread's columns (the same for every amplicon)
    float tdd_sum = 0.0f;
#pragma unroll
    for (int k = 0; k < K; ++k)
        tdd_sum += toD[k][kD];
    const uint64_t n_groups = (n_amps + A - 1) / A;
    for (uint64_t gi = blockIdx.x; gi < n_groups; gi += gridDim.x) {
        int len[A];
        uint32_t idx[A];
        int rows = 0;
        __syncthreads(); // the previous group's letters are no longer read
#pragma unroll
        for (int s = 0; s < A; ++s) {
            const uint64_t q = gi * A + s;
            len[s] = -1; // -1: no amplicon in this slot
            idx[s] = 0;
            if (q < n_amps) {
                idx[s] = order[q];
                const ah_amplicon am = amps[idx[s]];
                bool ok = am.contig < n_contigs && am.start <= am.end;
                if (ok)
                    ok = (uint64_t)am.end <= contig_off[am.contig + 1] - contig_off[am.contig] &&
                         am.end - am.start <= (uint32_t)max_len;
                if (ok) {
                    len[s] = (int)(am.end - am.start);
                    decode_letters(am, planes, contig_off, seq + s * max_len, len[s]);
                    rows = max(rows, len[s]);
                } else if (threadIdx.x == 0) { // checked on the host; reported, not read
                    atomicExch(err, kDevBounds);
                    score_out[idx[s]] = kNeg;
                }
            }
        }
        float pM[A][K], pI[A][K], pD[A][K];
#pragma unroll
        for (int s = 0; s < A; ++s)
#pragma unroll
            for (int k = 0; k < K; ++k) {
                pM[s][k] = (c0 + k == 0) ? 0.0f : kNeg;
                pI[s][k] = kNeg;
                pD[s][k] = kNeg;
            }
        // the delete chains of a row from its M and I values
        auto delete_chain = [&](const float (&cM)[A][K], const float (&cI)[A][K], float (&cD)[A][K]) {
            float lM[A], lI[A];
#pragma unroll
            for (int s = 0; s < A; ++s) {
                lM[s] = __shfl_up_sync(0xffffffffu, cM[s][K - 1], 1);
                lI[s] = __shfl_up_sync(0xffffffffu, cI[s][K - 1], 1);
                if (lane == 31) {
                    edge_cur[s][0][warp] = cM[s][K - 1];
                    edge_cur[s][1][warp] = cI[s][K - 1];
                }
            }
            __syncthreads();
            if (lane == 0)
#pragma unroll
                for (int s = 0; s < A; ++s) {
                    lM[s] = warp > 0 ? edge_cur[s][0][warp - 1] : kNeg;
                    lI[s] = warp > 0 ? edge_cur[s][1][warp - 1] : kNeg;
                }
            // per column: D_j = max(b_j, D_{j-1} + a_j); thread aggregate (a, b[s])
            float eb[A][K], agg_b[A];
#pragma unroll
            for (int s = 0; s < A; ++s) {
                float acc = kNeg;
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const float pm = k ? cM[s][k - 1] : lM[s], pi = k ? cI[s][k - 1] : lI[s];
                    eb[s][k] = Op::add(pm + toD[k][kM], pi + toD[k][kI]);
                    acc = Op::add(eb[s][k], acc + toD[k][kD]);
                }
                agg_b[s] = acc;
            }
            // inclusive warp scan: (a1, b1) then (a2, b2) = (a1 + a2, max(b2, b1 + a2))
            float inc_a = tdd_sum, inc_b[A];
#pragma unroll
            for (int s = 0; s < A; ++s)
                inc_b[s] = agg_b[s];
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const float oa = __shfl_up_sync(0xffffffffu, inc_a, d);
#pragma unroll
                for (int s = 0; s < A; ++s) {
                    const float ob = __shfl_up_sync(0xffffffffu, inc_b[s], d);
                    if (lane >= d)
                        inc_b[s] = Op::add(inc_b[s], ob + inc_a);
                }
                if (lane >= d)
                    inc_a = oa + inc_a;
            }
            if (lane == 31) {
                wtot_a[warp] = inc_a;
#pragma unroll
                for (int s = 0; s < A; ++s)
                    wtot_b[s][warp] = inc_b[s];
            }
            __syncthreads();
            if (warp == 0) {
                float wa = lane < nwarps ? wtot_a[lane] : 0.0f, wb[A];
#pragma unroll
                for (int s = 0; s < A; ++s)
                    wb[s] = lane < nwarps ? wtot_b[s][lane] : kNeg;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const float oa = __shfl_up_sync(0xffffffffu, wa, d);
#pragma unroll
                    for (int s = 0; s < A; ++s) {
                        const float ob = __shfl_up_sync(0xffffffffu, wb[s], d);
                        if (lane >= d)
                            wb[s] = Op::add(wb[s], ob + wa);
                    }
                    if (lane >= d)
                        wa = oa + wa;
                }
                // exclusive prefix of the warps
                const float xa = __shfl_up_sync(0xffffffffu, wa, 1);
                if (lane < nwarps)
                    wpre_a[lane] = lane ? xa : 0.0f;
#pragma unroll
                for (int s = 0; s < A; ++s) {
                    const float xb = __shfl_up_sync(0xffffffffu, wb[s], 1);
                    if (lane < nwarps)
                        wpre_b[s][lane] = lane ? xb : kNeg;
                }
            }
            __syncthreads();
            // this thread's exclusive prefix = (warps before) then (lanes before)
            const float xa = __shfl_up_sync(0xffffffffu, inc_a, 1);
#pragma unroll
            for (int s = 0; s < A; ++s) {
                float xb = __shfl_up_sync(0xffffffffu, inc_b[s], 1);
                if (lane == 0)
                    xb = kNeg;
                const float lane_a = lane ? xa : 0.0f;
                float d = Op::add(xb, wpre_b[s][warp] + lane_a); // D at column c0 - 1
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    d = Op::add(eb[s][k], d + toD[k][kD]);
                    cD[s][k] = d;
                }
            }
        };
        auto finish = [&](int i) { // amplicons whose last row is i: the holder of column m scores them
#pragma unroll
            for (int s = 0; s < A; ++s)
                if (len[s] == i)
#pragma unroll
                    for (int k = 0; k < K; ++k)
                        if (c0 + k == m)
                            score_out[idx[s]] =
                                Op::add(Op::add(pM[s][k] + t[m * 9 + kM * 3], pI[s][k] + t[m * 9 + kI * 3]),
                                      pD[s][k] + t[m * 9 + kD * 3]);
        };
        __syncthreads(); // the letters are decoded
        delete_chain(pM, pI, pD);
        finish(0);
        for (int i = 1; i <= rows; ++i) {
            float lM[A], lI[A], lD[A];
#pragma unroll
            for (int s = 0; s < A; ++s) {
                lM[s] = __shfl_up_sync(0xffffffffu, pM[s][K - 1], 1);
                lI[s] = __shfl_up_sync(0xffffffffu, pI[s][K - 1], 1);
                lD[s] = __shfl_up_sync(0xffffffffu, pD[s][K - 1], 1);
                if (lane == 31) {
                    edge_prev[s][0][warp] = pM[s][K - 1];
                    edge_prev[s][1][warp] = pI[s][K - 1];
                    edge_prev[s][2][warp] = pD[s][K - 1];
                }
            }
            __syncthreads();
            if (lane == 0)
#pragma unroll
                for (int s = 0; s < A; ++s) {
                    lM[s] = warp > 0 ? edge_prev[s][0][warp - 1] : kNeg;
                    lI[s] = warp > 0 ? edge_prev[s][1][warp - 1] : kNeg;
                    lD[s] = warp > 0 ? edge_prev[s][2][warp - 1] : kNeg;
                }
            float cM[A][K], cI[A][K], cD[A][K];
#pragma unroll
            for (int s = 0; s < A; ++s) {
                const int x = i <= len[s] ? seq[s * max_len + i - 1] : 4;
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const float qm = k ? pM[s][k - 1] : lM[s], qi = k ? pI[s][k - 1] : lI[s],
                                qd = k ? pD[s][k - 1] : lD[s];
                    // (a select, not an indexed load: the emission scores stay in registers)
                    const float ex = x == 0 ? em[k][0] : x == 1 ? em[k][1] : x == 2 ? em[k][2] : x == 3 ? em[k][3] : 0.0f;
                    cM[s][k] = ex + Op::add(Op::add(qm + toM[k][kM], qi + toM[k][kI]), qd + toM[k][kD]);
                    cI[s][k] = Op::add(Op::add(pM[s][k] + toI[k][kM], pI[s][k] + toI[k][kI]), pD[s][k] + toI[k][kD]);
                }
            }
            delete_chain(cM, cI, cD);
#pragma unroll
            for (int s = 0; s < A; ++s)
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    pM[s][k] = cM[s][k];
                    pI[s][k] = cI[s][k];
                    pD[s][k] = cD[s][k];
                }
            finish(i);
        }
    }
}

// NT: the most threads a block may have (the register budget per thread follows from it)
template <class Op, int K, int A, int NT>
bool launch_k(const ah_amplicon *amps, const uint32_t *order, uint64_t n, const uint32_t *planes,
              const uint64_t *contig_off, uint32_t n_contigs, const float *t, const float *e, int m, int max_len,
              float *out, int *err, int sms, cudaStream_t s)
{
    const int threads = 32 * (((m + 1) + 32 * K - 1) / (32 * K));
    if (threads > NT)
        return false; // the profile needs more columns than this variant holds
    const size_t smem = (size_t)A * (size_t)max_len;
    AH_CUDA(cudaFuncSetAttribute(hmm_score_kernel<Op, K, A, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)std::max<size_t>(smem, 1)));
    int per_sm = 1;
    AH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hmm_score_kernel<Op, K, A, NT>, threads, smem));
    const uint64_t groups = (n + A - 1) / A;
    const uint64_t blocks = std::min<uint64_t>(groups, (uint64_t)sms * (uint64_t)std::max(1, per_sm));
    hmm_score_kernel<Op, K, A, NT><<<(unsigned)blocks, threads, smem, s>>>(amps, order, n, planes, contig_off,
                                                                          n_contigs, t, e, m, max_len, out, err);
    AH_CUDA(cudaGetLastError());
    return true;
}

// Letter codes of amplicon `am` into seq, the warp's lanes in turn.
__device__ void decode_letters_warp(const ah_amplicon &am, const uint32_t *__restrict__ planes,
                                    const uint64_t *__restrict__ contig_off, uint8_t *seq, int len, int lane)
{
    const uint64_t base = contig_off[am.contig] + am.start;
    const bool rc = am.orient == 1;
    for (int q = lane; q < len; q += 32) {
        const uint64_t P = base + (rc ? (uint64_t)(len - 1 - q) : (uint64_t)q);
        const uint64_t tt = P / kTileBases, r = P % kTileBases;
        const int b = (int)(r / kTileW), j = (int)(r % kTileW);
        const uint32_t *w = planes + tt * 4 * kTileWX + j;
        int code = 4;
#pragma unroll
        for (int x = 0; x < 4; ++x)
            if ((__ldg(w + x * kTileWX) >> b) & 1u)
                code = x;
        if (code < 4 && rc)
            code = 3 - code;
        seq[q] = (uint8_t)code;
    }
}

constexpr int kWaveWarps = 4;        // warps (amplicons in flight) per block
constexpr int kWaveBlocksPerSm = 8;  // grid: at most this many blocks per SM
constexpr uint64_t kWaveScratchMax = 256ull << 20;

// One warp per amplicon; lanes over the columns of a stripe, steps over
// anti-diagonals (see the head of this file).  bnd_all: 3 * (max_len + 1)
// floats per warp of the grid (M, I, D of the column left of the stripe, per
// row).
template <class Op, int K>
__global__ void __launch_bounds__(32 * kWaveWarps) hmm_wave_kernel(
    const ah_amplicon *__restrict__ amps, const uint32_t *__restrict__ order, uint64_t n_amps,
    const uint32_t *__restrict__ planes, const uint64_t *__restrict__ contig_off, uint32_t n_contigs,
    const float *__restrict__ t, const float *__restrict__ e, int m, int max_len, float *__restrict__ bnd_all,
    float *__restrict__ score_out, int *__restrict__ err)
{
    extern __shared__ uint8_t wave_seq[]; // kWaveWarps x seq_stride letter codes
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int seq_stride = (max_len + 15) & ~15;
    uint8_t *seq = wave_seq + warp * seq_stride;
    const uint64_t slot = (uint64_t)blockIdx.x * kWaveWarps + warp;
    float *bnd = bnd_all + slot * 3ull * (uint64_t)(max_len + 1);
    constexpr int span = 32 * K;
    const int n_stripes = (m + 1 + span - 1) / span;
    const float endM = t[m * 9 + kM * 3], endI = t[m * 9 + kI * 3], endD = t[m * 9 + kD * 3];
    for (uint64_t q = slot; q < n_amps; q += (uint64_t)gridDim.x * kWaveWarps) {
        const uint32_t idx = order[q];
        const ah_amplicon am = amps[idx];
        bool ok = am.contig < n_contigs && am.start <= am.end;
        if (ok)
            ok = (uint64_t)am.end <= contig_off[am.contig + 1] - contig_off[am.contig] &&
                 am.end - am.start <= (uint32_t)max_len;
        if (!ok) { // checked on the host; reported, not read
            if (lane == 0) {
                atomicExch(err, kDevBounds);
                score_out[idx] = kNeg;
            }
            continue;
        }
        const int len = (int)(am.end - am.start);
        __syncwarp(); // the previous amplicon's letters are no longer read
        decode_letters_warp(am, planes, contig_off, seq, len, lane);
        __syncwarp();
        for (int s = 0; s < n_stripes; ++s) {
            const int c0 = s * span + lane * K;
            // scores of the moves into M_j (from j-1), into D_j (from j-1), into I_j (from j); M_j's emissions
            float toM[K][3], toD[K][3], toI[K][3], em[K][4];
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const int j = c0 + k;
#pragma unroll
                for (int x = 0; x < 3; ++x) {
                    toM[k][x] = (j >= 1 && j <= m) ? t[(j - 1) * 9 + x * 3 + 0] : kNeg;
                    toD[k][x] = (j >= 1 && j <= m) ? t[(j - 1) * 9 + x * 3 + 2] : kNeg;
                    toI[k][x] = (j <= m) ? t[j * 9 + x * 3 + 1] : kNeg;
                }
#pragma unroll
                for (int l = 0; l < 4; ++l)
                    em[k][l] = (j >= 1 && j <= m) ? e[j * 4 + l] : 0.0f;
            }
            float pM[K], pI[K], pD[K]; // this lane's columns at its previous row
#pragma unroll
            for (int k = 0; k < K; ++k)
                pM[k] = pI[k] = pD[k] = kNeg;
            float lpM = kNeg, lpI = kNeg, lpD = kNeg; // column c0 - 1 at the previous row
            float oM = kNeg, oI = kNeg, oD = kNeg;    // this lane's last column at its latest row
            const bool last_stripe = s + 1 == n_stripes;
            // the previous stripe's boundary, 32 rows per block, row 32 b + lane in each lane:
            // the block in use and the next one (loaded 32 steps before lane 0 needs it)
            float bM, bI, bD, nM, nI, nD;
            auto load_block = [&](int blk, float &M_, float &I_, float &D_) {
                const int r = blk * 32 + lane;
                M_ = I_ = D_ = kNeg;
                if (s > 0 && r <= len) {
                    M_ = bnd[3 * r];
                    I_ = bnd[3 * r + 1];
                    D_ = bnd[3 * r + 2];
                }
            };
            load_block(0, bM, bI, bD);
            load_block(1, nM, nI, nD);
            for (int st = 0; st < len + 32; ++st) {
                const int i = st - lane;
                // column c0 - 1 at row i: the left lane's latest row, or the previous stripe's boundary
                float rM = __shfl_up_sync(0xffffffffu, oM, 1);
                float rI = __shfl_up_sync(0xffffffffu, oI, 1);
                float rD = __shfl_up_sync(0xffffffffu, oD, 1);
                if (s > 0) {
                    const float gM = __shfl_sync(0xffffffffu, bM, st & 31);
                    const float gI = __shfl_sync(0xffffffffu, bI, st & 31);
                    const float gD = __shfl_sync(0xffffffffu, bD, st & 31);
                    if (lane == 0) {
                        rM = gM;
                        rI = gI;
                        rD = gD;
                    }
                    if ((st & 31) == 31) { // rows 32 b + 64 .. are not yet overwritten (row r at step r + 31)
                        bM = nM;
                        bI = nI;
                        bD = nD;
                        load_block((st >> 5) + 2, nM, nI, nD);
                    }
                } else if (lane == 0) {
                    rM = rI = rD = kNeg;
                }
                if (i < 0 || i > len)
                    continue;
                float cM[K], cI[K], cD[K];
                if (i == 0) { // B = M_0 at row 0; no letter consumed yet
#pragma unroll
                    for (int k = 0; k < K; ++k) {
                        cM[k] = (c0 + k == 0) ? 0.0f : kNeg;
                        cI[k] = kNeg;
                    }
                } else {
                    const int x = seq[i - 1];
#pragma unroll
                    for (int k = 0; k < K; ++k) {
                        const float qm = k ? pM[k - 1] : lpM, qi = k ? pI[k - 1] : lpI, qd = k ? pD[k - 1] : lpD;
                        // (a select, not an indexed load: the emission scores stay in registers)
                        const float ex =
                            x == 0 ? em[k][0] : x == 1 ? em[k][1] : x == 2 ? em[k][2] : x == 3 ? em[k][3] : 0.0f;
                        cM[k] = ex + Op::add(Op::add(qm + toM[k][kM], qi + toM[k][kI]), qd + toM[k][kD]);
                        cI[k] = Op::add(Op::add(pM[k] + toI[k][kM], pI[k] + toI[k][kI]), pD[k] + toI[k][kD]);
                    }
                }
                // the delete chain along the row
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const float lm = k ? cM[k - 1] : rM, li = k ? cI[k - 1] : rI, ld = k ? cD[k - 1] : rD;
                    cD[k] = Op::add(Op::add(lm + toD[k][kM], li + toD[k][kI]), ld + toD[k][kD]);
                }
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    pM[k] = cM[k];
                    pI[k] = cI[k];
                    pD[k] = cD[k];
                }
                lpM = rM;
                lpI = rI;
                lpD = rD;
                oM = cM[K - 1];
                oI = cI[K - 1];
                oD = cD[K - 1];
                if (lane == 31 && !last_stripe) {
                    bnd[3 * i] = oM;
                    bnd[3 * i + 1] = oI;
                    bnd[3 * i + 2] = oD;
                }
                if (i == len && last_stripe)
#pragma unroll
                    for (int k = 0; k < K; ++k)
                        if (c0 + k == m)
                            score_out[idx] = Op::add(Op::add(cM[k] + endM, cI[k] + endI), cD[k] + endD);
            }
            __syncwarp(); // the stripe's boundary is written before the next stripe reads it
        }
    }
}

uint64_t wave_blocks(uint64_t n, int max_len, int sms)
{
    const uint64_t per_block = (uint64_t)kWaveWarps * 3ull * (uint64_t)(max_len + 1) * sizeof(float);
    uint64_t b = std::min<uint64_t>((n + kWaveWarps - 1) / kWaveWarps, (uint64_t)sms * kWaveBlocksPerSm);
    b = std::min<uint64_t>(b, std::max<uint64_t>((uint64_t)sms, kWaveScratchMax / per_block));
    return std::max<uint64_t>(b, 1);
}

template <class Op, int K>
void launch_wave(const ah_amplicon *amps, const uint32_t *order, uint64_t n, const uint32_t *planes,
                 const uint64_t *contig_off, uint32_t n_contigs, const float *t, const float *e, int m, int max_len,
                 float *bnd, float *out, int *err, int sms, cudaStream_t s)
{
    const size_t smem = (size_t)kWaveWarps * (size_t)((max_len + 15) & ~15);
    AH_CUDA(cudaFuncSetAttribute(hmm_wave_kernel<Op, K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)std::max<size_t>(smem, 1)));
    const uint64_t blocks = wave_blocks(n, max_len, sms);
    hmm_wave_kernel<Op, K><<<(unsigned)blocks, 32 * kWaveWarps, smem, s>>>(amps, order, n, planes, contig_off,
                                                                           n_contigs, t, e, m, max_len, bnd, out, err);
    AH_CUDA(cudaGetLastError());
}

} // namespace

size_t hmm_scratch_bytes(uint64_t n, int max_len, int sms)
{
    return wave_blocks(n, max_len, sms) * (uint64_t)kWaveWarps * 3ull * (uint64_t)(max_len + 1) * sizeof(float);
}

bool hmm_use_wave(bool forward)
{
    // measured on 639 columns x 5,023 amplicons: Forward 108 GCUPS on the wavefront against 91 on
    // the block kernel; Viterbi 310 against 457
    const char *kern = getenv("AH_HMM_KERNEL");
    if (kern && strcmp(kern, "rows") == 0)
        return false;
    if (kern && strcmp(kern, "wave") == 0)
        return true;
    return forward;
}

void launch_hmm_wave(const ah_amplicon *amps, const uint32_t *order, uint64_t n, const uint32_t *planes,
                     const uint64_t *contig_off, uint32_t n_contigs, const float *t, const float *e, int m,
                     int max_len, bool forward, float *bnd, float *score_out, int *err, int sms, cudaStream_t s)
{
    if (n == 0)
        return;
    if (m + 1 > kHmmMaxColumns)
        throw Error(AH_ERR_ARG, "ah_hmm_score: profile longer than " + std::to_string(kHmmMaxColumns) + " columns");
    if (forward)
        launch_wave<LogSum, 4>(amps, order, n, planes, contig_off, n_contigs, t, e, m, max_len, bnd, score_out, err,
                               sms, s);
    else
        launch_wave<MaxSum, 4>(amps, order, n, planes, contig_off, n_contigs, t, e, m, max_len, bnd, score_out, err,
                               sms, s);
}

void launch_hmm_score(const ah_amplicon *amps, const uint32_t *order, uint64_t n, const uint32_t *planes,
                      const uint64_t *contig_off, uint32_t n_contigs, const float *t, const float *e, int m,
                      int max_len, bool forward, float *score_out, int *err, int sms, cudaStream_t s)
{
    if (n == 0)
        return;
    const int cols = m + 1;
    // AH_HMM_VARIANT="K,A" picks columns per thread and amplicons per block (profiling aid)
    int vk = 0, va = 0;
    if (const char *v = getenv("AH_HMM_VARIANT"))
        if (sscanf(v, "%d,%d", &vk, &va) != 2)
            vk = va = 0;
#define AH_HMM_TRY_OP(OP_, K_, A_, NT_)                                                                          \
    if ((vk == 0 || (vk == K_ && va == A_)) &&                                                                   \
        launch_k<OP_, K_, A_, NT_>(amps, order, n, planes, contig_off, n_contigs, t, e, m, max_len, score_out, err, \
                                   sms, s))                                                                      \
        return;
    if (forward) { // the default variants only
        vk = va = 0;
        AH_HMM_TRY_OP(LogSum, 4, 2, 512)
        AH_HMM_TRY_OP(LogSum, 6, 1, 512)
        throw Error(AH_ERR_ARG, "ah_hmm_forward: profile longer than " + std::to_string(kHmmMaxColumns) + " columns");
    }
#define AH_HMM_TRY(K_, A_, NT_) AH_HMM_TRY_OP(MaxSum, K_, A_, NT_)
    if (vk) { // the named variant (when it covers the profile)
        AH_HMM_TRY(2, 2, 512)
        AH_HMM_TRY(4, 1, 512)
        AH_HMM_TRY(4, 2, 512)
        AH_HMM_TRY(4, 4, 256)
        AH_HMM_TRY(8, 2, 256)
        AH_HMM_TRY(8, 1, 256)
        vk = va = 0;
    }
    // default (measured on 639 columns: 4 columns x 2 amplicons 398 GCUPS; 2 x 2 272; 4 x 1 315;
    // 8 x 1 234, register-capped); longer profiles take 6 columns x 1 amplicon
    AH_HMM_TRY(4, 2, 512)
    AH_HMM_TRY(6, 1, 512)
#undef AH_HMM_TRY
#undef AH_HMM_TRY_OP
    throw Error(AH_ERR_ARG, "ah_hmm_score: profile longer than " + std::to_string(kHmmMaxColumns) + " columns");
}

} // namespace ah

// The profile of a training set without a context or a GPU (development aid:
// lets the host-side builder be compared with an independent implementation on
// machines without a GPU).  Returns 0 and writes m and the reference index;
// when t and e are not NULL they receive (m + 1) * 9 and (m + 1) * 4 scores.
// Returns 1 for no training sequence, 2 when t or e is given and m exceeds
// m_cap.
extern "C" int ah_debug_hmm_profile(const char *seqs, const uint64_t *offsets, uint64_t n, uint64_t m_cap,
                                    uint64_t *m_out, uint64_t *reference_out, float *t, float *e)
{
    if (n == 0 || !offsets || !m_out || !reference_out)
        return 1;
    ah::HmmProfile p;
    ah::build_profile(seqs, offsets, n, p);
    *m_out = (uint64_t)p.m;
    *reference_out = p.reference;
    if (t || e) {
        if ((uint64_t)p.m > m_cap)
            return 2;
        if (t)
            memcpy(t, p.t.data(), p.t.size() * sizeof(float));
        if (e)
            memcpy(e, p.e.data(), p.e.size() * sizeof(float));
    }
    return 0;
}
