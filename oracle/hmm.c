/*
 * Oracle for profile-HMM scoring of amplicons (test infrastructure only; see
 * oracle.c for the rules on who may use it).
 *
 * The paper (Sec. 2.1, Amplicon analysis, item 2) builds a profile HMM from
 * the amplicons whose primers match exactly and scores every predicted
 * amplicon against it for homology.  It names no aligner,
 * model topology or scoring mode; the reading taken here, in plain steps:
 *
 *   Profile (or_hmm_build):
 *   1. Letters: A C G T; every other letter is "unknown".
 *   2. The reference R is the most frequent training sequence (ties: the one
 *      that occurs first); m = |R| match columns.
 *   3. Each training sequence S is aligned globally to R with unit costs
 *      (0 for equal known letters, 1 for any other pair, 1 per gap).  The
 *      traceback from (|S|, m) prefers, in this order, a diagonal step, a
 *      step that consumes a letter of S only (an insertion after the current
 *      column) and a step that consumes a column of R only (a deletion).
 *   4. Reading the alignment from the start, the state path runs from the
 *      begin state B = M_0 through M_j (diagonal step at column j), I_j
 *      (insertion after column j, j = 0..m) and D_j (deleted column j) to the
 *      end state E.  From any state at position j the moves are to the next
 *      column's M_{j+1}, to I_j, or to D_{j+1}; at j = m the "next" move is E
 *      and there is no D move.  Transition counts are those of the path;
 *      match emissions count the known letters emitted by M_j.
 *   5. Probabilities: counts + 1 over the allowed moves of each state, and
 *      counts + 1 over A C G T for each match column.  Insert states emit the
 *      background (1/4 each).
 *   6. Scores in bits against the i.i.d. background 1/4: match emission
 *      log2(p / (1/4)), 0 for an unknown letter; insert emissions 0;
 *      transitions log2(probability).
 *
 *   Score (or_hmm_viterbi): the glocal Viterbi log-odds score of a sequence
 *   against the profile -- the best path from B through the states to E,
 *   every letter emitted by an M or I state -- in bits.
 *
 *   Score (or_hmm_forward): the glocal Forward log-odds score -- log2 of the
 *   sum, over every such path, of 2 to the path's score -- in bits: the same
 *   recurrence with the maximum of the three predecessors replaced by
 *   log2(2^a + 2^b + 2^c).
 *
 * Table layout shared with the tests (not with the library): per position
 * j = 0..m, 9 transition scores t[j][X][Y] with X, Y in (M, I, D) (Y = M
 * meaning the next move, which is E at j = m), -INFINITY where a move does
 * not exist; per column j = 1..m, 4 emission scores e[j][x] (e[0] unused).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { ST_M = 0, ST_I = 1, ST_D = 2 };

static int letter(char c)
{
    switch (c) {
    case 'A': case 'a': return 0;
    case 'C': case 'c': return 1;
    case 'G': case 'g': return 2;
    case 'T': case 't': return 3;
    default: return 4;
    }
}

/* 0 when both letters are the same known letter, else 1 */
static int subst_cost(char a, char b)
{
    int x = letter(a), y = letter(b);
    return (x < 4 && x == y) ? 0 : 1;
}

/* Unit-cost global alignment distance (exported for the pins). */
int64_t or_edit_distance(const char *s, int64_t n, const char *r, int64_t m)
{
    int64_t *prev = malloc((size_t)(m + 1) * sizeof(int64_t));
    int64_t *cur = malloc((size_t)(m + 1) * sizeof(int64_t));
    for (int64_t j = 0; j <= m; j++)
        prev[j] = j;
    for (int64_t i = 1; i <= n; i++) {
        cur[0] = i;
        for (int64_t j = 1; j <= m; j++) {
            int64_t d = prev[j - 1] + subst_cost(s[i - 1], r[j - 1]);
            int64_t u = prev[j] + 1, l = cur[j - 1] + 1;
            cur[j] = d < u ? (d < l ? d : l) : (u < l ? u : l);
        }
        int64_t *t = prev;
        prev = cur;
        cur = t;
    }
    int64_t out = prev[m];
    free(prev);
    free(cur);
    return out;
}

/* Alignment of S to R as the state sequence of step 4 (ST_M / ST_I / ST_D per
 * alignment column, in order).  Returns the number of columns. */
static int64_t align_states(const char *s, int64_t n, const char *r, int64_t m, uint8_t *path)
{
    int64_t W = m + 1;
    int64_t *D = malloc((size_t)(n + 1) * (size_t)W * sizeof(int64_t));
    for (int64_t j = 0; j <= m; j++)
        D[j] = j;
    for (int64_t i = 1; i <= n; i++) {
        D[i * W] = i;
        for (int64_t j = 1; j <= m; j++) {
            int64_t d = D[(i - 1) * W + j - 1] + subst_cost(s[i - 1], r[j - 1]);
            int64_t u = D[(i - 1) * W + j] + 1, l = D[i * W + j - 1] + 1;
            int64_t best = d < u ? d : u;
            D[i * W + j] = best < l ? best : l;
        }
    }
    /* traceback, then reverse */
    int64_t i = n, j = m, k = 0;
    while (i > 0 || j > 0) {
        if (i > 0 && j > 0 && D[i * W + j] == D[(i - 1) * W + j - 1] + subst_cost(s[i - 1], r[j - 1])) {
            path[k++] = ST_M;
            i--;
            j--;
        } else if (i > 0 && D[i * W + j] == D[(i - 1) * W + j] + 1) {
            path[k++] = ST_I;
            i--;
        } else {
            path[k++] = ST_D;
            j--;
        }
    }
    for (int64_t a = 0, b = k - 1; a < b; a++, b--) {
        uint8_t t = path[a];
        path[a] = path[b];
        path[b] = t;
    }
    free(D);
    return k;
}

/* Build the profile of step 1-6 from n training sequences (seqs + offsets).
 * Writes m to *m_out; when t and e are not NULL they receive (m + 1) * 9
 * transition scores and (m + 1) * 4 emission scores.  Returns the index of
 * the reference sequence, or -1 when there is no training sequence. */
int64_t or_hmm_build(const char *seqs, const uint64_t *off, int64_t n, int64_t *m_out, double *t, double *e)
{
    if (n <= 0)
        return -1;
    /* step 2: most frequent sequence, first occurrence on ties */
    int64_t best = 0, best_count = 0;
    for (int64_t a = 0; a < n; a++) {
        int64_t la = (int64_t)(off[a + 1] - off[a]), count = 0;
        int seen_before = 0;
        for (int64_t b = 0; b < n; b++) {
            int64_t lb = (int64_t)(off[b + 1] - off[b]);
            if (lb == la && memcmp(seqs + off[a], seqs + off[b], (size_t)la) == 0) {
                if (b < a)
                    seen_before = 1;
                count++;
            }
        }
        if (!seen_before && count > best_count) {
            best = a;
            best_count = count;
        }
    }
    const char *R = seqs + off[best];
    int64_t m = (int64_t)(off[best + 1] - off[best]);
    *m_out = m;
    if (!t || !e)
        return best;
    /* step 4: counts */
    double *ct = calloc((size_t)(m + 1) * 9, sizeof(double));
    double *ce = calloc((size_t)(m + 1) * 4, sizeof(double));
    for (int64_t q = 0; q < n; q++) {
        const char *S = seqs + off[q];
        int64_t ls = (int64_t)(off[q + 1] - off[q]);
        uint8_t *path = malloc((size_t)(ls + m + 1));
        int64_t k = align_states(S, ls, R, m, path);
        int x = ST_M; /* B = M_0 */
        int64_t j = 0, i = 0;
        for (int64_t c = 0; c < k; c++) {
            int y = path[c];
            /* move from X_j: to M_{j+1} (y = M), I_j (y = I), D_{j+1} (y = D) */
            ct[j * 9 + x * 3 + y] += 1.0;
            if (y == ST_M) {
                j++;
                int l = letter(S[i]);
                if (l < 4)
                    ce[j * 4 + l] += 1.0;
                i++;
            } else if (y == ST_I) {
                i++;
            } else {
                j++;
            }
            x = y;
        }
        ct[j * 9 + x * 3 + ST_M] += 1.0; /* to E (j = m) */
        free(path);
    }
    /* steps 5-6 */
    for (int64_t j = 0; j <= m; j++) {
        for (int x = 0; x < 3; x++) {
            double *tt = t + j * 9 + x * 3;
            if (j == 0 && x == ST_D) { /* D_0 does not exist */
                tt[0] = tt[1] = tt[2] = -INFINITY;
                continue;
            }
            int has_d = j < m;
            double tot = 0.0;
            for (int y = 0; y < 3; y++)
                if (y != ST_D || has_d)
                    tot += ct[j * 9 + x * 3 + y] + 1.0;
            for (int y = 0; y < 3; y++)
                tt[y] = (y != ST_D || has_d) ? log2((ct[j * 9 + x * 3 + y] + 1.0) / tot) : -INFINITY;
        }
        for (int l = 0; l < 4; l++) {
            if (j == 0) {
                e[l] = 0.0;
                continue;
            }
            double tot = ce[j * 4 + 0] + ce[j * 4 + 1] + ce[j * 4 + 2] + ce[j * 4 + 3] + 4.0;
            e[j * 4 + l] = log2((ce[j * 4 + l] + 1.0) / tot / 0.25);
        }
    }
    free(ct);
    free(ce);
    return best;
}

static double max3(double a, double b, double c)
{
    double m = a > b ? a : b;
    return m > c ? m : c;
}

/* Glocal Viterbi log-odds score (bits) of x[0..n) against the profile. */
double or_hmm_viterbi(const double *t, const double *e, int64_t m, const char *x, int64_t n)
{
    const double NEG = -INFINITY;
    int64_t W = m + 1;
    double *VM = malloc((size_t)(n + 1) * (size_t)W * sizeof(double));
    double *VI = malloc((size_t)(n + 1) * (size_t)W * sizeof(double));
    double *VD = malloc((size_t)(n + 1) * (size_t)W * sizeof(double));
#define T(j, X, Y) t[(j) * 9 + (X) * 3 + (Y)]
    for (int64_t i = 0; i <= n; i++) {
        for (int64_t j = 0; j <= m; j++) {
            double vm = NEG, vi = NEG, vd = NEG;
            if (i == 0 && j == 0) {
                vm = 0.0;
            } else {
                if (i > 0 && j > 0) {
                    int l = letter(x[i - 1]);
                    double em = l < 4 ? e[j * 4 + l] : 0.0;
                    vm = em + max3(VM[(i - 1) * W + j - 1] + T(j - 1, ST_M, ST_M),
                                   VI[(i - 1) * W + j - 1] + T(j - 1, ST_I, ST_M),
                                   VD[(i - 1) * W + j - 1] + T(j - 1, ST_D, ST_M));
                }
                if (i > 0)
                    vi = max3(VM[(i - 1) * W + j] + T(j, ST_M, ST_I), VI[(i - 1) * W + j] + T(j, ST_I, ST_I),
                              VD[(i - 1) * W + j] + T(j, ST_D, ST_I));
                if (j > 0)
                    vd = max3(VM[i * W + j - 1] + T(j - 1, ST_M, ST_D), VI[i * W + j - 1] + T(j - 1, ST_I, ST_D),
                              VD[i * W + j - 1] + T(j - 1, ST_D, ST_D));
            }
            VM[i * W + j] = vm;
            VI[i * W + j] = vi;
            VD[i * W + j] = vd;
        }
    }
    double s = max3(VM[n * W + m] + T(m, ST_M, ST_M), VI[n * W + m] + T(m, ST_I, ST_M),
                    VD[n * W + m] + T(m, ST_D, ST_M));
#undef T
    free(VM);
    free(VI);
    free(VD);
    return s;
}

/* log2(2^a + 2^b + 2^c), -INFINITY when all three are -INFINITY */
static double lse3(double a, double b, double c)
{
    double m = max3(a, b, c);
    if (m == -INFINITY)
        return -INFINITY;
    return m + log2(exp2(a - m) + exp2(b - m) + exp2(c - m));
}

/* Glocal Forward log-odds score (bits) of x[0..n) against the profile. */
double or_hmm_forward(const double *t, const double *e, int64_t m, const char *x, int64_t n)
{
    const double NEG = -INFINITY;
    int64_t W = m + 1;
    double *FM = malloc((size_t)(n + 1) * (size_t)W * sizeof(double));
    double *FI = malloc((size_t)(n + 1) * (size_t)W * sizeof(double));
    double *FD = malloc((size_t)(n + 1) * (size_t)W * sizeof(double));
#define T(j, X, Y) t[(j) * 9 + (X) * 3 + (Y)]
    for (int64_t i = 0; i <= n; i++) {
        for (int64_t j = 0; j <= m; j++) {
            double fm = NEG, fi = NEG, fd = NEG;
            if (i == 0 && j == 0) {
                fm = 0.0; /* B: the empty path */
            } else {
                if (i > 0 && j > 0) {
                    int l = letter(x[i - 1]);
                    double em = l < 4 ? e[j * 4 + l] : 0.0;
                    fm = em + lse3(FM[(i - 1) * W + j - 1] + T(j - 1, ST_M, ST_M),
                                   FI[(i - 1) * W + j - 1] + T(j - 1, ST_I, ST_M),
                                   FD[(i - 1) * W + j - 1] + T(j - 1, ST_D, ST_M));
                }
                if (i > 0)
                    fi = lse3(FM[(i - 1) * W + j] + T(j, ST_M, ST_I), FI[(i - 1) * W + j] + T(j, ST_I, ST_I),
                              FD[(i - 1) * W + j] + T(j, ST_D, ST_I));
                if (j > 0)
                    fd = lse3(FM[i * W + j - 1] + T(j - 1, ST_M, ST_D), FI[i * W + j - 1] + T(j - 1, ST_I, ST_D),
                              FD[i * W + j - 1] + T(j - 1, ST_D, ST_D));
            }
            FM[i * W + j] = fm;
            FI[i * W + j] = fi;
            FD[i * W + j] = fd;
        }
    }
    double s = lse3(FM[n * W + m] + T(m, ST_M, ST_M), FI[n * W + m] + T(m, ST_I, ST_M),
                    FD[n * W + m] + T(m, ST_D, ST_M));
#undef T
    free(FM);
    free(FI);
    free(FD);
    return s;
}
