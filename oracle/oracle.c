/*
 * oracle.c -- plain, slow, obviously-correct CPU oracle for the in-silico PCR
 * hot path of AmpliconHunter (Howard-Stone & Mandoiu, arXiv 2509.13300).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this file.  It shares no code,
 * header, table or constant with the GPU library: every definition below is
 * written out from the paper (and, where the paper names an external model,
 * from that model's published definition) in the most direct form.
 *
 * What it computes, with the passage each part follows:
 *   or_scan   primer matching with <= k substitutions on both strands, with
 *             the optional 3' clamp (Sec. 2.1 "Primer matching"; degenerate
 *             primers as IUPAC strings, Sec. 1).
 *   or_tm     maximum nearest-neighbour melting temperature over all
 *             oligonucleotides of the degenerate primer, with the salt and
 *             concentration parameters of Sec. 2.1 "Melting temperature
 *             filtering", in fp64.
 *   or_pair   amplicon calling: sites on opposite strands inside the length
 *             window, labelled FR/RF/FF/RR (Sec. 2.1 "Amplicon calling",
 *             "Amplicon analysis" item 1, Appendix A).
 *   or_fetch  amplicon sequences (Sec. 2.1 "Visualization": the main output
 *             is a FASTA of amplicon sequences with coordinates).
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *   - a mismatch is a position whose genome base is not in the primer's IUPAC
 *     set; a genome character other than A/C/G/T (any case) mismatches every
 *     primer position, including N;
 *   - "+" site: the primer X matches the + strand at [pos, pos+L); "-" site:
 *     the reverse complement of X matches the + strand at [pos, pos+L);
 *   - amplicon = left "+" site at s, right "-" site at t >= s in the same
 *     contig, length t + L_right - s inside [min_len, max_len] (inclusive);
 *   - Tm is the max over ALL oligos of the primer; a site whose template
 *     window holds a non-ACGT base has Tm = NaN (never passes a threshold);
 *   - NN model: SantaLucia (1998) unified Watson-Crick stacks and terminal
 *     initiation; a stack containing a mismatch contributes (0, 0) and a
 *     terminal mismatch takes the initiation of the primer base's own class
 *     (the published mismatch tables are not available), unless the caller
 *     passes a full table.
 *
 * Build: gcc -O2 -fopenmp -shared -fPIC oracle.c -lm
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Records (same field order as the library's, declared independently).      */
/* ------------------------------------------------------------------------ */
typedef struct {
    uint32_t genome, contig, pos;
    uint8_t primer; /* 0 = forward, 1 = reverse */
    uint8_t strand; /* 0 = '+', 1 = '-' */
    uint8_t mm;
    uint8_t pair;
} or_site;

typedef struct {
    uint32_t genome, contig, start, end, left, right;
    uint8_t orient; /* 0 FR, 1 RF, 2 FF, 3 RR */
    uint8_t pair;
    uint8_t pad0, pad1;
} or_amplicon;

typedef struct {
    double stack_dH[256]; /* [top5'][top3'][bottom under top5'][bottom under top3'], A=0 C=1 G=2 T=3 */
    double stack_dS[256];
    double term_dH[16]; /* [primer base][template base] at a duplex end */
    double term_dS[16];
} or_nn_table;

typedef struct {
    double dnac1_nM, dnac2_nM, Na_mM, K_mM, Tris_mM, Mg_mM, dNTPs_mM;
    double tm_min;
    int32_t saltcorr;
    int32_t pad;
} or_tm_params;

/* ------------------------------------------------------------------------ */
/* IUPAC nucleotide codes (Sec. 1: each letter stands for a set of bases).   */
/* ------------------------------------------------------------------------ */

/* Does IUPAC letter `code` admit base letter `base` (one of A, C, G, T)? */
static int iupac_admits(char code, char base)
{
    const char *set;
    switch (code) {
    case 'A': set = "A"; break;
    case 'C': set = "C"; break;
    case 'G': set = "G"; break;
    case 'T': set = "T"; break;
    case 'R': set = "AG"; break;
    case 'Y': set = "CT"; break;
    case 'S': set = "CG"; break;
    case 'W': set = "AT"; break;
    case 'K': set = "GT"; break;
    case 'M': set = "AC"; break;
    case 'B': set = "CGT"; break;
    case 'D': set = "AGT"; break;
    case 'H': set = "ACT"; break;
    case 'V': set = "ACG"; break;
    case 'N': set = "ACGT"; break;
    default: return 0;
    }
    return strchr(set, base) != NULL;
}

/* Complement of an IUPAC letter (the set of complements of its bases). */
static char iupac_complement(char code)
{
    switch (code) {
    case 'A': return 'T';
    case 'T': return 'A';
    case 'C': return 'G';
    case 'G': return 'C';
    case 'R': return 'Y';
    case 'Y': return 'R';
    case 'K': return 'M';
    case 'M': return 'K';
    case 'S': return 'S';
    case 'W': return 'W';
    case 'B': return 'V';
    case 'V': return 'B';
    case 'D': return 'H';
    case 'H': return 'D';
    case 'N': return 'N';
    default: return '?';
    }
}

static char upper_char(uint8_t c)
{
    if (c >= 'a' && c <= 'z')
        return (char)(c - 'a' + 'A');
    return (char)c;
}

/* Genome base as one of A/C/G/T, or 0 when it is anything else. */
static char genome_base(uint8_t c)
{
    char u = upper_char(c);
    if (u == 'A' || u == 'C' || u == 'G' || u == 'T')
        return u;
    return 0;
}

static char base_complement(char b)
{
    switch (b) {
    case 'A': return 'T';
    case 'C': return 'G';
    case 'G': return 'C';
    case 'T': return 'A';
    default: return 0;
    }
}

/* Pattern matched on the + strand: the primer itself for strand '+', its
 * reverse complement for strand '-' (Sec. 2.1 Primer matching; Sec. 2.1
 * Amplicon calling pairs sites "found on opposite strands"). */
static void make_pattern(const char *primer, int strand, char *pat)
{
    int L = (int)strlen(primer);
    for (int i = 0; i < L; i++) {
        char c = upper_char((uint8_t)primer[i]);
        if (strand == 0)
            pat[i] = c;
        else
            pat[L - 1 - i] = iupac_complement(c);
    }
    pat[L] = 0;
}

/* Number of mismatches of pattern `pat` against g[0..L). */
static int count_mismatches(const uint8_t *g, const char *pat, int L)
{
    int mm = 0;
    for (int i = 0; i < L; i++) {
        char b = genome_base(g[i]);
        if (b == 0 || !iupac_admits(pat[i], b))
            mm++;
    }
    return mm;
}

/* 3' clamp of length c (Sec. 2.1 Primer matching): no mismatch in the c
 * 3'-most primer bases.  For a '+' site the primer's 3' end is the right end
 * of the window; for a '-' site it is the left end. */
static int clamp_holds(const uint8_t *g, const char *pat, int L, int strand, int c)
{
    for (int j = 0; j < c && j < L; j++) {
        int i = (strand == 0) ? (L - 1 - j) : j;
        char b = genome_base(g[i]);
        if (b == 0 || !iupac_admits(pat[i], b))
            return 0;
    }
    return 1;
}

/* ------------------------------------------------------------------------ */
/* Scan (Sec. 2.1 Primer matching).                                          */
/* ------------------------------------------------------------------------ */

/* Visit every (pair, contig, pos, primer, strand) in canonical order and
 * report each window with <= k mismatches whose clamp holds.  When `out` is
 * NULL only counts.  Returns the number of sites of contig `c` for pair `j`. */
static int64_t scan_contig(const uint8_t *seq, const uint64_t *contig_off, const uint32_t *contig_genome,
                           uint32_t c, int j, const char *pats[2][2], const int Ls[2], int k, int clamp,
                           or_site *out)
{
    uint64_t lo = contig_off[c], hi = contig_off[c + 1];
    uint64_t len = hi - lo;
    int64_t n = 0;
    for (uint64_t p = 0; p < len; p++) {
        for (int primer = 0; primer < 2; primer++) {
            int L = Ls[primer];
            if (p + (uint64_t)L > len)
                continue;
            for (int strand = 0; strand < 2; strand++) {
                const uint8_t *g = seq + lo + p;
                int mm = count_mismatches(g, pats[primer][strand], L);
                if (mm > k)
                    continue;
                if (clamp > 0 && !clamp_holds(g, pats[primer][strand], L, strand, clamp))
                    continue;
                if (out) {
                    or_site *s = &out[n];
                    s->genome = contig_genome[c];
                    s->contig = c;
                    s->pos = (uint32_t)p;
                    s->primer = (uint8_t)primer;
                    s->strand = (uint8_t)strand;
                    s->mm = (uint8_t)mm;
                    s->pair = (uint8_t)j;
                }
                n++;
            }
        }
    }
    return n;
}

int64_t or_scan(const uint8_t *seq, const uint64_t *contig_off, uint32_t n_contigs, const uint32_t *contig_genome,
                const char *const *fwd, const char *const *rev, const int32_t *k, const int32_t *clamp,
                int32_t n_pairs, or_site *out, int64_t cap, int32_t n_threads)
{
#ifdef _OPENMP
    if (n_threads > 0)
        omp_set_num_threads(n_threads);
#else
    (void)n_threads;
#endif
    int64_t ngroups = (int64_t)n_pairs * n_contigs;
    int64_t *cnt = (int64_t *)calloc((size_t)ngroups + 1, sizeof(int64_t));
    char(*pat)[2][2][64] = malloc(sizeof(char[2][2][64]) * (size_t)(n_pairs > 0 ? n_pairs : 1));
    int(*Ls)[2] = malloc(sizeof(int[2]) * (size_t)(n_pairs > 0 ? n_pairs : 1));
    for (int j = 0; j < n_pairs; j++) {
        for (int s = 0; s < 2; s++) {
            make_pattern(fwd[j], s, pat[j][0][s]);
            make_pattern(rev[j], s, pat[j][1][s]);
        }
        Ls[j][0] = (int)strlen(fwd[j]);
        Ls[j][1] = (int)strlen(rev[j]);
    }
    /* pass 1: count per (pair, contig) */
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t gi = 0; gi < ngroups; gi++) {
        int j = (int)(gi / n_contigs);
        uint32_t c = (uint32_t)(gi % n_contigs);
        const char *pp[2][2] = {{pat[j][0][0], pat[j][0][1]}, {pat[j][1][0], pat[j][1][1]}};
        cnt[gi + 1] = scan_contig(seq, contig_off, contig_genome, c, j, pp, Ls[j], k[j], clamp[j], NULL);
    }
    for (int64_t gi = 0; gi < ngroups; gi++)
        cnt[gi + 1] += cnt[gi];
    int64_t total = cnt[ngroups];
    /* pass 2: write (only when everything fits) */
    if (out && total <= cap) {
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t gi = 0; gi < ngroups; gi++) {
            int j = (int)(gi / n_contigs);
            uint32_t c = (uint32_t)(gi % n_contigs);
            const char *pp[2][2] = {{pat[j][0][0], pat[j][0][1]}, {pat[j][1][0], pat[j][1][1]}};
            scan_contig(seq, contig_off, contig_genome, c, j, pp, Ls[j], k[j], clamp[j], out + cnt[gi]);
        }
    }
    free(cnt);
    free(pat);
    free(Ls);
    return total;
}

/* Mismatch count of one window against one primer/strand (for tests). */
int32_t or_window_mismatches(const uint8_t *g, const char *primer, int32_t strand)
{
    char pat[64];
    make_pattern(primer, strand, pat);
    return count_mismatches(g, pat, (int)strlen(primer));
}

/* ------------------------------------------------------------------------ */
/* Nearest-neighbour melting temperature (Sec. 2.1 Melting temperature).     */
/* The paper uses Biopython's NN model; the model it implements is the       */
/* two-state NN model with the SantaLucia (1998) unified parameters:          */
/*   Tm = 1000 dH / (dS + R ln(x)) - 273.15,  x = (dnac1 - dnac2/2) 1e-9,      */
/* dH, dS = sum of NN stack terms + initiation at both duplex ends.           */
/* ------------------------------------------------------------------------ */

/* SantaLucia (1998) PNAS 95:1460, Table 1: unified Watson-Crick NN
 * parameters, written "top 5'->3' / bottom 3'->5'": dH kcal/mol, dS e.u. */
static const struct {
    const char *key;
    double dH, dS;
} WC_STACKS[] = {
    {"AA/TT", -7.9, -22.2}, {"AT/TA", -7.2, -20.4}, {"TA/AT", -7.2, -21.3}, {"CA/GT", -8.5, -22.7},
    {"GT/CA", -8.4, -22.4}, {"CT/GA", -7.8, -21.0}, {"GA/CT", -8.2, -22.2}, {"CG/GC", -10.6, -27.2},
    {"GC/CG", -9.8, -24.4}, {"GG/CC", -8.0, -19.9},
};
/* Initiation with a terminal G.C pair and with a terminal A.T pair. */
static const double INIT_GC_dH = 0.1, INIT_GC_dS = -2.8;
static const double INIT_AT_dH = 2.3, INIT_AT_dS = 4.1;
static const double GAS_R = 1.987; /* cal / (K mol) */

static int is_wc(char a, char b) { return base_complement(a) == b; }

/* Stack (top t0 t1 / bottom b0 b1): the table entry, looked up directly or
 * after reading the duplex from the other end (5'-b1 b0-3' / 3'-t1 t0-5').
 * A stack containing a mismatch contributes nothing (see header). */
static void default_stack(char t0, char t1, char b0, char b1, double *dH, double *dS)
{
    *dH = 0.0;
    *dS = 0.0;
    if (!is_wc(t0, b0) || !is_wc(t1, b1))
        return;
    char key[6] = {t0, t1, '/', b0, b1, 0};
    char rot[6] = {b1, b0, '/', t1, t0, 0};
    for (size_t i = 0; i < sizeof(WC_STACKS) / sizeof(WC_STACKS[0]); i++) {
        if (strcmp(WC_STACKS[i].key, key) == 0 || strcmp(WC_STACKS[i].key, rot) == 0) {
            *dH = WC_STACKS[i].dH;
            *dS = WC_STACKS[i].dS;
            return;
        }
    }
}

/* Initiation term of a duplex end whose primer base is p and template base
 * is t.  A Watson-Crick end takes its pair class; a mismatched end takes the
 * class of the primer base (see header). */
static void default_terminal(char p, char t, double *dH, double *dS)
{
    (void)t;
    if (p == 'G' || p == 'C') {
        *dH = INIT_GC_dH;
        *dS = INIT_GC_dS;
    } else {
        *dH = INIT_AT_dH;
        *dS = INIT_AT_dS;
    }
}

static int base_index(char b)
{
    switch (b) {
    case 'A': return 0;
    case 'C': return 1;
    case 'G': return 2;
    case 'T': return 3;
    default: return -1;
    }
}

/* The default table as a full 4x4x4x4 array (for callers that want to pass
 * one explicitly, and for the test that both lookups agree). */
void or_default_table(or_nn_table *tab)
{
    const char B[4] = {'A', 'C', 'G', 'T'};
    for (int a = 0; a < 4; a++)
        for (int b = 0; b < 4; b++)
            for (int c = 0; c < 4; c++)
                for (int d = 0; d < 4; d++) {
                    double h, s;
                    default_stack(B[a], B[b], B[c], B[d], &h, &s);
                    tab->stack_dH[((a * 4 + b) * 4 + c) * 4 + d] = h;
                    tab->stack_dS[((a * 4 + b) * 4 + c) * 4 + d] = s;
                }
    for (int p = 0; p < 4; p++)
        for (int t = 0; t < 4; t++) {
            double h, s;
            default_terminal(B[p], B[t], &h, &s);
            tab->term_dH[p * 4 + t] = h;
            tab->term_dS[p * 4 + t] = s;
        }
}

/* Sum of NN terms of duplex top o[0..L) (5'->3') over bottom b[0..L), where
 * b[i] is the template base opposite o[i].  `tab` NULL = default model. */
static void duplex_terms(const char *o, const char *b, int L, const or_nn_table *tab, double *dH, double *dS)
{
    double H = 0.0, S = 0.0, h, s;
    for (int i = 0; i + 1 < L; i++) {
        if (tab) {
            int idx = ((base_index(o[i]) * 4 + base_index(o[i + 1])) * 4 + base_index(b[i])) * 4 + base_index(b[i + 1]);
            h = tab->stack_dH[idx];
            s = tab->stack_dS[idx];
        } else {
            default_stack(o[i], o[i + 1], b[i], b[i + 1], &h, &s);
        }
        H += h;
        S += s;
    }
    /* initiation at the two ends */
    if (tab) {
        int e0 = base_index(o[0]) * 4 + base_index(b[0]);
        int e1 = base_index(o[L - 1]) * 4 + base_index(b[L - 1]);
        H += tab->term_dH[e0];
        S += tab->term_dS[e0];
        H += tab->term_dH[e1];
        S += tab->term_dS[e1];
    } else {
        default_terminal(o[0], b[0], &h, &s);
        H += h;
        S += s;
        default_terminal(o[L - 1], b[L - 1], &h, &s);
        H += h;
        S += s;
    }
    *dH = H;
    *dS = S;
}

/* Monovalent-equivalent cation concentration in mM (von Ahsen et al. 2001):
 * Na + K + Tris/2 + 120 sqrt(Mg - dNTPs) when Mg > dNTPs. */
static double na_equivalent_mM(const or_tm_params *p)
{
    double mon = p->Na_mM + p->K_mM + p->Tris_mM / 2.0;
    if (p->Mg_mM > p->dNTPs_mM)
        mon += 120.0 * sqrt(p->Mg_mM - p->dNTPs_mM);
    return mon;
}

/* Tm in deg C of one duplex of length L (Sec. 2.1: dnac1, dnac2, Na, K, Tris,
 * Mg, dNTPs and the salt correction method are parameters).  Salt methods:
 * 0 none; 1 Tm shift 16.6 log10[Na] (Schildkraut-Lifson 1965); 5 entropy
 * term 0.368 (L-1) ln[Na] (SantaLucia 1998).  [Na] in mol/L.  Other method
 * numbers give NaN (the library rejects them). */
static double duplex_tm(const char *o, const char *b, int L, const or_nn_table *tab, const or_tm_params *p)
{
    double H, S;
    duplex_terms(o, b, L, tab, &H, &S);
    double na = na_equivalent_mM(p) / 1000.0;
    if (p->saltcorr == 5)
        S += 0.368 * (double)(L - 1) * log(na);
    double x = (p->dnac1_nM - p->dnac2_nM / 2.0) * 1e-9;
    double tm = 1000.0 * H / (S + GAS_R * log(x)) - 273.15;
    if (p->saltcorr == 1)
        tm += 16.6 * log10(na);
    else if (p->saltcorr != 0 && p->saltcorr != 5)
        tm = NAN;
    return tm;
}

/* Tm of one explicit oligo against an explicit template window (tests). */
double or_duplex_tm(const char *oligo, const char *bottom, const or_nn_table *tab, const or_tm_params *p)
{
    return duplex_tm(oligo, bottom, (int)strlen(oligo), tab, p);
}

/* Max Tm over every oligo of degenerate primer X at one site (Sec. 2.1: a
 * site passes when its best oligo reaches the threshold; every oligo of the
 * primer is evaluated on its own). */
static double site_max_tm(const uint8_t *window, int strand, const char *primer, const or_nn_table *tab,
                          const or_tm_params *p)
{
    int L = (int)strlen(primer);
    char bottom[64], oligo[64];
    /* bottom[i] = template base opposite primer position i */
    for (int i = 0; i < L; i++) {
        char g = (strand == 0) ? genome_base(window[i]) : genome_base(window[L - 1 - i]);
        if (g == 0)
            return NAN;
        bottom[i] = (strand == 0) ? base_complement(g) : g;
    }
    bottom[L] = 0;
    /* enumerate the oligos with a mixed-radix counter over the IUPAC sets */
    char sets[64][5];
    int nset[64], digit[64];
    for (int i = 0; i < L; i++) {
        char code = upper_char((uint8_t)primer[i]);
        nset[i] = 0;
        const char *all = "ACGT";
        for (int q = 0; q < 4; q++)
            if (iupac_admits(code, all[q]))
                sets[i][nset[i]++] = all[q];
        digit[i] = 0;
    }
    double best = -INFINITY;
    for (;;) {
        for (int i = 0; i < L; i++)
            oligo[i] = sets[i][digit[i]];
        oligo[L] = 0;
        double tm = duplex_tm(oligo, bottom, L, tab, p);
        if (tm > best)
            best = tm;
        int i = L - 1;
        while (i >= 0 && ++digit[i] == nset[i]) {
            digit[i] = 0;
            i--;
        }
        if (i < 0)
            break;
    }
    return best;
}

void or_tm(const uint8_t *seq, const uint64_t *contig_off, const or_site *sites, int64_t n, const char *const *fwd,
           const char *const *rev, const or_tm_params *params, const or_nn_table *tab, double *tm_out,
           uint8_t *pass_out, int32_t n_threads)
{
#ifdef _OPENMP
    if (n_threads > 0)
        omp_set_num_threads(n_threads);
#else
    (void)n_threads;
#endif
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; i++) {
        const or_site *s = &sites[i];
        const char *X = s->primer ? rev[s->pair] : fwd[s->pair];
        const uint8_t *w = seq + contig_off[s->contig] + s->pos;
        double tm = site_max_tm(w, s->strand, X, tab, &params[s->pair]);
        tm_out[i] = tm;
        if (pass_out)
            pass_out[i] = (tm >= params[s->pair].tm_min) ? 1 : 0; /* NaN fails */
    }
}

/* ------------------------------------------------------------------------ */
/* Amplicon calling (Sec. 2.1 Amplicon calling; orientation labels from       */
/* Sec. 2.1 Amplicon analysis item 1).                                        */
/* ------------------------------------------------------------------------ */

static int amp_cmp(const void *pa, const void *pb)
{
    const or_amplicon *a = pa, *b = pb;
#define CMPF(f)          \
    if (a->f != b->f)    \
        return a->f < b->f ? -1 : 1;
    CMPF(pair)
    CMPF(contig)
    CMPF(start)
    CMPF(end)
    CMPF(orient)
#undef CMPF
    return 0;
}

/* Sites must be in canonical order (pair, contig, pos, primer, strand), as
 * or_scan returns them.  Every '+' site pairs with every '-' site of the same
 * pair and contig at t >= s whose amplicon length lies in the window; when
 * `pass` is given both ends must pass the Tm threshold. */
int64_t or_pair(const or_site *sites, int64_t n, const uint8_t *pass, const int32_t *Lf, const int32_t *Lr,
                const int32_t *min_len, const int32_t *max_len, or_amplicon *out, int64_t cap)
{
    int64_t cnt = 0;
    int64_t g0 = 0;
    while (g0 < n) {
        int64_t g1 = g0;
        while (g1 < n && sites[g1].pair == sites[g0].pair && sites[g1].contig == sites[g0].contig)
            g1++;
        for (int64_t a = g0; a < g1; a++) {
            if (sites[a].strand != 0)
                continue;
            for (int64_t b = g0; b < g1; b++) {
                if (sites[b].strand != 1 || sites[b].pos < sites[a].pos)
                    continue;
                int j = sites[a].pair;
                int64_t Lright = sites[b].primer ? Lr[j] : Lf[j];
                int64_t end = (int64_t)sites[b].pos + Lright;
                int64_t len = end - (int64_t)sites[a].pos;
                if (len < min_len[j] || len > max_len[j])
                    continue;
                if (pass && !(pass[a] && pass[b]))
                    continue;
                if (out && cnt < cap) {
                    or_amplicon *o = &out[cnt];
                    memset(o, 0, sizeof(*o));
                    o->genome = sites[a].genome;
                    o->contig = sites[a].contig;
                    o->start = sites[a].pos;
                    o->end = (uint32_t)end;
                    o->left = (uint32_t)a;
                    o->right = (uint32_t)b;
                    /* left primer X, right primer Y: FR, RF, FF, RR */
                    int X = sites[a].primer, Y = sites[b].primer;
                    o->orient = (uint8_t)((X == 0 && Y == 1) ? 0 : (X == 1 && Y == 0) ? 1 : (X == 0) ? 2 : 3);
                    o->pair = (uint8_t)j;
                }
                cnt++;
            }
        }
        g0 = g1;
    }
    if (out && cnt <= cap)
        qsort(out, (size_t)cnt, sizeof(or_amplicon), amp_cmp);
    return cnt;
}

/* ------------------------------------------------------------------------ */
/* Amplicon sequences (Sec. 2.1 Visualization: FASTA of amplicon sequences). */
/* Upper-case; every non-ACGT character becomes N; an RF amplicon is reverse- */
/* complemented so that it reads from the forward primer.                     */
/* ------------------------------------------------------------------------ */
int64_t or_fetch(const uint8_t *seq, const uint64_t *contig_off, const or_amplicon *a, int64_t n, char *out,
                 int64_t cap, uint64_t *offsets)
{
    int64_t total = 0;
    for (int64_t i = 0; i < n; i++) {
        offsets[i] = (uint64_t)total;
        total += (int64_t)a[i].end - (int64_t)a[i].start;
    }
    offsets[n] = (uint64_t)total;
    if (!out || total > cap)
        return total;
    for (int64_t i = 0; i < n; i++) {
        const uint8_t *g = seq + contig_off[a[i].contig];
        int64_t len = (int64_t)a[i].end - (int64_t)a[i].start;
        char *o = out + offsets[i];
        for (int64_t q = 0; q < len; q++) {
            char b = genome_base(g[a[i].start + q]);
            o[q] = b ? b : 'N';
        }
        if (a[i].orient == 1) {
            for (int64_t q = 0; q < len / 2; q++) {
                char t = o[q];
                o[q] = o[len - 1 - q];
                o[len - 1 - q] = t;
            }
            for (int64_t q = 0; q < len; q++)
                o[q] = (o[q] == 'N') ? 'N' : base_complement(o[q]);
        }
    }
    return total;
}

/* Degeneracy (number of oligos) of a primer; 0 if it holds a non-IUPAC
 * letter.  Saturates at 2^62. */
int64_t or_degeneracy(const char *primer)
{
    int64_t d = 1;
    for (const char *c = primer; *c; c++) {
        char u = upper_char((uint8_t)*c);
        int n = iupac_admits(u, 'A') + iupac_admits(u, 'C') + iupac_admits(u, 'G') + iupac_admits(u, 'T');
        if (n == 0)
            return 0;
        if (d > ((int64_t)1 << 62) / 4)
            return (int64_t)1 << 62;
        d *= n;
    }
    return d;
}
