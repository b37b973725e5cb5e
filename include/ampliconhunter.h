/*
 * ampliconhunter.h -- C ABI of the GB300 (sm_103a) in-silico PCR hot path.
 *
 * The operations are those of AmpliconHunter (Howard-Stone & Mandoiu,
 * arXiv 2509.13300): find the binding sites of a degenerate primer pair on
 * both strands of every genome with at most k mismatches (Sec. 2.1, Primer
 * matching), score each site's nearest-neighbour melting temperature as the
 * maximum over the primer's oligonucleotides (Sec. 2.1, Melting temperature
 * filtering), pair sites on opposite strands into amplicons inside the
 * length window (Sec. 2.1, Amplicon calling) with FR/RF/FF/RR labels (Sec.
 * 2.1, Amplicon analysis, item 1) and return the amplicon sequences (Sec.
 * 2.1, Visualization).  The inputs follow the paper's (Sec. 1): genome
 * sequences with contigs, degenerate primers, annealing temperature,
 * mismatch limit, amplicon length bounds, and the concentration and salt
 * parameters of the NN model.
 *
 * Conventions for every call:
 *  - Coordinates are 0-based, half-open and relative to the contig.
 *  - Bulk arrays marked "host or device" may be host memory (pageable or
 *    pinned) or device memory of the context's GPU; the library detects which.
 *    Arrays marked "host" must be host memory.  The caller owns every array
 *    it passes; the library owns the packed genome sets (until
 *    ah_unload_genomes or ah_destroy) and its own scratch memory.
 *  - `stream` is a cudaStream_t (NULL: the context's own stream).  Work is
 *    ordered after earlier work on that stream.  Every call returns only
 *    when its outputs are written (host outputs included).
 *  - Outputs with a capacity: if `cap` is smaller than the number of records
 *    needed, nothing is written, `*n_out` receives the needed count and the
 *    call returns AH_ERR_OVERFLOW.  cap = 0 is therefore a size query.
 *  - Canonical order (results are deterministic and bit-exact across runs):
 *    sites by (pair, contig, pos, primer, strand); amplicons by
 *    (pair, contig, start, end, orient).  "contig" is the index of the contig
 *    in the order the genome set was loaded.
 *  - A context is thread-compatible, not thread-safe: calls on one context
 *    must not overlap.  Different contexts are independent.
 *  - On any error the call returns a non-zero status; ah_last_error() gives a
 *    one-line message.  No call aborts the process.
 */
#ifndef AMPLICONHUNTER_H
#define AMPLICONHUNTER_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t ah_status;
#define AH_OK 0
#define AH_ERR_ARG 1          /* invalid argument: null pointer, bad size, unknown id, bad parameter */
#define AH_ERR_PRIMER 2       /* primer rejected: non-IUPAC letter, length < 5 or > 32, degeneracy > 10000, k > 10 */
#define AH_ERR_OOM 3          /* device memory allocation failed */
#define AH_ERR_BUDGET 4       /* the request would exceed the context's device-memory budget */
#define AH_ERR_OVERFLOW 5     /* output capacity too small; *n_out holds the needed count */
#define AH_ERR_CUDA 6         /* CUDA runtime error (message in ah_last_error) */
#define AH_ERR_TIMEOUT 7      /* a bounded device-side wait ran out; the context stays usable */
#define AH_ERR_JIT 8          /* run-time compilation of a specialised kernel failed */
#define AH_ERR_DEVICE_CHECK 9 /* a device-side consistency check failed */

/* Server limits of Sec. 2.2 (the paper's web server), enforced by ah_set_primers. */
#define AH_MAX_DEGENERACY 10000
#define AH_MAX_MISMATCHES 10
#define AH_MIN_PRIMER_LEN 5
/* Kernel limit of this library: a primer holds at most 32 positions. */
#define AH_MAX_PRIMER_LEN 32
/* Most primer pairs one ah_scan call fuses into one pass over the genomes. */
#define AH_MAX_PAIRS_PER_SCAN 16

typedef struct ah_ctx ah_ctx;

/* PCR parameters of one primer pair (Sec. 1 and Sec. 2.1).
 * k         mismatches allowed per primer site, 0..10 (Sec. 2.2 limit)
 * clamp     3' clamp length: no mismatch in the clamp 3'-most primer bases (0 = off)
 * min_len, max_len
 *           amplicon length window, inclusive; the length is the outer length
 *           end - start, both primer sites included
 * tm_min    minimum melting temperature in deg C; a site passes when the max
 *           Tm over its primer's oligos is >= tm_min (ah_tm pass flags)
 * dnac1_nM  primer concentration; dnac2_nM template concentration (nM);
 *           the NN model uses x = (dnac1 - dnac2/2) * 1e-9, which must be > 0
 * Na_mM, K_mM, Tris_mM, Mg_mM, dNTPs_mM
 *           ion concentrations (mM); [Na_eq] = Na + K + Tris/2
 *           + 120 sqrt(Mg - dNTPs) when Mg > dNTPs (von Ahsen 2001)
 * saltcorr  0 none; 1 Tm += 16.6 log10[Na_eq] (Schildkraut-Lifson 1965);
 *           5 dS += 0.368 (L - 1) ln[Na_eq] (SantaLucia 1998); [Na_eq] in
 *           mol/L.  Other methods are rejected (AH_ERR_ARG). */
typedef struct ah_pcr_params {
    int32_t k;
    int32_t clamp;
    int32_t min_len;
    int32_t max_len;
    double tm_min;
    double dnac1_nM;
    double dnac2_nM;
    double Na_mM;
    double K_mM;
    double Tris_mM;
    double Mg_mM;
    double dNTPs_mM;
    int32_t saltcorr;
    int32_t reserved;
} ah_pcr_params;

/* One primer binding site (Sec. 2.1 Primer matching).
 * strand 0 ('+'): the primer matches the + strand at [pos, pos + L);
 * strand 1 ('-'): the primer's reverse complement matches the + strand at
 * [pos, pos + L).  mm = mismatches (<= k).  pair = index into the pair_ids
 * array of the ah_scan call that produced it. */
typedef struct ah_site {
    uint32_t genome;
    uint32_t contig;
    uint32_t pos;
    uint8_t primer; /* 0 forward, 1 reverse */
    uint8_t strand; /* 0 '+', 1 '-' */
    uint8_t mm;
    uint8_t pair;
} ah_site;

/* One amplicon (Sec. 2.1 Amplicon calling): a '+' site at `start` (index
 * `left` in the site array) and a '-' site ending at `end` (index `right`) in
 * the same contig.  orient: 0 FR, 1 RF, 2 FF, 3 RR = (primer of the left
 * site, primer of the right site) (Sec. 2.1 Amplicon analysis, item 1). */
typedef struct ah_amplicon {
    uint32_t genome;
    uint32_t contig;
    uint32_t start;
    uint32_t end;
    uint32_t left;
    uint32_t right;
    uint8_t orient;
    uint8_t pair;
    uint8_t pad0;
    uint8_t pad1;
} ah_amplicon;

/* Nearest-neighbour parameter table (Sec. 2.1: the NN model of DNA duplex
 * stability).  Base index A=0 C=1 G=2 T=3.
 * stack_dH/dS[((t0*4 + t1)*4 + b0)*4 + b1]: stack of top 5'-t0 t1-3' over the
 *   template bases b0 (opposite t0) and b1 (opposite t1); kcal/mol, cal/(K mol).
 * term_dH/dS[p*4 + t]: initiation term of a duplex end whose primer base is p
 *   and template base is t.
 * The default table (used when none is set) holds the SantaLucia (1998)
 * unified Watson-Crick stacks and terminal initiation terms; a stack holding
 * a mismatched pair contributes (0, 0) and a mismatched end takes the
 * initiation term of the primer base's class (A/T or G/C). */
typedef struct ah_nn_table {
    double stack_dH[256];
    double stack_dS[256];
    double term_dH[16];
    double term_dS[16];
} ah_nn_table;

/* Create a context on CUDA device `device`.  mem_budget_bytes caps the device
 * memory the context may hold (packed genomes + scratch); 0 = no cap.
 * Returns AH_ERR_ARG for a bad device or null out, AH_ERR_CUDA on a CUDA
 * failure. */
ah_status ah_create(int device, size_t mem_budget_bytes, ah_ctx **out);

/* Destroy a context and free everything it owns.  Null is a no-op. */
void ah_destroy(ah_ctx *ctx);

/* Message of the last error on this context (library-owned, valid until the
 * next call on the context).  Null ctx: the last ah_create error. */
const char *ah_last_error(const ah_ctx *ctx);

/* Device bytes the context holds now (pool + scratch). */
size_t ah_device_bytes(const ah_ctx *ctx);

/* Load a genome collection (Sec. 1: genome sequences in FASTA form, here
 * already parsed).  seq (host or device): n_bases ASCII letters, all contigs
 * concatenated; any case; letters other than A/C/G/T (N, IUPAC codes, gaps)
 * are kept as "no base", which mismatches every primer position.
 * contig_off (host): n_contigs + 1 non-decreasing offsets into seq, first 0,
 * last n_bases.  contig_genome (host): genome id of each contig.
 * The library packs the sequence on the device into its own layout (4 one-hot
 * bitplanes A/C/G/T) and returns an id in *set_id_out.  Host arrays are not
 * referenced after the call: a host seq is copied through a staging buffer
 * on the device (the whole sequence when it fits in 4 GiB, else chunks of that
 * size through two buffers, the copies overlapping the packing; at most 1/16
 * of a memory budget; the context keeps the buffers for later loads) and the
 * call waits for the copies, not for the packing.  A device seq is read by work queued
 * on `stream` (stream-ordered, like any CUDA call): it must stay valid until
 * that work has run; the call returns without waiting for it.  A device seq
 * at a 16-byte aligned address is staged by bulk copies; at any other address
 * the packing reads it byte by byte, several times slower.  Every later
 * call that reads the set orders itself after the packing, whatever stream
 * it is given.  A device-side failure of the packing is reported by the next
 * call on the context that synchronises (ah_unload_genomes at the latest).
 * Errors: AH_ERR_ARG (null pointers, non-monotone offsets, n_contigs = 0),
 * AH_ERR_BUDGET, AH_ERR_OOM, AH_ERR_TIMEOUT, AH_ERR_CUDA. */
ah_status ah_load_genomes(ah_ctx *ctx, const uint8_t *seq, uint64_t n_bases, const uint64_t *contig_off,
                          uint32_t n_contigs, const uint32_t *contig_genome, uint32_t *set_id_out, void *stream);

/* ah_load_genomes with options.  flags: AH_LOAD_REVERSED packs every contig
 * reversed, not complemented (position p of contig c holds the base at
 * len_c - 1 - p of the input contig): the decoy collection of Sec. 2.1
 * (Amplicon analysis: decoy genomes estimate the off-target rate as decoy
 * amplicons / real amplicons).  Every later call on the set works on the
 * reversed contigs, in their own coordinates.  A reversed load always waits
 * for its packing before it returns.  Unknown flag bits: AH_ERR_ARG.
 * Other arguments, ownership and errors as ah_load_genomes. */
#define AH_LOAD_REVERSED 1u
/* flags: AH_LOAD_HOST_ASYNC (ah_load_genomes_ex, ah_load_genomes_2bit_ex): a
 * host seq (or host codes and gaps) is read by copies the call queues and does
 * not wait for, so a host load can overlap the caller's next calls (a run in
 * flight).  The caller keeps those host arrays valid and unchanged until the
 * set is ready: until a call that reads the set and synchronises (ah_scan,
 * ah_run, ah_run_end, ...) or ah_unload_genomes of the set has returned.
 * Ignored for device input and for reversed loads (which always wait). */
#define AH_LOAD_HOST_ASYNC 2u
ah_status ah_load_genomes_ex(ah_ctx *ctx, const uint8_t *seq, uint64_t n_bases, const uint64_t *contig_off,
                             uint32_t n_contigs, const uint32_t *contig_genome, uint32_t flags, uint32_t *set_id_out,
                             void *stream);

/* ah_load_genomes from 2-bit base codes (the loaded set is the same as from
 * the ASCII letters they encode): a quarter of the bytes over the host link.
 * The idea is that of 2-bit genome files: two bits per base and a list of the
 * runs that are no base (N, IUPAC codes, gaps).
 * codes (host or device): ceil(n_bases / 4) bytes; base p is bits
 * 2 (p % 4) .. 2 (p % 4) + 1 of byte p / 4, A 0, C 1, G 2, T 3.  Device
 * codes must be 16-byte aligned (else AH_ERR_ARG).
 * gaps (host): n_gaps (start, length) pairs of uint64, sorted by start,
 * disjoint, length >= 1, inside [0, n_bases), at most 2^32 - 1 of them: the
 * positions that are no base, whatever their codes hold.
 * contig_off, contig_genome, set_id_out, stream, ownership, the waiting
 * rules and errors: as ah_load_genomes (the call also returns AH_ERR_ARG for
 * gaps that are unsorted, overlapping, empty or outside the set). */
ah_status ah_load_genomes_2bit(ah_ctx *ctx, const uint8_t *codes, uint64_t n_bases, const uint64_t *gaps,
                               uint64_t n_gaps, const uint64_t *contig_off, uint32_t n_contigs,
                               const uint32_t *contig_genome, uint32_t *set_id_out, void *stream);
/* ah_load_genomes_2bit with flags (AH_LOAD_HOST_ASYNC; other bits: AH_ERR_ARG). */
ah_status ah_load_genomes_2bit_ex(ah_ctx *ctx, const uint8_t *codes, uint64_t n_bases, const uint64_t *gaps,
                                  uint64_t n_gaps, const uint64_t *contig_off, uint32_t n_contigs,
                                  const uint32_t *contig_genome, uint32_t flags, uint32_t *set_id_out,
                                  void *stream);

/* Free a loaded genome set (after its packing has run).  AH_ERR_ARG for an
 * unknown id; AH_ERR_TIMEOUT for a packing that failed on the device and was
 * not reported before (the set is freed either way). */
ah_status ah_unload_genomes(ah_ctx *ctx, uint32_t set_id);

/* Register a degenerate primer pair with its PCR parameters (Sec. 1, Sec.
 * 2.1).  fwd, rev: NUL-terminated IUPAC strings (A C G T R Y S W K M B D H V N,
 * any case), 5'->3'.  Validation follows the limits of Sec. 2.2: each primer
 * at least 5 letters and degeneracy at most 10000, k at most 10; this library
 * also requires at most 32 letters.  Errors: AH_ERR_PRIMER for a primer or k
 * outside the limits, AH_ERR_ARG for other bad parameters (clamp < 0,
 * min_len > max_len, x <= 0, salt method other than 0, 1 or 5, [Na_eq] <= 0
 * with a salt method). */
ah_status ah_set_primers(ah_ctx *ctx, const char *fwd, const char *rev, const ah_pcr_params *params,
                         uint32_t *pair_id_out);

/* Replace the NN parameter table of a registered pair (host struct, copied).
 * Null restores the default table.  AH_ERR_ARG for an unknown pair or a
 * non-finite entry. */
ah_status ah_set_nn_table(ah_ctx *ctx, uint32_t pair_id, const ah_nn_table *table);

/* Primer matching (Sec. 2.1): every site of every listed pair on both strands
 * of every contig of the set with <= k mismatches (and the 3' clamp when
 * set), in canonical order.  A mismatch is a genome position whose base is not
 * in the primer position's IUPAC set; a non-ACGT genome letter mismatches
 * every position.  Windows never cross a contig end.  All listed pairs share
 * one pass over the packed genomes.  pair_ids (host): n_pairs ids, 1..16.
 * out (host or device): cap records.  *n_out (host): number of sites.
 * Errors: AH_ERR_ARG, AH_ERR_OVERFLOW, AH_ERR_JIT, AH_ERR_TIMEOUT, AH_ERR_CUDA. */
ah_status ah_scan(ah_ctx *ctx, uint32_t set_id, const uint32_t *pair_ids, uint32_t n_pairs, ah_site *out,
                  uint64_t cap, uint64_t *n_out, void *stream);

/* Variant of the generated scan kernel picked by ah_tune_scan. */
typedef struct ah_tune_result {
    int32_t R;             /* 32-start words per thread */
    int32_t arith_pct;     /* share of full adders whose sum uses integer adds instead of a LOP3 */
    int32_t min_blocks;    /* occupancy hint given to the compiler */
    int32_t order;         /* 0 word-major, 1 pattern-major code order */
    int32_t stages;        /* bulk-copy stages per warp */
    int32_t warps_per_cta; /* warps per thread block */
    int32_t regs;          /* registers per thread of the chosen variant */
    int32_t reserved;
    double us_per_tile;    /* measured time per 32768-base tile (all launches of the scan) */
    uint64_t tiles;        /* tiles in the timed sample */
} ah_tune_result;

/* Autotuner of the scan (a performance aid; it does not change results):
 * compiles the candidate variants of the scan kernel specialised to these
 * pairs, times each on the first sample_tiles tiles of the set (0 = 4096),
 * and keeps the fastest for every later ah_scan of the same pattern set on
 * this context.  A scan of several pairs whose networks are large runs as
 * one launch per group of pairs; each group is tuned on its own, and
 * best_out (host, may be null) receives the slowest group's variant with
 * the groups' summed time.
 * Errors: AH_ERR_ARG, AH_ERR_JIT, AH_ERR_CUDA. */
ah_status ah_tune_scan(ah_ctx *ctx, uint32_t set_id, const uint32_t *pair_ids, uint32_t n_pairs,
                       uint64_t sample_tiles, ah_tune_result *best_out, void *stream);

/* Melting temperature (Sec. 2.1): for each site, the maximum over every
 * oligonucleotide of its primer of the NN Tm (deg C) of that oligo against the
 * template at the site, computed in fp32 (NaN when the template window holds a
 * non-ACGT letter).  sites (host or device) as returned by ah_scan with the
 * same pair_ids.  tm_out (host or device, n floats).  pass_out (host or
 * device, n bytes, may be null): 1 when the site's max Tm >= its pair's
 * tm_min; the decision is taken in fp64 whenever the fp32 value lies within
 * 0.05 deg C of tm_min, so it equals the fp64 decision.
 * Errors: AH_ERR_ARG, AH_ERR_CUDA. */
ah_status ah_tm(ah_ctx *ctx, uint32_t set_id, const uint32_t *pair_ids, uint32_t n_pairs, const ah_site *sites,
                uint64_t n, float *tm_out, uint8_t *pass_out, void *stream);

/* Amplicon calling (Sec. 2.1): every '+' site at s paired with every '-' site
 * at t >= s of the same pair and contig whose amplicon [s, t + L_right) has
 * length in [min_len, max_len]; when `pass` (host or device, n bytes) is
 * given, both sites must have pass = 1 (the Tm filter).  sites (host or
 * device) must be in canonical order (as ah_scan returns them).  out (host or
 * device, cap records) in canonical order; *n_out (host).
 * Errors: AH_ERR_ARG, AH_ERR_OVERFLOW, AH_ERR_CUDA. */
ah_status ah_pair(ah_ctx *ctx, uint32_t set_id, const uint32_t *pair_ids, uint32_t n_pairs, const ah_site *sites,
                  const uint8_t *pass, uint64_t n, ah_amplicon *out, uint64_t cap, uint64_t *n_out, void *stream);

/* Amplicon sequences (Sec. 2.1: the main output is a FASTA of amplicon
 * sequences with coordinates and orientations).  For each amplicon the bases
 * [start, end) of its contig, upper case, every non-ACGT letter as 'N'; an RF
 * amplicon is reverse-complemented so it reads from the forward primer.
 * seq_out (host or device, cap bytes, no separators); offsets_out (host or
 * device, n + 1 entries): amplicon i is seq_out[offsets[i], offsets[i+1]).
 * On AH_ERR_OVERFLOW offsets_out is written and offsets_out[n] is the size
 * needed.  Errors: AH_ERR_ARG, AH_ERR_OVERFLOW, AH_ERR_CUDA. */
ah_status ah_fetch(ah_ctx *ctx, uint32_t set_id, const ah_amplicon *amplicons, uint64_t n, char *seq_out,
                   uint64_t cap, uint64_t *offsets_out, void *stream);

/* Outputs of ah_run.  The caller sets the buffers and capacities (host or
 * device memory, any may be null with capacity 0); ah_run fills the counts.
 * tm and pass hold n_sites entries (capacity sites_cap); seq_offsets holds
 * n_amplicons + 1 entries (capacity amplicons_cap + 1). */
typedef struct ah_run_out {
    ah_site *sites;
    uint64_t sites_cap;
    uint64_t n_sites;
    float *tm;
    uint8_t *pass;
    ah_amplicon *amplicons;
    uint64_t amplicons_cap;
    uint64_t n_amplicons;
    char *seq;
    uint64_t seq_cap;
    uint64_t n_seq;
    uint64_t *seq_offsets;
    int32_t tm_filter; /* 1: amplicons only from sites whose Tm passes (Sec. 2.1: filter, then pair) */
    int32_t reserved;
} ah_run_out;

/* The whole hot path of Sec. 2.1 in one call: primer matching (as ah_scan),
 * the Tm of every site with pass flags (as ah_tm), amplicon calling on the
 * sites (as ah_pair; with tm_filter only sites that pass) and the amplicon
 * sequences (as ah_fetch), for the listed pairs on one loaded set.  The
 * results are identical to that sequence of calls; only the number of host
 * synchronisations differs: one when every count fits the sizes the call's
 * launches are sized for (at most 16384 sites and the sites capacity when the
 * site outputs are device memory; the amplicon and sequence capacities when
 * those outputs are device memory, else sizes the context grows from earlier
 * calls; fewer than 65536 amplicons), else the call continues step by step
 * with up to three more.  Device outputs are complete when the call returns
 * (copies to host outputs too).  An output whose capacity is too small is not
 * written, its count is still reported, the others are written, and the call
 * returns AH_ERR_OVERFLOW.
 * Errors: AH_ERR_ARG, AH_ERR_OVERFLOW, AH_ERR_JIT, AH_ERR_TIMEOUT, AH_ERR_CUDA. */
ah_status ah_run(ah_ctx *ctx, uint32_t set_id, const uint32_t *pair_ids, uint32_t n_pairs, ah_run_out *out,
                 void *stream);

/* ah_run in two halves, for pipelines over many genome sets (this library's
 * addition; the paper processes one collection per run).  ah_run_begin
 * checks the arguments and queues the work on `stream` (a cudaStream_t, or
 * null for the context's stream) and returns; when scan_done (a cudaEvent_t
 * created by the caller, or null) is given it is recorded on that stream
 * right after the primer-matching kernel, so that work on another stream --
 * packing the next set with ah_load_genomes, say -- can wait for the scan
 * (cudaStreamWaitEvent) instead of competing with it, and then overlaps the
 * rest of the run.  ah_run_end waits for the queued work and completes `out`
 * exactly as ah_run does (same results, counts and errors, including
 * AH_ERR_OVERFLOW).  `out` and its buffers, the set and the pairs must stay
 * as they are until ah_run_end returns.  While a run is pending the only
 * calls accepted on the context are ah_load_genomes (not reversed),
 * ah_run_end, ah_get_profile, ah_last_error, ah_device_bytes and ah_destroy;
 * every other call returns AH_ERR_ARG.  When the last run needed the
 * step-by-step form, ah_run_begin already does the whole run and
 * ah_run_end returns its status.
 * Errors (begin): AH_ERR_ARG, AH_ERR_JIT, AH_ERR_CUDA; (end): those of ah_run. */
ah_status ah_run_begin(ah_ctx *ctx, uint32_t set_id, const uint32_t *pair_ids, uint32_t n_pairs, ah_run_out *out,
                       void *stream, void *scan_done);
ah_status ah_run_end(ah_ctx *ctx);

/* Tm-threshold sweep (Sec. 3.3, Annealing Temperature Optimization: how the
 * number of amplicons, the share of genomes amplified and the off-target
 * pattern counts move with the minimum annealing temperature).  sites (host
 * or device): n_sites records of the set and pairs, as ah_scan returns them;
 * amplicons (host or device): the set's amplicons called on those sites
 * without a Tm filter (ah_pair with pass = NULL), whose left/right fields
 * index `sites`.  thresholds (host): n_thresholds (1..64) values in deg C.
 * For threshold j, an amplicon counts when both of its sites pass, a site
 * passing when its maximum Tm over the primer's oligos is >= thresholds[j],
 * decided as the fp64 definition decides (as ah_tm's pass flag).  rows (host
 * or device): per threshold, the amplicons, those with orientation FF or RR,
 * and the genomes with at least one amplicon; *n_genomes_out: the set's
 * distinct genomes (the denominator of the share amplified).
 * Errors: AH_ERR_ARG (bad records or thresholds), AH_ERR_CUDA. */
typedef struct {
    uint64_t amplicons;
    uint64_t ff_rr;
    uint64_t genomes_amplified;
} ah_sweep_row;
ah_status ah_tm_sweep(ah_ctx *ctx, uint32_t set_id, const uint32_t *pair_ids, uint32_t n_pairs, const ah_site *sites,
                      uint64_t n_sites, const ah_amplicon *amplicons, uint64_t n_amplicons, const double *thresholds,
                      uint32_t n_thresholds, ah_sweep_row *rows, uint64_t *n_genomes_out, void *stream);

/* Amplicon sequence variants and amplitypes (Sec. 3.3, Amplicon Pattern
 * Visualization: the amplitype of a genome is which variants it carries and
 * how many copies of each).  amplicons (host or device): n records of the set (as
 * ah_pair returns them); the sequence of each is the one ah_fetch returns (RF
 * reverse-complemented, N for non-ACGT), hashed on the device (two
 * polynomial hashes modulo 2^61 - 1: 122 bits).  variant_out (host or device,
 * may be null): per amplicon, its variant id, numbered 0, 1, ... in order of
 * first occurrence in `amplicons`.  rows (host or device): one row per genome
 * with at least one amplicon, in ascending genome id: the genome, its
 * amplitype id (numbered by first occurrence in that order: genomes with the
 * same multiset of (variant, copy number) share it), its amplicon count and
 * its variant count; cap rows fit (cap = 0: size query; too small: nothing
 * written, *n_rows_out set, AH_ERR_OVERFLOW).  *n_variants_out and
 * *n_amplitypes_out: the distinct variants and amplitypes.
 * Errors: AH_ERR_ARG (records outside the set, genome not its contig's),
 * AH_ERR_OVERFLOW, AH_ERR_CUDA. */
typedef struct {
    uint32_t genome;
    uint32_t amplitype;
    uint32_t n_amplicons;
    uint32_t n_variants;
} ah_genome_amplitype;
ah_status ah_amplitypes(ah_ctx *ctx, uint32_t set_id, const ah_amplicon *amplicons, uint64_t n, uint32_t *variant_out,
                        ah_genome_amplitype *rows, uint64_t cap, uint64_t *n_rows_out, uint64_t *n_variants_out,
                        uint64_t *n_amplitypes_out, void *stream);

/* Synthetic genome bases on the device from a counter-based generator
 * (Philox4x32-10, Salmon et al., SC 2011) -- the library's input generator for
 * collections too large to build on the host (no counterpart in the paper).
 * Position P of the collection: the 32-bit draw u = output (P mod 4) of
 * Philox(counter = (P div 4 low 32 bits, high 32 bits, 0, 0), key = (seed low,
 * seed high)); in the segment holding P, the base is `letter` when non-zero,
 * else A if u < t_a, C if u < t_c, G if u < t_g, else T.  Segments (host) tile
 * the collection in order: segment i covers [end of i-1 (0 for the first),
 * end).  Patches (may be empty) then set out[pos - base0] = byte for every
 * pos inside the range.  out (device): n bytes for positions
 * [base0, base0 + n); base0 must be a multiple of 4, and the segments must
 * reach base0 + n.  Segments and patches are either host arrays (checked,
 * copied, and the call waits for the work) or device arrays of the whole
 * collection (stream-ordered: the call returns without waiting; a range the
 * segments do not cover is written as N and reported as AH_ERR_DEVICE_CHECK
 * by the next call that synchronises).
 * Errors: AH_ERR_ARG, AH_ERR_CUDA, AH_ERR_DEVICE_CHECK. */
typedef struct {
    uint64_t end;
    uint32_t t_a, t_c, t_g;
    uint32_t letter;
} ah_gen_segment;
ah_status ah_generate_bases(ah_ctx *ctx, uint64_t seed, const ah_gen_segment *segments, uint64_t n_segments,
                            const uint64_t *patch_pos, const uint8_t *patch_bytes, uint64_t n_patches, uint64_t base0,
                            uint64_t n, uint8_t *out, void *stream);

/* Measurement: per-stage device time, host time and kernel launches.
 * ah_set_profiling clears the counters; enable = 1 then brackets each stage
 * of each call with CUDA events on the stream the stage runs on and times
 * host sections, enable = 2 times host sections only, enable = 3 brackets
 * only the "pack" and "scan" stages (the streaming kernels; fewer events in
 * the stream) and times host sections, 0 stops.  Device
 * stages: "pack", "tables" (ah_load_genomes), "scan", "sort", "decode" (ah_scan),
 * "validate" (record checks of ah_tm / ah_pair), "tm", "pair", "fetch",
 * "sweep" (ah_tm_sweep), "amplitype" (ah_amplitypes), "generate"
 * (ah_generate_bases), "hmm" (ah_hmm_score).  Host sections (wall time
 * inside the library): "host.load", "host.load.alloc", "host.load.tables",
 * "host.load.pack", "host.run", "host.run.prep", "host.run.launch",
 * "host.run.wait", "host.unload", and for a server's batches
 * "host.serve.batch", "host.serve.tiles", "host.serve.device",
 * "host.serve.filter_wait", "host.serve.fetch".  ah_get_profile returns,
 * for one stage or section, the summed milliseconds, the kernels launched
 * and the number of bracketed calls; stage = NULL gives the sums over device
 * stages and the count of every kernel the library launched since the last
 * clear (counted whether or not profiling is on).  Event timings are read
 * lazily (at ah_get_profile at the latest).  Output pointers may be null. */
ah_status ah_set_profiling(ah_ctx *ctx, int enable);
ah_status ah_get_profile(const ah_ctx *ctx, const char *stage, double *ms, uint64_t *launches, uint64_t *calls);

/* Amplicon calling that allocates nothing (the paper has no counterpart: this
 * is a deployment variant of ah_pair).  For callers that must not allocate
 * device memory during the call -- an application whose own allocator owns
 * all of device memory, or a latency-bound loop that must stay off the
 * driver's allocator (cudaMalloc/cudaFree are slow and cudaFree synchronises
 * the device).  It runs the same pairing as ah_pair on the current CUDA
 * device and takes no context: its scratch lives in one fixed device array of
 * about 4.4 MB compiled into the library, which every GPU that loads the
 * library holds until the process exits.  The call waits on `stream` (it
 * reads the error word and the amplicon count back to the host).
 * pair_windows (host): n_pairs x 4 int32 {L_fwd, L_rev, min_len, max_len},
 *   indexed by ah_site.pair; 1 <= n_pairs <= 16, 1 <= L <= 32; checked on
 *   every call, also when n = 0.
 * sites, pass (may be null), out: device memory of the current device; sites
 *   in canonical order as ah_scan returns them.  n <= 262144 (1 << 18);
 *   larger n returns AH_ERR_ARG, as do host pointers, records whose pair,
 *   primer or strand is out of range, and lists out of canonical order.
 * Overflow contract as for every call (cap = 0 is a size query); *n_out host.
 * The first call on each device looks up the array's device address and
 * keeps it for the life of the process (the device's primary context must
 * not be reset in between).  All calls share the one array: calls that
 * overlap on the GPU (two streams or two threads) race and must not be made.
 * Errors: AH_ERR_ARG, AH_ERR_OVERFLOW, AH_ERR_CUDA (no message string). */
ah_status ah_pair_noalloc(const int32_t *pair_windows, uint32_t n_pairs, const ah_site *sites, const uint8_t *pass,
                          uint64_t n, ah_amplicon *out, uint64_t cap, uint64_t *n_out, void *stream);

/* Serving: continuous batching of requests over one resident genome set (a
 * deployment form with no counterpart in the paper; each request is the
 * paper's in-silico PCR of Sec. 2.1 restricted to some genomes of the set).
 * A request names genomes of the set (ids as in the load's contig_genome),
 * one primer pair (from ah_set_primers), a mismatch limit k (0..10, in place
 * of the pair's own) and whether the Tm filter applies.  Its result is what
 * the path gives for those genomes alone: the sites of the pair on their
 * contigs with mm <= k, in canonical order, and the amplicons among them
 * (both ends passing the Tm threshold when tm_filter is set), with `left`
 * and `right` indexing the request's own site list; contig ids are those of
 * the set.  A result does not depend on the other requests batched with it.
 *
 * ah_serve_start hands the context to a worker thread, which runs batches
 * back to back: each time the GPU is free it admits queued requests in
 * arrival order while their estimated device memory (sites and amplicons
 * scale with the request's bases) stays within cfg->mem_budget bytes, at
 * most cfg->max_batch of them and always at least one, and runs them
 * together (one scan per primer pair and k over the union of their genomes'
 * tiles).
 * Until ah_serve_stop no other call may use the context.
 * ah_serve_submit (any thread) queues a copy of the request and returns a
 * ticket.  ah_serve_wait (any thread) blocks until the ticket's request is
 * done, fills *info and copies its sites, amplicons and (when
 * seq_offsets_out is not NULL) the amplicon sequences, as ah_fetch gives
 * them, to the host arrays: seq_offsets_out takes n_amplicons + 1 offsets
 * into seq_out.  If a capacity is too small it returns AH_ERR_OVERFLOW with
 * the counts in *info and keeps the result for another wait; otherwise (or
 * on an error status) the ticket is released.  Times are milliseconds since
 * ah_serve_start on a steady clock: submit, start of the batch that ran the
 * request, and completion.  ah_serve_stop finishes the queued requests, joins
 * the worker and frees the server (unreleased results are dropped).
 * Errors: AH_ERR_ARG (bad argument, unknown pair, stopped server, unknown
 * ticket), AH_ERR_OVERFLOW, and any status of the underlying path. */
typedef struct ah_server ah_server;
typedef struct {
    size_t mem_budget;  /* bytes of device scratch one batch may plan for */
    uint32_t max_batch; /* requests per batch, >= 1 */
    uint32_t reserved;
} ah_serve_config;
typedef struct {
    const uint32_t *genomes; /* host: genome ids (duplicates and unknown ids are ignored) */
    uint32_t n_genomes;
    uint32_t pair_id;
    int32_t k;
    int32_t tm_filter;
} ah_request;
typedef struct {
    ah_status status;
    uint32_t batch;       /* 1-based number of the batch that ran the request */
    uint32_t batch_size;  /* requests in that batch */
    uint32_t reserved;
    uint64_t n_sites, n_amplicons, n_seq, bases; /* n_seq: sequence bytes */
    double submit_ms, start_ms, done_ms;
} ah_request_info;
ah_status ah_serve_start(ah_ctx *ctx, uint32_t set_id, const ah_serve_config *cfg, ah_server **out);
ah_status ah_serve_submit(ah_server *srv, const ah_request *req, uint64_t *ticket_out);
ah_status ah_serve_wait(ah_server *srv, uint64_t ticket, ah_request_info *info, ah_site *sites_out, uint64_t sites_cap,
                        ah_amplicon *amps_out, uint64_t amps_cap, char *seq_out, uint64_t seq_cap,
                        uint64_t *seq_offsets_out);
ah_status ah_serve_stop(ah_server *srv);

/* Profile-HMM homology scores (Sec. 2.1, Amplicon analysis, item 2: a profile
 * HMM trained on amplicons whose primers match exactly scores every predicted
 * amplicon).  The paper names no aligner, topology or score; this library
 * takes the following reading.  Profile: the most frequent training sequence
 * is the reference (the first on ties), m = its length (1..3071); each
 * training sequence is aligned to it globally with unit costs (0 for equal
 * A/C/G/T letters, 1 for any other pair and per gap), the traceback
 * preferring a diagonal step, then an insertion, then a deletion; the
 * alignments' state paths (begin B = M_0, match M_j, insert I_j after column
 * j, delete D_j, end E) give move counts from each state to the next
 * column's M (E after column m), to I_j and to the next column's D, and
 * letter counts per match column; probabilities are counts + 1 over the
 * allowed moves and over A/C/G/T; insert states emit the background.  Score:
 * the glocal Viterbi log-odds score (bits, uniform background; unknown
 * letters score 0) of an amplicon's sequence as ah_fetch returns it (RF
 * reverse-complemented), fp32; ah_hmm_forward gives the Forward score.
 * ah_hmm_build: training sequences (host, concatenated; offsets host, n + 1,
 *   from 0) -> a profile id; the profile lives on the device until
 *   ah_hmm_free or ah_destroy.  Errors: AH_ERR_ARG, AH_ERR_OOM.
 * ah_hmm_tables: m, the reference's index, and (when not NULL) the move
 *   scores t[(m + 1) * 9] = t[j][from][to] (from, to in M, I, D; -inf for a
 *   move that does not exist) and match emissions e[(m + 1) * 4] (row 0 is
 *   0), host arrays.
 * ah_hmm_score: one score per amplicon of the set (host or device records and
 *   scores); amplicons of up to 16,384 letters.  Errors: AH_ERR_ARG (unknown
 *   id, a record outside its contig, too long), AH_ERR_CUDA. */
ah_status ah_hmm_build(ah_ctx *ctx, const char *seqs, const uint64_t *offsets, uint64_t n, uint32_t *hmm_id_out);
ah_status ah_hmm_tables(ah_ctx *ctx, uint32_t hmm_id, uint64_t *m_out, uint64_t *reference_out, float *t_out,
                        float *e_out);
ah_status ah_hmm_score(ah_ctx *ctx, uint32_t set_id, uint32_t hmm_id, const ah_amplicon *amplicons, uint64_t n,
                       float *score_out, void *stream);
/* ah_hmm_forward: as ah_hmm_score, with the glocal Forward log-odds score
 * instead of Viterbi: log2 of the sum, over every state path from B to E that
 * emits the amplicon's sequence, of 2 to the path's score (bits, fp32; the
 * Viterbi recurrence with the maximum of the predecessors replaced by
 * log2(2^a + 2^b)).  Same arguments, limits and errors. */
ah_status ah_hmm_forward(ah_ctx *ctx, uint32_t set_id, uint32_t hmm_id, const ah_amplicon *amplicons, uint64_t n,
                         float *score_out, void *stream);
ah_status ah_hmm_free(ah_ctx *ctx, uint32_t hmm_id);

#ifdef __cplusplus
}
#endif

#endif /* AMPLICONHUNTER_H */
