// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "../../include/ampliconhunter.h"

namespace ah {

// ---------------------------------------------------------------------------
// Packed genome layout in HBM ("tile-strided one-hot bitplanes").
//
// The flat position space is the concatenation of all contigs of a set.  It
// is cut into tiles of kTileBases = 32 * kTileW positions.  Tile t stores, for
// each base plane x in {A, C, G, T}, kTileWX 32-bit words; bit b of word j of
// plane x is 1 iff the base at flat position
//     t * kTileBases + b * kTileW + j
// is x (upper or lower case).  For j >= kTileW the formula reaches into the
// next tile: these kTileExt "extension" words let a thread read the window
// of positions p .. p + L - 1 for every start p of its own words as plain
// word offsets j .. j + L - 1, with no funnel shifts (L <= 32).  A non-ACGT
// letter, and every position at or past the end of the set, has all four
// planes 0.  Layout: planes[(t * 4 + x) * kTileWX + j], 0.516 bytes per base.
// ---------------------------------------------------------------------------
constexpr int kTileW = 1024;
constexpr int kTileExt = 32;
constexpr int kTileWX = kTileW + kTileExt;
constexpr uint64_t kTileBases = 32ull * kTileW;
constexpr size_t kTileBytes = 4ull * kTileWX * sizeof(uint32_t);

struct GenomeSet {
    uint64_t n_bases = 0;
    uint32_t n_contigs = 0;
    uint64_t n_tiles = 0;
    uint32_t *planes = nullptr;        // device, n_tiles * kTileBytes
    uint64_t *contig_off = nullptr;    // device, n_contigs + 1
    uint32_t *contig_genome = nullptr; // device, n_contigs
    // device, n_tiles + 1: tile_contig[t] = the last contig starting at or before
    // position t * kTileBases (the contigs a tile's starts can fall in begin there)
    uint32_t *tile_contig = nullptr;
    // device, n_tiles + 1: bases from position t * kTileBases to the end of
    // contig tile_contig[t] (0 past the last base, capped at 2^32 - 1)
    uint32_t *tile_room = nullptr;
    // device, the no-base runs of a 2-bit load (read by its packing; the set owns
    // them so that loads in flight on other streams never share them)
    uint64_t *gaps = nullptr;
    size_t gaps_bytes = 0;
    size_t bytes = 0;
    // recorded after the work that fills the set (the packing); every call that
    // reads the set waits for it on its own stream, and unloading waits for it
    cudaEvent_t ready = nullptr;
    uint32_t max_genome = 0; // largest genome id
    uint64_t n_genomes = 0;  // distinct genome ids
    std::vector<uint64_t> contig_off_h;    // host copies (request planning of the server)
    std::vector<uint32_t> contig_genome_h;
};

// One registered primer pair.  mask[i] is the 4-bit IUPAC set of primer
// position i (A=1 C=2 G=4 T=8), 5'->3'.
struct PrimerPair {
    std::string fwd, rev;
    int L[2] = {0, 0};
    uint8_t mask[2][AH_MAX_PRIMER_LEN] = {};
    ah_pcr_params params{};
    ah_nn_table table{};
};

// One scan pattern: the primer (strand '+') or its reverse complement
// (strand '-') as matched against the + strand.
struct ScanPattern {
    int L = 0;
    int k = 0;
    int clamp = 0;
    int pair = 0;   // index in the ah_scan call's pair list
    int primer = 0; // 0 forward, 1 reverse
    int strand = 0; // 0 '+', 1 '-'
    uint8_t mask[AH_MAX_PRIMER_LEN] = {};
};

// A profile HMM (hmm.cu): m match columns; t[(m + 1) * 9] move scores
// t[j][from][to] (from, to in M, I, D; "to M" at j = m is the end state),
// -inf where a move does not exist; e[(m + 1) * 4] match emission scores
// (row 0 unused); bits against the uniform background.
constexpr int kHmmMaxColumns = 6 * 512; // m + 1 at most
constexpr uint32_t kHmmMaxLetters = 65536; // longest scored amplicon (shared memory of the kernel)
struct HmmProfile {
    int m = 0;
    uint64_t reference = 0; // index of the training sequence used as the reference
    std::vector<float> t, e;
    float *d_t = nullptr, *d_e = nullptr;
};
void build_profile(const char *seqs, const uint64_t *off, uint64_t n, HmmProfile &p);
// order: n indices into amps, amplicons of similar length next to each other;
// forward: the Forward (log-sum over paths) score instead of Viterbi
void launch_hmm_score(const ah_amplicon *amps, const uint32_t *order, uint64_t n, const uint32_t *planes,
                      const uint64_t *contig_off, uint32_t n_contigs, const float *t, const float *e, int m,
                      int max_len, bool forward, float *score_out, int *err, int sms, cudaStream_t s);

// Tunables of the generated scan kernel (autotuned per pattern set).
struct ScanTuning {
    int R = 4;            // 32-start words per thread (4 or 8: the loader reads 16-byte vectors at lane * R)
    int arith_pct = 0;    // share of full adders that form the sum with integer adds
    int min_blocks = 1;   // __launch_bounds__ minimum blocks per SM (with warps: a register cap)
    int order = 0;        // 0: word-major, 1: pattern-major code order
    int stages = 4;       // TMA stages per warp (2..4)
    int warps = 16;       // warps per CTA (1..16); 16 warps = a 128-register cap
    int resident = 0;     // CTAs launched per SM (0: as many as fit); fewer leave room for a
                          // kernel that runs beside the scan (the next set's packing)
};

struct ScanKernel {
    cudaLibrary_t lib = nullptr;
    cudaKernel_t fn = nullptr;
    int threads = 0;
    int blocks_per_sm = 0;
    size_t smem = 0;
    int regs = -1;
    std::string log;
};

class Error : public std::exception {
  public:
    Error(ah_status s, std::string m) : status(s), msg(std::move(m)) {}
    const char *what() const noexcept override { return msg.c_str(); }
    ah_status status;
    std::string msg;
};

#define AH_CUDA(call)                                                                                    \
    do {                                                                                                 \
        cudaError_t e_ = (call);                                                                         \
        if (e_ != cudaSuccess)                                                                           \
            throw ::ah::Error(AH_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));          \
    } while (0)

// Scratch buffer that grows on demand inside the context's budget.
struct Scratch {
    void *p = nullptr;
    size_t bytes = 0;
};

// Device error word layout (written by kernels, read by the host).
enum DeviceErr : int { kDevOk = 0, kDevTimeout = 1, kDevBounds = 2, kDevCheck = 3 };

// IUPAC letter -> 4-bit base set (A=1 C=2 G=4 T=8), 0 if not a code; and the
// complement of a base set (A<->T, C<->G).  Defined in ah_api.cu.
int iupac_mask(char ch);
int comp_mask(int m);

// ---- generated scan kernel (scan_jit.cu) ----
// Compile (no load) the scan kernel of one pair; for CPU-side checks of the
// generator.  Returns the NVRTC log (ptxas register report included).
std::string scan_compile_only(const std::vector<ScanPattern> &pats, const ScanTuning &t, bool *ok);
std::string scan_source(const std::vector<ScanPattern> &pats, const ScanTuning &t);
ScanKernel *scan_kernel(const std::vector<ScanPattern> &pats, const ScanTuning &t, int device);
// Launch groups of a pattern list, as [first, end) pattern index ranges:
// consecutive pairs share a launch while their generated network stays small
// (a larger one spills registers and misses in the instruction cache); a pair
// is never split.  At most AH_MAX_PAIRS_PER_SCAN groups.
std::vector<std::pair<int, int>> scan_launch_groups(const std::vector<ScanPattern> &pats);

// ---- kernel launchers ----
// pack.cu: pack tiles [t0, t1) from seq, which holds flat positions
// [seq_base, seq_base + seq_len) of a set of n_bases bases.
void launch_pack(const uint8_t *seq, uint64_t seq_base, uint64_t seq_len, uint64_t n_bases, uint32_t *planes,
                 uint64_t t0, uint64_t t1, int *err, cudaStream_t s);
// pack.cu: word copy by a kernel (src may be mapped host memory: no copy engine involved)
void launch_copy_words(const uint32_t *src, uint32_t *dst, uint64_t n_words, cudaStream_t s);
// Pack tiles [t0, t1) from 2-bit codes (A 0, C 1, G 2, T 3; base p in bits
// 2 (p % 4) of byte p / 4) whose first byte holds position base0 (a tile
// boundary) and that hold n_avail positions; gaps (device, n_gaps (start,
// length) pairs, sorted, disjoint) and positions >= n_bases are no base;
// tile_gap (device, one per tile + 1): the index of the first gap that ends
// after the tile's first position.  codes must be 16-byte aligned.
void launch_pack2(const uint8_t *codes, uint64_t base0, uint64_t n_avail, uint64_t n_bases, const uint64_t *gaps,
                  uint64_t n_gaps, const uint32_t *tile_gap, uint32_t *planes, uint64_t t0, uint64_t t1,
                  cudaStream_t s);
// One stretch of a contig-wise reversal: dst[k] = src[mirror - k] for k in
// [start, start + len) (mirror = 2 * contig start + contig length - 1).
struct RevChunk {
    uint64_t start, mirror;
    uint64_t len;
};
void launch_reverse_contigs(const uint8_t *src, uint8_t *dst, const RevChunk *chunks, uint64_t n_chunks,
                            cudaStream_t s);
void launch_unpack_check(const uint32_t *planes, uint64_t n_tiles, uint8_t *codes, uint64_t n_bases,
                         cudaStream_t s);

// sites.cu
size_t sort_keys_temp_bytes(uint64_t n, int end_bit);
void sort_keys(void *temp, size_t temp_bytes, const uint64_t *in, uint64_t *out, uint64_t n, int begin_bit,
               int end_bit, cudaStream_t s);
void launch_decode_keys(const uint64_t *keys, uint64_t n, int pbits, const uint64_t *contig_off, uint32_t n_contigs,
                        const uint32_t *contig_genome, ah_site *out, cudaStream_t s);
// Rank sort + decode (canonical order) for up to kSmallSort keys in one
// launch.  Host-count form: n_dev = nullptr, n = the count.  Device-count form
// (one-synchronisation path): the count is *n_dev and n is the largest count
// the launch was sized for; above it the kernel writes *n_out = 0, sets
// kRedoSites in *redo and sorts nothing.  Otherwise *n_out = the count.
// key32: the sort bits [8, end_bit) fit in 32 bits.
constexpr uint64_t kSmallSort = 16384;
void launch_rank_sort_decode(const uint64_t *keys, uint64_t n, const uint64_t *n_dev, bool key32, int pbits,
                             const uint64_t *contig_off, uint32_t n_contigs, const uint32_t *contig_genome,
                             ah_site *out, uint64_t *n_out, uint64_t *redo, cudaStream_t s);

// Device flag block of a context (u64 words, read by the host with one copy).
// The error word is last so that one memset clears every other word; it is
// cleared only after the host has read a non-zero value, so an error raised
// by a call that returns without synchronising reaches the next call that does.
enum FlagWord : int {
    kFlagCounter = 0, // scan hits appended
    kFlagAux = 1,     // a total computed on the device
    kFlagTmQueue = 2, // two words: sites queued for the exhaustive fp64 Tm and finished
                      // blocks (two u32), then sites deferred by the fast Tm kernel (u64)
    kFlagSites = 4,   // one-synchronisation path: sites sorted
    kFlagAmps = 5,    // ... amplicons
    kFlagSeq = 6,     // ... sequence bytes
    kFlagRedo = 7,    // ... kRedo* bits: a count above what the launches were sized for
    kFlagWork = 8,    // scan: slices claimed so far, one word per launch group (zeroed before a scan)
    kFlagErr = kFlagWork + AH_MAX_PAIRS_PER_SCAN, // DeviceErr (low 32 bits)
    kFlagWords = kFlagErr + 1
};
constexpr uint64_t kRedoSites = 1, kRedoAmps = 2, kRedoSeq = 4;

// Count of a kernel that may read it on the device: min(*n_dev, n), or n.
__device__ __forceinline__ uint64_t dev_count(uint64_t n, const uint64_t *n_dev)
{
    return n_dev ? (*n_dev < n ? *n_dev : n) : n;
}

struct PairDev;
// Check user-supplied sites before any kernel indexes memory with them:
// pair < n_pairs, primer and strand in {0, 1}, contig < n_contigs, and the
// window inside its contig.  Sets *err = kDevBounds on a bad record.
void launch_validate_sites(const ah_site *sites, uint64_t n, const PairDev *pairs_d, int n_pairs,
                           const uint64_t *contig_off, uint32_t n_contigs, int *err, cudaStream_t s);

// Per-pair constants for the Tm and pair kernels.  The fp64 fields are the
// exact host values of the model's constants (same expressions as the
// reference definition), so device fp64 Tm values can be bit-identical.
struct PairDev {
    int L[2];
    int min_len, max_len;
    uint8_t mask[2][AH_MAX_PRIMER_LEN];
    // Tm shortest-path steps: positions 0 and L-1 and every degenerate position, ascending
    int nkey[2];
    uint8_t key[2][AH_MAX_PRIMER_LEN];
    // 1 when every duplex of either primer has dS + C < 0 (a bound from the table's
    // largest entries): only sites within ~1e-9 K of tm_min can need exhaustive fp64
    int few_exact;
    float tm_min_f;
    int saltcorr;
    double tm_min;
    double thr;      // tm_min as a ratio 1000 dH / (dS + C) in kelvin: tm_min + 273.15 (- shift, methods 1-4)
    double sconst;   // R ln(x), x = (dnac1 - dnac2/2) 1e-9
    double log_na;   // ln([Na_eq] in mol/L); salt method 5 adds 0.368 (L-1) log_na to dS
    double tm_shift; // salt methods 1-4
    float stack_dH[256], stack_dS[256], term_dH[16], term_dS[16];
    double stack_dH_d[256], stack_dS_d[256], term_dH_d[16], term_dS_d[16];
};

// tm.cu
// queue: n entries of scratch for the sites decided by exhaustive fp64
// enumeration; queue_n: four device u32 words (queue length, finished
// blocks, then a u64 count of deferred sites; zeroed here).  queue holds 2 n
// entries: the exhaustive queue, then the list of deferred sites.  seg_max:
// the largest nkey - 1 over the pairs' primers.  few_exact (all pairs'
// few_exact): a thread-per-site kernel computes every site and defers those
// within 0.01 C of tm_min to the four-lane kernel, whose last block evaluates
// the exhaustive queue; else the four-lane kernel takes every site and a
// second kernel works off the queue, a block per site.
// n_dev: optional device count (min(*n_dev, n) sites).
void launch_tm(const ah_site *sites, uint64_t n, const uint64_t *n_dev, const PairDev *pairs_d, int n_pairs, const uint32_t *planes,
               const uint64_t *contig_off, float *tm_out, uint8_t *pass_out, uint32_t *queue, uint32_t *queue_n,
               int seg_max, bool few_exact, int *err, cudaStream_t s);

// Tm-threshold sweep (tm.cu): per-site pass bits for n_thr <= 64 thresholds
// (thr_d: deg C, device), then per threshold the amplicons whose two sites
// pass, those with orientation FF or RR, and the genomes with at least one.
// counts: 192 device words ([0, 64) amplicons, [64, 128) FF/RR, [128, 192)
// genomes); W: n_pairs * n_thr * 272 words; pass_mask: n_sites words; gmask:
// max_genome + 1 words.  tm: the sites' fp32 maxima (launch_tm).
constexpr int kSweepThresholds = 64;
void launch_tm_sweep(const ah_site *sites, uint64_t n_sites, const ah_amplicon *amps, uint64_t n_amps,
                     const PairDev *pairs_d, int n_pairs, const uint32_t *planes, const uint64_t *contig_off,
                     const float *tm, const double *thr_d, int n_thr, long long *W, bool few_exact,
                     uint64_t *pass_mask, unsigned long long *gmask, uint32_t max_genome, unsigned long long *counts,
                     int *err, cudaStream_t s);

// pair.cu
// n_dev (here and below): optional device count, min(*n_dev, n) records.
void launch_pair_count(const ah_site *sites, uint64_t n, const uint64_t *n_dev, const uint8_t *pass,
                       const PairDev *pairs_d, uint64_t *counts, cudaStream_t s);
// *out = offs[m-1] + counts[m-1] (the total of an exclusive scan over m values,
// m = n or min(*n_dev + add, n)).  With eff != nullptr also *eff = the total if it
// is at most cap, else 0 with redo_bit set in *redo.
void launch_total(const uint64_t *offs, const uint64_t *counts, uint64_t n, const uint64_t *n_dev, uint64_t add,
                  uint64_t *out, uint64_t cap, uint64_t *eff, uint64_t *redo, uint64_t redo_bit, cudaStream_t s);
size_t scan_u64_temp_bytes(uint64_t n);
// Exclusive scan of n u64 values; one block (no temporary) for n <= kSmallScan, CUB above.
constexpr uint64_t kSmallScan = 65536;
// number of kernels exclusive_scan_u64 launches for n values
int scan_u64_launches(uint64_t n);
void exclusive_scan_u64(void *temp, size_t temp_bytes, const uint64_t *in, uint64_t *out, uint64_t n, cudaStream_t s);
// One-block exclusive scan of min(*n_dev + add, n) values (n <= kSmallScan);
// with tot also their sum, and with eff the capacity check of launch_total.
void exclusive_scan_u64_dev(const uint64_t *in, uint64_t *out, uint64_t n, const uint64_t *n_dev, uint64_t add,
                            uint64_t *tot, uint64_t cap, uint64_t *eff, uint64_t *redo, uint64_t redo_bit,
                            cudaStream_t s);
// skip: optional device word; the kernel writes nothing when (*skip & skip_bit) != 0.
void launch_pair_write(const ah_site *sites, uint64_t n, const uint64_t *n_dev, const uint8_t *pass,
                       const PairDev *pairs_d, const uint64_t *offsets, ah_amplicon *out, uint64_t cap,
                       const uint64_t *skip, uint64_t skip_bit, cudaStream_t s);

// amplitype.cu: sequence variants and amplitypes.  Every array holds at
// least the largest count it serves (amplicons, or genomes with amplicons).
struct AmpliTypeScratch {
    uint32_t *idx = nullptr, *idx_b = nullptr, *run_pos = nullptr;
    uint64_t *keys_a = nullptr, *keys_b = nullptr, *keys_s = nullptr;
    uint64_t *head = nullptr, *head_excl = nullptr, *is_first = nullptr, *rank = nullptr;
    bool keys_b_valid = false;
    void *temp = nullptr; // CUB sort storage
    size_t temp_bytes = 0;
    void *scan_temp = nullptr; // CUB scan storage (more than kSmallScan values)
    size_t scan_bytes = 0;
    // stable sort of the element indices by (ka, kb) (kb may be null)
    void sort_by(const uint64_t *ka, const uint64_t *kb, uint64_t n, cudaStream_t s);
    // runs of equal keys after sort_by; with id_out, first-occurrence ids per element
    void ids(uint64_t n, uint32_t *id_out, uint64_t *n_runs_dev, cudaStream_t s);
    // after sort_by + ids over (genome << 32 | variant) keys: per-genome multiset sums and counts
    void genome_sums(uint64_t n, const uint64_t *n_runs_dev, unsigned long long *g1, unsigned long long *g2,
                     unsigned int *gamp, unsigned int *gvar, cudaStream_t s);
    static size_t cub_bytes(uint64_t n);
};
void launch_amp_hash(const ah_amplicon *a, uint64_t n, const uint32_t *planes, const uint64_t *contig_off,
                     uint64_t *h1, uint64_t *h2, cudaStream_t s);
// key (genome << 32 | variant) per amplicon; an amplicon whose genome differs
// from its contig's, or with orientation > 3, sets *err = kDevBounds
void launch_genome_key(const ah_amplicon *a, const uint32_t *variant, uint64_t n, const uint32_t *contig_genome,
                       uint64_t *keys, int *err, cudaStream_t s);
void launch_genome_compact(const unsigned int *gamp, uint64_t n_ids, uint64_t *has, uint64_t *pos, void *scan_temp,
                           size_t scan_bytes, const unsigned long long *g1, const unsigned long long *g2, uint32_t *gid,
                           uint64_t *k1, uint64_t *k2, uint64_t *n_out_dev, cudaStream_t s);
void launch_amplitype_rows(const uint32_t *gid, const uint32_t *type, uint64_t m, const unsigned int *gamp,
                           const unsigned int *gvar, ah_genome_amplitype *rows, cudaStream_t s);

// gen.cu: counter-based synthetic bases (device segments and patches)
void launch_generate_bases(const ah_gen_segment *segs, uint64_t n_segs, uint64_t seed, const uint64_t *patch_pos,
                           const uint8_t *patch_bytes, uint64_t n_patches, uint64_t base0, uint64_t n, uint8_t *out,
                           int *err, cudaStream_t s);

// fetch.cu
// lengths of the amplicons; a record outside its contig sets *err = kDevBounds (length 0)
// With n_dev the kernel also writes len[count] = 0 (the scan's closing entry).
void launch_fetch_lengths(const ah_amplicon *a, uint64_t n, const uint64_t *n_dev, const uint64_t *contig_off,
                          uint32_t n_contigs, uint64_t *len, int *err, cudaStream_t s);
void launch_fetch(const ah_amplicon *a, uint64_t n, const uint64_t *n_dev, const uint64_t *offsets,
                  const uint32_t *planes, const uint64_t *contig_off, char *out, const uint64_t *skip,
                  uint64_t skip_bit, cudaStream_t s);

} // namespace ah
