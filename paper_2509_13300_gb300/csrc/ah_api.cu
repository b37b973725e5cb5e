// C ABI of the in-silico PCR hot path: context, genome pool, primer
// registry, pointer staging and the call sequences of ah_scan / ah_tm /
// ah_pair / ah_fetch.  All arithmetic runs in the kernels of this library.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <condition_variable>
#include <deque>
#include <future>
#include <mutex>
#include <new>
#include <thread>

#include "ah_internal.h"
#include "hmm.h"

using namespace ah;

struct ah_ctx {
    int device = 0;
    int sms = 0;
    size_t budget = 0; // 0 = unlimited
    size_t used = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    std::map<uint32_t, std::unique_ptr<GenomeSet>> sets;
    uint32_t next_set = 1;
    std::map<uint32_t, PrimerPair> pairs;
    std::map<uint32_t, HmmProfile> hmms;
    uint32_t next_hmm = 1;
    uint32_t next_pair = 1;
    std::map<std::string, Scratch> scratch;
    // device flag block (FlagWord layout)
    uint64_t *d_flags = nullptr;
    uint64_t *d_counter = nullptr;
    uint64_t *d_aux = nullptr;
    int *d_err = nullptr;
    cudaStream_t copy_stream = nullptr; // host->device copies that overlap packing
    // ah_run's kernels go on this stream, created with the highest priority and
    // joined to the caller's stream by events: when the next set's packing runs
    // beside a run's later stages, the block scheduler prefers the run's blocks
    cudaStream_t run_stream = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaEvent_t ev_copied[2] = {nullptr, nullptr}, ev_packed[2] = {nullptr, nullptr};
    cudaEvent_t ev_load_start = nullptr; // a host load's copies start after the caller's earlier work
    cudaEvent_t ev_last_copy = nullptr;  // recorded after a host load's last copy
    uint64_t *h_flags = nullptr;     // pinned host mirror of the flag block
    // test of the timeout path (ah_debug_scan_stall): each warp's first slice
    // is armed without a copy and the per-slice wait limit drops to 20 us
    bool scan_stall_first = false;
    bool flags_dirty = false;        // work was queued that may set the error word, not read since
    std::vector<cudaEvent_t> set_events; // free "ready" events of genome sets
    // mapped pinned staging of the contig tables, read on the device by a copy
    // kernel (a copy-engine transfer would queue behind large host->device
    // copies of the caller's); a ring of slots, so that a load waits only for
    // the reads of the load four before it
    static constexpr int kPinSlots = 4;
    struct PinSlot {
        uint8_t *p = nullptr;  // host address
        uint8_t *dp = nullptr; // device address of the same memory
        size_t bytes = 0;
        cudaEvent_t ev = nullptr; // recorded after the reads out of the slot
    } pin[kPinSlots];
    int pin_next = 0;
    std::vector<PairDev> pairdev_h;  // host source of the last per-pair upload
    std::vector<uint32_t> pairdev_ids; // pair ids of that upload
    uint64_t pairdev_version = 0;      // pairs_version at that upload
    const PairDev *pairdev_d = nullptr;
    uint64_t pairs_version = 1;        // bumped whenever a registered pair changes
    ScanTuning tuning;                          // default tuning
    std::map<std::string, ScanTuning> tuned;    // autotuned, per pattern-set signature
    uint64_t key_cap = 1 << 20;
    // one-synchronisation run: sizes of its scratch outputs, grown from the
    // counts of runs that needed more; the last run's site count
    uint64_t fast_amps = 16384, fast_seq = 4u << 20;
    uint64_t last_sites = 0;
    // a run queued by ah_run_begin and not yet completed by ah_run_end
    struct FastRun {
        bool sites_direct = false, amps_direct = false, seq_direct = false;
        uint64_t *keys = nullptr;
        ah_site *sites = nullptr;
        float *tm = nullptr;
        uint8_t *pass = nullptr;
        ah_amplicon *amps = nullptr;
        uint64_t *qoff = nullptr;
        char *seq = nullptr;
    };
    struct RunPending {
        bool active = false, done = false; // done: completed already by ah_run_begin
        bool scan_only = false;            // only the scan was queued: ah_run_end finishes step by step
        ah_status status = AH_OK;
        std::string msg;
        uint32_t set_id = 0;
        std::vector<uint32_t> pair_ids;
        ah_run_out *o = nullptr;
        cudaStream_t st = nullptr;     // the run stream
        cudaStream_t caller = nullptr; // the caller's stream
        const PairDev *pd = nullptr;
        FastRun fr;
    } pend;
    cudaEvent_t ev_run = nullptr; // recorded after the flag copy of a queued run
    bool serving = false;         // a server's worker thread owns the context
    // caching allocator: large blocks released by the library are kept for reuse
    std::map<void *, size_t> live;             // block -> bytes
    std::multimap<size_t, void *> cached;      // bytes -> block
    // per-stage profiling (CUDA events on the launching stream)
    struct Prof {
        double ms = 0;
        uint64_t launches = 0, calls = 0;
    };
    struct Pending {
        std::string stage;
        cudaEvent_t a, b;
        int launches;
    };
    bool profiling = false;  // stage events
    bool prof_streaming_only = false; // events on the "pack" and "scan" stages only
    bool host_timing = false; // host sections
    std::map<std::string, Prof> prof;
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> events;
    uint64_t launches_total = 0;
};

namespace {

std::mutex g_create_mu;
std::string g_create_err;

void prof_flush(ah_ctx *c);

template <class F> ah_status guarded(ah_ctx *ctx, F &&f)
{
    try {
        if (ctx)
            AH_CUDA(cudaSetDevice(ctx->device));
        f();
        if (ctx && ctx->pending.size() >= 4096) // event timings are read lazily
            prof_flush(ctx);
        return AH_OK;
    } catch (const Error &e) {
        if (ctx)
            ctx->err = e.msg;
        return e.status;
    } catch (const std::bad_alloc &) {
        if (ctx)
            ctx->err = "host allocation failed";
        return AH_ERR_OOM;
    } catch (const std::exception &e) {
        if (ctx)
            ctx->err = e.what();
        return AH_ERR_ARG;
    }
}

// (a literal message builds no string unless the check fails: these run in per-contig loops)
void require(bool cond, ah_status st, const char *msg)
{
    if (!cond)
        throw Error(st, msg);
}

void require(bool cond, ah_status st, const std::string &msg)
{
    if (!cond)
        throw Error(st, msg);
}


void release_cached(ah_ctx *c, size_t need)
{
    // free cached blocks (largest first) until `need` more bytes fit the budget
    while (!c->cached.empty() && (need == SIZE_MAX || (c->budget && c->used + need > c->budget))) {
        auto it = std::prev(c->cached.end());
        cudaFree(it->second);
        c->used -= std::min(c->used, it->first);
        c->live.erase(it->second);
        c->cached.erase(it);
    }
}

void *dev_alloc(ah_ctx *c, size_t bytes)
{
    if (bytes == 0)
        bytes = 16;
    { // reuse a cached block of at most twice the size (cudaFree would synchronise the device)
        auto it = c->cached.lower_bound(bytes);
        if (it != c->cached.end() && it->first <= 2 * bytes) {
            void *p = it->second;
            c->cached.erase(it);
            return p;
        }
    }
    if (c->budget && c->used + bytes > c->budget)
        release_cached(c, bytes);
    if (c->budget && c->used + bytes > c->budget)
        throw Error(AH_ERR_BUDGET, "device-memory budget exceeded: need " + std::to_string(bytes) + " more bytes, " +
                                       std::to_string(c->budget - c->used) + " left");
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        release_cached(c, SIZE_MAX);
        e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            throw Error(AH_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
        }
    }
    c->used += bytes;
    c->live[p] = bytes;
    return p;
}

void dev_free(ah_ctx *c, void *p, size_t)
{
    if (!p)
        return;
    auto it = c->live.find(p);
    if (it == c->live.end())
        return;
    c->cached.emplace(it->second, p); // kept for reuse; released under budget pressure or at ah_destroy
}

cudaEvent_t get_event(ah_ctx *c)
{
    if (!c->events.empty()) {
        cudaEvent_t e = c->events.back();
        c->events.pop_back();
        return e;
    }
    cudaEvent_t e;
    AH_CUDA(cudaEventCreate(&e));
    return e;
}

// Scope of one pipeline stage: counts its kernel launches and, when
// profiling, brackets it with events on the launching stream.
struct Stage {
    ah_ctx *c;
    const char *name;
    cudaStream_t st;
    int launches;
    cudaEvent_t a = nullptr;
    Stage(ah_ctx *c_, const char *n, cudaStream_t s, int l) : c(c_), name(n), st(s), launches(l)
    {
        c->launches_total += (uint64_t)l;
        if (c->profiling && (!c->prof_streaming_only || !strcmp(n, "pack") || !strcmp(n, "scan"))) {
            a = get_event(c);
            cudaEventRecord(a, st);
        }
    }
    ~Stage()
    {
        if (a) {
            cudaEvent_t b = get_event(c);
            cudaEventRecord(b, st);
            c->pending.push_back({name, a, b, launches});
        }
    }
};

// Host wall time of one section of a call, when host timing is on.
struct HostSpan {
    ah_ctx *c;
    const char *name;
    std::chrono::steady_clock::time_point t0;
    HostSpan(ah_ctx *c_, const char *n) : c(c_), name(n)
    {
        if (c->host_timing)
            t0 = std::chrono::steady_clock::now();
    }
    ~HostSpan()
    {
        if (c->host_timing) {
            auto &q = c->prof[name];
            q.ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
            q.calls += 1;
        }
    }
};

// Kernels CUB launches for our calls (counted in an ncu launch list on a
// GB300): a one-sweep radix sort runs a histogram kernel, an exclusive-sum
// kernel and one pass per 8 key bits; a device-wide scan runs an init kernel
// and a scan kernel.
int cub_sort_launches(uint64_t n, int bits) { return n <= 1 ? 0 : 2 + (bits + 7) / 8; }

void prof_flush(ah_ctx *c)
{
    for (auto &p : c->pending) {
        float ms = 0;
        if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            auto &q = c->prof[p.stage];
            q.ms += ms;
            q.launches += (uint64_t)p.launches;
            q.calls += 1;
        }
        cudaGetLastError();
        c->events.push_back(p.a);
        c->events.push_back(p.b);
    }
    c->pending.clear();
}

void *scratch(ah_ctx *c, const std::string &name, size_t bytes)
{
    Scratch &s = c->scratch[name];
    if (s.bytes >= bytes && s.p)
        return s.p;
    if (s.p) {
        AH_CUDA(cudaStreamSynchronize(c->stream));
        dev_free(c, s.p, s.bytes);
        s.p = nullptr;
        s.bytes = 0;
    }
    size_t want = std::max<size_t>(bytes + bytes / 4, 4096);
    s.p = dev_alloc(c, want);
    s.bytes = want;
    return s.p;
}

// The next mapped pinned slot of the ring, holding at least `bytes`: host data
// that a copy kernel reads over the link (a copy-engine transfer would queue
// behind a large host->device copy still in flight); waits only for the reads
// of the slot's earlier use.
ah_ctx::PinSlot &pin_slot(ah_ctx *c, size_t bytes)
{
    ah_ctx::PinSlot &sl = c->pin[c->pin_next];
    c->pin_next = (c->pin_next + 1) % ah_ctx::kPinSlots;
    AH_CUDA(cudaEventSynchronize(sl.ev)); // the slot's earlier reads are done
    if (sl.bytes < bytes) {
        if (sl.p)
            AH_CUDA(cudaFreeHost(sl.p));
        sl.p = sl.dp = nullptr;
        sl.bytes = 0;
        // a power of two: slots grow rarely (freeing pinned memory synchronises the device)
        size_t want = (size_t)1 << 20;
        while (want < bytes)
            want <<= 1;
        AH_CUDA(cudaHostAlloc((void **)&sl.p, want, cudaHostAllocMapped));
        sl.bytes = want;
        AH_CUDA(cudaHostGetDevicePointer((void **)&sl.dp, sl.p, 0));
    }
    return sl;
}

// The staging buffers of host loads: one holding a set's whole input when it
// fits (at most kHostStageMax bytes, and 1/16 of a memory budget), so that its
// copy runs beside the previous run's scan instead of waiting for the packing of
// earlier pieces; else two of that size, used in turn.  Before a buffer is
// replaced, every earlier copy into it and every packing from it has finished.
// Returns the bytes each buffer in use holds (stage[1] is null for one buffer).
constexpr uint64_t kHostStageMax = (4ull << 30) + (1ull << 20);
uint64_t host_stage(ah_ctx *c, uint64_t want, uint8_t *stage[2])
{
    uint64_t cap = std::min<uint64_t>(want, kHostStageMax);
    if (const char *e = getenv("AH_HOST_STAGE_MB")) // profiling aid: a smaller cap
        if (atoll(e) > 0)
            cap = std::min<uint64_t>(cap, (uint64_t)atoll(e) << 20);
    if (c->budget)
        cap = std::min<uint64_t>(cap, std::max<uint64_t>(c->budget / 16, 64ull << 20));
    cap = std::max<uint64_t>(cap, 1ull << 20);
    const bool two = want > cap;
    Scratch &s0 = c->scratch["load_stage0"], &s1 = c->scratch["load_stage1"];
    if (s0.bytes < cap || (two && s1.bytes < cap)) {
        for (int b = 0; b < 2; ++b) {
            AH_CUDA(cudaEventSynchronize(c->ev_copied[b]));
            AH_CUDA(cudaEventSynchronize(c->ev_packed[b]));
        }
        AH_CUDA(cudaEventSynchronize(c->ev_last_copy));
    }
    stage[0] = (uint8_t *)scratch(c, "load_stage0", cap);
    stage[1] = two ? (uint8_t *)scratch(c, "load_stage1", cap) : nullptr;
    return two ? std::min(c->scratch["load_stage0"].bytes, c->scratch["load_stage1"].bytes)
               : c->scratch["load_stage0"].bytes;
}

bool is_device_ptr(ah_ctx *c, const void *p)
{
    if (!p)
        return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) {
        if (a.type == cudaMemoryTypeDevice && a.device != c->device)
            throw Error(AH_ERR_ARG, "device pointer belongs to another GPU");
        return true;
    }
    return false;
}

cudaStream_t stream_of(ah_ctx *c, void *s) { return s ? (cudaStream_t)s : c->stream; }

template <class T> const T *stage_in(ah_ctx *c, const char *name, const T *p, uint64_t count, cudaStream_t st)
{
    if (is_device_ptr(c, p) || count == 0)
        return p;
    T *d = (T *)scratch(c, name, count * sizeof(T));
    AH_CUDA(cudaMemcpyAsync(d, p, count * sizeof(T), cudaMemcpyHostToDevice, st));
    return d;
}

template <class T> T *out_buf(ah_ctx *c, const char *name, T *p, uint64_t count)
{
    if (count == 0 || is_device_ptr(c, p))
        return p;
    return (T *)scratch(c, name, count * sizeof(T));
}

template <class T> void out_finish(T *user, T *dev, uint64_t count, cudaStream_t st)
{
    if (count && user != dev)
        AH_CUDA(cudaMemcpyAsync(user, dev, count * sizeof(T), cudaMemcpyDeviceToHost, st));
}

// Zero every flag word but the error word.
void reset_flags(ah_ctx *c, cudaStream_t st)
{
    AH_CUDA(cudaMemsetAsync(c->d_flags, 0, kFlagErr * sizeof(uint64_t), st));
}

// One device->host copy of the flag block and one synchronisation; returns
// the device error word and clears it on the device when it is set.
int read_flags(ah_ctx *c, cudaStream_t st)
{
    AH_CUDA(cudaMemcpyAsync(c->h_flags, c->d_flags, kFlagWords * sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    AH_CUDA(cudaStreamSynchronize(st));
    c->flags_dirty = false;
    const int e = (int)(c->h_flags[kFlagErr] & 0xffffffffu);
    if (e != 0)
        AH_CUDA(cudaMemsetAsync(c->d_flags + kFlagErr, 0, sizeof(uint64_t), st));
    return e;
}

void raise_device_error(int e)
{
    if (e == kDevTimeout)
        throw Error(AH_ERR_TIMEOUT, "a device-side wait ran out of iterations");
    if (e == kDevBounds)
        throw Error(AH_ERR_ARG, "input record out of range (pair, contig or position)");
    if (e != 0)
        throw Error(AH_ERR_DEVICE_CHECK, "device consistency check failed (code " + std::to_string(e) + ")");
}

// read_flags, then raise on a device-reported error.  h_flags[kFlagCounter]
// = scan hits, h_flags[kFlagAux] = a device total.
void check_flags(ah_ctx *c, cudaStream_t st) { raise_device_error(read_flags(c, st)); }

GenomeSet &get_set(ah_ctx *c, uint32_t id)
{
    auto it = c->sets.find(id);
    require(it != c->sets.end(), AH_ERR_ARG, "unknown genome set id " + std::to_string(id));
    return *it->second;
}

// Order the caller's stream after the work that filled the set (which may
// have been queued on another stream without a synchronisation).
void wait_ready(const GenomeSet &gs, cudaStream_t st)
{
    if (gs.ready)
        AH_CUDA(cudaStreamWaitEvent(st, gs.ready, 0));
}

PrimerPair &get_pair(ah_ctx *c, uint32_t id)
{
    auto it = c->pairs.find(id);
    require(it != c->pairs.end(), AH_ERR_ARG, "unknown primer pair id " + std::to_string(id));
    return it->second;
}

} // namespace

// IUPAC letter -> 4-bit base set (A=1 C=2 G=4 T=8); 0 for anything else.
int ah::iupac_mask(char ch)
{
    switch (ch >= 'a' && ch <= 'z' ? ch - 32 : ch) {
    case 'A': return 1;
    case 'C': return 2;
    case 'G': return 4;
    case 'T': return 8;
    case 'R': return 1 | 4;
    case 'Y': return 2 | 8;
    case 'S': return 2 | 4;
    case 'W': return 1 | 8;
    case 'K': return 4 | 8;
    case 'M': return 1 | 2;
    case 'B': return 2 | 4 | 8;
    case 'D': return 1 | 4 | 8;
    case 'H': return 1 | 2 | 8;
    case 'V': return 1 | 2 | 4;
    case 'N': return 15;
    default: return 0;
    }
}

// complement of a base set: A<->T, C<->G
int ah::comp_mask(int m) { return ((m & 1) << 3) | ((m & 8) >> 3) | ((m & 2) << 1) | ((m & 4) >> 1); }

namespace {

// Default NN table: SantaLucia (1998) unified Watson-Crick parameters, here
// indexed by the top-strand dinucleotide (each has exactly one Watson-Crick
// stack), and terminal initiation by the class of the primer base.
void default_table(ah_nn_table *t)
{
    static const double dH[4][4] = {{-7.9, -8.4, -7.8, -7.2},
                                    {-8.5, -8.0, -10.6, -7.8},
                                    {-8.2, -9.8, -8.0, -8.4},
                                    {-7.2, -8.2, -8.5, -7.9}};
    static const double dS[4][4] = {{-22.2, -22.4, -21.0, -20.4},
                                    {-22.7, -19.9, -27.2, -21.0},
                                    {-22.2, -24.4, -19.9, -22.4},
                                    {-21.3, -22.2, -22.7, -22.2}};
    memset(t, 0, sizeof(*t));
    for (int x = 0; x < 4; ++x)
        for (int y = 0; y < 4; ++y) {
            const int idx = ((x * 4 + y) * 4 + (3 - x)) * 4 + (3 - y);
            t->stack_dH[idx] = dH[x][y];
            t->stack_dS[idx] = dS[x][y];
        }
    for (int p = 0; p < 4; ++p)
        for (int q = 0; q < 4; ++q) {
            const bool gc = (p == 1 || p == 2);
            t->term_dH[p * 4 + q] = gc ? 0.1 : 2.3;
            t->term_dS[p * 4 + q] = gc ? -2.8 : 4.1;
        }
}

double na_eq_mM(const ah_pcr_params &p)
{
    double mon = p.Na_mM + p.K_mM + p.Tris_mM / 2.0;
    if (p.Mg_mM > p.dNTPs_mM)
        mon += 120.0 * std::sqrt(p.Mg_mM - p.dNTPs_mM);
    return mon;
}

PairDev make_pair_dev(const PrimerPair &pp)
{
    PairDev d;
    memset(&d, 0, sizeof(d));
    d.L[0] = pp.L[0];
    d.L[1] = pp.L[1];
    d.min_len = pp.params.min_len;
    d.max_len = pp.params.max_len;
    memcpy(d.mask, pp.mask, sizeof(d.mask));
    for (int x = 0; x < 2; ++x) { // Tm shortest-path keys: both ends and every degenerate position
        int nk = 0;
        for (int q = 0; q < pp.L[x]; ++q)
            if (q == 0 || q == pp.L[x] - 1 || __builtin_popcount(pp.mask[x][q]) > 1)
                d.key[x][nk++] = (uint8_t)q;
        d.nkey[x] = nk;
    }
    d.tm_min = pp.params.tm_min;
    d.tm_min_f = (float)pp.params.tm_min;
    const double x = (pp.params.dnac1_nM - pp.params.dnac2_nM / 2.0) * 1e-9;
    d.sconst = 1.987 * std::log(x);
    const double na = na_eq_mM(pp.params) / 1000.0;
    d.saltcorr = pp.params.saltcorr;
    d.log_na = pp.params.saltcorr == 5 ? std::log(na) : 0.0;
    d.tm_shift = pp.params.saltcorr == 1 ? 16.6 * std::log10(na) : 0.0; // Schildkraut-Lifson (1965)
    d.thr = d.tm_min + 273.15 - d.tm_shift;
    for (int i = 0; i < 256; ++i) {
        d.stack_dH[i] = (float)pp.table.stack_dH[i];
        d.stack_dS[i] = (float)pp.table.stack_dS[i];
        d.stack_dH_d[i] = pp.table.stack_dH[i];
        d.stack_dS_d[i] = pp.table.stack_dS[i];
    }
    for (int i = 0; i < 16; ++i) {
        d.term_dH[i] = (float)pp.table.term_dH[i];
        d.term_dS[i] = (float)pp.table.term_dS[i];
        d.term_dH_d[i] = pp.table.term_dH[i];
        d.term_dS_d[i] = pp.table.term_dS[i];
    }
    // largest possible dS + C of a duplex of each primer, from the table's largest entries
    double max_st = -INFINITY, max_tm = -INFINITY;
    for (int i = 0; i < 256; ++i)
        max_st = std::max(max_st, pp.table.stack_dS[i]);
    for (int i = 0; i < 16; ++i)
        max_tm = std::max(max_tm, pp.table.term_dS[i]);
    d.few_exact = 1;
    for (int x = 0; x < 2; ++x) {
        const int L = pp.L[x];
        const double salt = d.saltcorr == 5 ? 0.368 * (double)(L - 1) * d.log_na : 0.0;
        if (!((L - 1) * max_st + 2 * max_tm + d.sconst + salt < -1e-3))
            d.few_exact = 0;
    }
    return d;
}

const PairDev *upload_pairs(ah_ctx *c, const uint32_t *pair_ids, uint32_t n_pairs, cudaStream_t st)
{
    require(pair_ids != nullptr, AH_ERR_ARG, "pair_ids is null");
    require(n_pairs >= 1 && n_pairs <= AH_MAX_PAIRS_PER_SCAN, AH_ERR_ARG, "n_pairs must be 1..16");
    // the same pairs, unchanged since the last upload: the device copy is current
    if (c->pairdev_d && c->pairdev_version == c->pairs_version && c->pairdev_ids.size() == n_pairs &&
        std::equal(pair_ids, pair_ids + n_pairs, c->pairdev_ids.begin()))
        return c->pairdev_d;
    c->pairdev_h.resize(n_pairs);
    for (uint32_t j = 0; j < n_pairs; ++j)
        c->pairdev_h[j] = make_pair_dev(get_pair(c, pair_ids[j]));
    c->pairdev_d = nullptr;
    PairDev *d = (PairDev *)scratch(c, "pairdev", n_pairs * sizeof(PairDev));
    // the source stays alive in the context until the next upload, which
    // follows a synchronisation (every call that uploads synchronises before it returns)
    AH_CUDA(cudaMemcpyAsync(d, c->pairdev_h.data(), n_pairs * sizeof(PairDev), cudaMemcpyHostToDevice, st));
    c->pairdev_ids.assign(pair_ids, pair_ids + n_pairs);
    c->pairdev_version = c->pairs_version;
    c->pairdev_d = d;
    return d;
}

// All pairs of the last upload have few_exact set.
bool tm_few_exact(const ah_ctx *c)
{
    for (const PairDev &d : c->pairdev_h)
        if (!d.few_exact)
            return false;
    return true;
}

// Largest Tm segment count (keys - 1) over the primers of the last upload.
int tm_seg_max(const ah_ctx *c)
{
    int m = 1;
    for (const PairDev &d : c->pairdev_h)
        m = std::max(m, std::max(d.nkey[0], d.nkey[1]) - 1);
    return m;
}

int bit_length(uint64_t v)
{
    int b = 0;
    while (v) {
        ++b;
        v >>= 1;
    }
    return b;
}

std::string signature(const std::vector<ScanPattern> &pats)
{
    std::string k;
    for (auto &p : pats) {
        k += std::to_string(p.L) + "," + std::to_string(p.k) + "," + std::to_string(p.clamp) + ",";
        for (int i = 0; i < p.L; ++i)
            k += (char)('a' + p.mask[i]);
        k += ";";
    }
    return k;
}

const ScanTuning &tuning_for(ah_ctx *c, const std::vector<ScanPattern> &pats)
{
    auto it = c->tuned.find(signature(pats));
    return it != c->tuned.end() ? it->second : c->tuning;
}

// Launch the generated scan kernel over tiles [0, n_tiles) of a set.
// Scan n_tiles tiles: the first n_tiles of the set, or tile_list[0 .. n_tiles) (device) when given.
// The caller resets the flag block (the work counter included) on the same stream first.
// work: the launch's slice counter (a flag word zeroed by the caller's reset_flags).
void launch_scan(ah_ctx *c, ScanKernel *k, const GenomeSet &gs, uint64_t n_tiles, uint64_t *keys, uint64_t cap,
                 int pbits, cudaStream_t st, const uint64_t *tile_list, uint64_t *work)
{
    const uint64_t grid = std::min<uint64_t>(n_tiles, (uint64_t)c->sms * k->blocks_per_sm);
    const uint32_t *planes = gs.planes;
    const uint64_t *coff = gs.contig_off;
    uint32_t nc = gs.n_contigs;
    const uint32_t *tcont = gs.tile_contig, *troom = gs.tile_room;
    uint64_t wait_ns = c->scan_stall_first ? 20000ull : 2000000000ull;
    int stall = c->scan_stall_first ? 1 : 0;
    void *args[] = {&planes, &n_tiles,  &coff, &nc,        &keys,  &cap,   &c->d_counter,
                    &pbits,  &c->d_err, &work, &tile_list, &tcont, &troom, &wait_ns, &stall};
    AH_CUDA(cudaLaunchKernel((const void *)k->fn, dim3((unsigned)grid), dim3(k->threads), args, k->smem, st));
}

// The scan patterns of the listed pairs (k_override >= 0: that k for every pair).
std::vector<ScanPattern> patterns_of(ah_ctx *c, const uint32_t *pair_ids, uint32_t n_pairs, int k_override = -1)
{
    std::vector<ScanPattern> pats;
    for (uint32_t j = 0; j < n_pairs; ++j) {
        const PrimerPair &pp = get_pair(c, pair_ids[j]);
        for (int primer = 0; primer < 2; ++primer)
            for (int strand = 0; strand < 2; ++strand) {
                ScanPattern p;
                p.L = pp.L[primer];
                p.k = k_override >= 0 ? k_override : pp.params.k;
                p.clamp = std::min(pp.params.clamp, p.L);
                p.pair = (int)j;
                p.primer = primer;
                p.strand = strand;
                for (int i = 0; i < p.L; ++i)
                    p.mask[i] = strand == 0 ? pp.mask[primer][i] : (uint8_t)comp_mask(pp.mask[primer][p.L - 1 - i]);
                pats.push_back(p);
            }
    }
    return pats;
}

// The patterns of each launch group (scan_launch_groups).
std::vector<std::vector<ScanPattern>> split_launches(const std::vector<ScanPattern> &pats)
{
    std::vector<std::vector<ScanPattern>> out;
    for (const auto &g : scan_launch_groups(pats))
        out.emplace_back(pats.begin() + g.first, pats.begin() + g.second);
    return out;
}

// Scan kernels over n_tiles tiles of a set (or tile_list), one launch per
// launch group, all appending to keys; returns the number of launches.  The
// caller resets the flag block (the groups' work counters included) first.
int launch_scans(ah_ctx *c, const GenomeSet &gs, const std::vector<ScanPattern> &pats, uint64_t n_tiles,
                 uint64_t *keys, uint64_t cap, int pbits, cudaStream_t st, const uint64_t *tile_list = nullptr)
{
    const auto parts = split_launches(pats);
    for (size_t i = 0; i < parts.size(); ++i) {
        ScanKernel *k = scan_kernel(parts[i], tuning_for(c, parts[i]), c->device);
        launch_scan(c, k, gs, n_tiles, keys, cap, pbits, st, tile_list, c->d_flags + kFlagWork + i);
    }
    return (int)parts.size();
}

} // namespace

namespace {

// ---- stages shared by ah_scan and ah_run ----

// Scan kernel over the whole set; keys land in the "scan_keys" scratch.
// Returns the number of sites (one synchronisation; rerun once with a
// larger key buffer if it overflowed).
// tile_list (device, n_list entries): scan only those tiles.
uint64_t scan_keys(ah_ctx *c, const GenomeSet &gs, const std::vector<ScanPattern> &pats, uint64_t **keys_out,
                   cudaStream_t st, const uint64_t *tile_list = nullptr, uint64_t n_list = 0)
{
    const int pbits = std::max(1, bit_length(gs.n_bases));
    uint64_t count = 0;
    *keys_out = nullptr;
    const uint64_t n_tiles = tile_list ? n_list : gs.n_tiles;
    if (!n_tiles)
        return 0;
    for (int attempt = 0; attempt < 2; ++attempt) {
        uint64_t *keys = (uint64_t *)scratch(c, "scan_keys", c->key_cap * sizeof(uint64_t));
        reset_flags(c, st);
        {
            Stage sg(c, "scan", st, (int)scan_launch_groups(pats).size());
            launch_scans(c, gs, pats, n_tiles, keys, c->key_cap, pbits, st, tile_list);
        }
        check_flags(c, st);
        count = c->h_flags[0];
        *keys_out = keys;
        if (count <= c->key_cap)
            break;
        c->key_cap = count;
    }
    return count;
}

// Sort keys into canonical order and decode them into site records.
void sort_decode(ah_ctx *c, const GenomeSet &gs, uint32_t n_pairs, const uint64_t *keys, uint64_t count, ah_site *dst,
                 cudaStream_t st)
{
    const int pbits = std::max(1, bit_length(gs.n_bases));
    const int end_bit = 10 + pbits + bit_length(n_pairs - 1);
    if (count <= kSmallSort) { // one launch: rank sort and decode
        Stage sg(c, "sort", st, 1);
        launch_rank_sort_decode(keys, count, nullptr, end_bit - 8 <= 32, pbits, gs.contig_off, gs.n_contigs,
                                gs.contig_genome, dst, nullptr, nullptr, st);
        return;
    }
    size_t tb = sort_keys_temp_bytes(count, end_bit);
    void *temp = scratch(c, "sort_temp", tb);
    uint64_t *sorted = (uint64_t *)scratch(c, "scan_keys_sorted", count * sizeof(uint64_t));
    {
        Stage sg(c, "sort", st, cub_sort_launches(count, end_bit - 8));
        sort_keys(temp, tb, keys, sorted, count, 8, end_bit, st);
    }
    {
        Stage sg(c, "decode", st, 1);
        launch_decode_keys(sorted, count, pbits, gs.contig_off, gs.n_contigs, gs.contig_genome, dst, st);
    }
}

// Buffer for an output of `count` records: the caller's own device buffer
// when it is on this device and large enough, else a scratch buffer.
template <class T> T *direct_or_scratch(ah_ctx *c, const char *name, T *user, uint64_t cap, uint64_t count)
{
    if (user && count <= cap && is_device_ptr(c, user))
        return user;
    return (T *)scratch(c, name, std::max<uint64_t>(count, 1) * sizeof(T));
}

// Copy a finished output to the caller's buffer when it was not written in place.
template <class T> bool deliver(T *user, uint64_t cap, const T *dev, uint64_t count, cudaStream_t st)
{
    if (count > cap)
        return false; // overflow: nothing written
    if (user && count && user != dev)
        AH_CUDA(cudaMemcpyAsync(user, dev, count * sizeof(T), cudaMemcpyDefault, st));
    return true;
}


// ---------------------------------------------------------------------------
// ah_run in two forms.
//
// One synchronisation (run_fast): every count stays on the device and every
// launch is sized for the largest count it accepts -- sites: kSmallSort, the
// key buffer and the caller's capacity; amplicons and sequence bytes: the
// caller's device buffers, else scratch sized from earlier runs.  A count above
// its launch size sets a kRedo* bit and the later kernels see zero records; the
// host then finishes with the step-by-step form (run_steps), which reuses the
// scan's keys when they all fit.  Step by step (run_steps): one
// synchronisation per data-dependent size, any size.
// ---------------------------------------------------------------------------
enum FastResult { kFastDone, kFastKeys, kFastRescan };

// Queue the one-synchronisation form; scan_done (optional) is recorded right
// after the scan.  The flag block is copied to the host after the last kernel.
void fast_begin(ah_ctx *c, const GenomeSet &gs, const std::vector<ScanPattern> &pats, const PairDev *pd,
                uint32_t n_pairs, ah_run_out *o, cudaStream_t st, cudaEvent_t scan_done, ah_ctx::FastRun *fr)
{
    std::unique_ptr<HostSpan> span(new HostSpan(c, "host.run.prep"));
    uint64_t *F = c->d_flags;
    const int pbits = std::max(1, bit_length(gs.n_bases));
    const int end_bit = 10 + pbits + bit_length(n_pairs - 1);
    // where each output is written: the caller's device buffer, else scratch
    const bool sites_direct = o->sites_cap && is_device_ptr(c, o->sites) && (!o->tm || is_device_ptr(c, o->tm)) &&
                              (!o->pass || is_device_ptr(c, o->pass));
    uint64_t ns_max = std::min<uint64_t>(kSmallSort, c->key_cap);
    if (sites_direct)
        ns_max = std::min<uint64_t>(ns_max, o->sites_cap);
    const bool amps_direct = o->amplicons_cap && is_device_ptr(c, o->amplicons) &&
                             (!o->seq_offsets || is_device_ptr(c, o->seq_offsets));
    const uint64_t na_max = std::min<uint64_t>(amps_direct ? o->amplicons_cap : c->fast_amps, kSmallScan - 1);
    const bool seq_direct = o->seq_cap && is_device_ptr(c, o->seq);
    const uint64_t nq_max = seq_direct ? o->seq_cap : c->fast_seq;

    uint64_t *keys = (uint64_t *)scratch(c, "scan_keys", c->key_cap * sizeof(uint64_t));
    ah_site *sites = sites_direct ? o->sites : (ah_site *)scratch(c, "run_sites", ns_max * sizeof(ah_site));
    float *tm = sites_direct && o->tm ? o->tm : (float *)scratch(c, "run_tm", ns_max * sizeof(float));
    uint8_t *pass = sites_direct && o->pass ? o->pass : (uint8_t *)scratch(c, "run_pass", ns_max);
    uint32_t *queue = (uint32_t *)scratch(c, "tm_queue", 2 * ns_max * sizeof(uint32_t));
    uint64_t *counts = (uint64_t *)scratch(c, "pair_counts", ns_max * sizeof(uint64_t));
    uint64_t *offs = (uint64_t *)scratch(c, "pair_offsets", ns_max * sizeof(uint64_t));
    ah_amplicon *amps = amps_direct ? o->amplicons : (ah_amplicon *)scratch(c, "run_amps", na_max * sizeof(ah_amplicon));
    uint64_t *qoff = amps_direct && o->seq_offsets ? o->seq_offsets
                                                   : (uint64_t *)scratch(c, "run_qoff", (na_max + 1) * sizeof(uint64_t));
    uint64_t *len = (uint64_t *)scratch(c, "fetch_len", (na_max + 1) * sizeof(uint64_t));
    char *seq = seq_direct ? o->seq : (char *)scratch(c, "run_seq", nq_max);
    const uint8_t *filt = o->tm_filter ? pass : nullptr;

    const int n_launch = (int)scan_launch_groups(pats).size();
    span.reset(new HostSpan(c, "host.run.launch"));
    reset_flags(c, st);
    {
        Stage sg(c, "scan", st, n_launch);
        launch_scans(c, gs, pats, gs.n_tiles, keys, c->key_cap, pbits, st);
    }
    if (scan_done)
        AH_CUDA(cudaEventRecord(scan_done, st));
    {
        Stage sg(c, "sort", st, 1);
        launch_rank_sort_decode(keys, ns_max, F + kFlagCounter, end_bit - 8 <= 32, pbits, gs.contig_off,
                                gs.n_contigs, gs.contig_genome, sites, F + kFlagSites, F + kFlagRedo, st);
    }
    {
        Stage sg(c, "tm", st, 2);
        launch_tm(sites, ns_max, F + kFlagSites, pd, (int)n_pairs, gs.planes, gs.contig_off, tm, pass, queue,
                  (uint32_t *)(F + kFlagTmQueue), tm_seg_max(c), tm_few_exact(c), c->d_err, st);
    }
    {
        Stage sg(c, "pair", st, 3);
        launch_pair_count(sites, ns_max, F + kFlagSites, filt, pd, counts, st);
        exclusive_scan_u64_dev(counts, offs, ns_max, F + kFlagSites, 0, F + kFlagAux, na_max, F + kFlagAmps,
                               F + kFlagRedo, kRedoAmps, st);
        launch_pair_write(sites, ns_max, F + kFlagSites, filt, pd, offs, amps, na_max, F + kFlagRedo, kRedoAmps, st);
    }
    {
        Stage sg(c, "fetch", st, 3);
        launch_fetch_lengths(amps, na_max, F + kFlagAmps, gs.contig_off, gs.n_contigs, len, c->d_err, st);
        exclusive_scan_u64_dev(len, qoff, na_max + 1, F + kFlagAmps, 1, F + kFlagAux, nq_max, F + kFlagSeq,
                               F + kFlagRedo, kRedoSeq, st);
        launch_fetch(amps, na_max, F + kFlagAmps, qoff, gs.planes, gs.contig_off, seq, F + kFlagRedo, kRedoSeq, st);
    }
    AH_CUDA(cudaMemcpyAsync(c->h_flags, c->d_flags, kFlagWords * sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    AH_CUDA(cudaEventRecord(c->ev_run, st));
    *fr = {sites_direct, amps_direct, seq_direct, keys, sites, tm, pass, amps, qoff, seq};
}

// Wait for a queued one-synchronisation run and complete `o`, or report that
// a count went above the launch sizes (kFastKeys: the keys are complete).
FastResult fast_end(ah_ctx *c, ah_run_out *o, cudaStream_t st, const ah_ctx::FastRun &fr, uint64_t **keys_out,
                    uint64_t *ns_out)
{
    {
        HostSpan span(c, "host.run.wait");
        AH_CUDA(cudaEventSynchronize(c->ev_run)); // the one synchronisation
    }
    c->flags_dirty = false;
    const uint64_t *H = c->h_flags;
    const int e = (int)(H[kFlagErr] & 0xffffffffu);
    if (e != 0) {
        AH_CUDA(cudaMemsetAsync(c->d_flags + kFlagErr, 0, sizeof(uint64_t), st));
        raise_device_error(e);
    }
    const uint64_t ns = H[kFlagCounter];
    *keys_out = fr.keys;
    *ns_out = ns;
    c->last_sites = ns;
    if (H[kFlagRedo])
        return ns <= c->key_cap ? kFastKeys : kFastRescan;
    const uint64_t na = H[kFlagAmps], nq = H[kFlagSeq];
    o->n_sites = ns;
    o->n_amplicons = na;
    o->n_seq = nq;
    bool overflow = !deliver(o->sites, o->sites_cap, fr.sites, ns, st);
    if (o->tm)
        overflow |= !deliver(o->tm, o->sites_cap, fr.tm, ns, st);
    if (o->pass)
        overflow |= !deliver(o->pass, o->sites_cap, fr.pass, ns, st);
    overflow |= !deliver(o->amplicons, o->amplicons_cap, fr.amps, na, st);
    if (o->seq_offsets)
        overflow |= !deliver(o->seq_offsets, o->amplicons_cap + 1, fr.qoff, na + 1, st);
    overflow |= !deliver(o->seq, o->seq_cap, fr.seq, nq, st);
    if (!(fr.sites_direct && fr.amps_direct && fr.seq_direct)) // copies to host memory land before the call returns
        AH_CUDA(cudaStreamSynchronize(st));
    if (overflow)
        throw Error(AH_ERR_OVERFLOW, "ah_run: an output buffer is too small (counts are in the out struct)");
    return kFastDone;
}

// Calls that touch the context's scratch, pair uploads or flag block wait for
// no queued run: they return an error while one is pending.
void require_idle(ah_ctx *c)
{
    require(!c->pend.active, AH_ERR_ARG, "a run is pending: complete it with ah_run_end first");
    require(!c->serving, AH_ERR_ARG, "a server owns the context: stop it first");
}

// A run's work goes on the run stream, after the caller's earlier work; the
// caller's stream then waits for everything the run queued.
cudaStream_t enter_run_stream(ah_ctx *c, cudaStream_t caller)
{
    AH_CUDA(cudaEventRecord(c->ev_in, caller));
    AH_CUDA(cudaStreamWaitEvent(c->run_stream, c->ev_in, 0));
    return c->run_stream;
}

void leave_run_stream(ah_ctx *c, cudaStream_t caller)
{
    AH_CUDA(cudaEventRecord(c->ev_out, c->run_stream));
    AH_CUDA(cudaStreamWaitEvent(caller, c->ev_out, 0));
}

void run_steps(ah_ctx *c, const GenomeSet &gs, const PairDev *pd, uint32_t n_pairs, uint64_t *keys, uint64_t ns,
               ah_run_out *o, cudaStream_t st)
{
    bool overflow = false;
    o->n_sites = ns;
    c->last_sites = ns;
    ah_site *sites = direct_or_scratch(c, "run_sites", o->sites, o->sites_cap, ns);
    float *tm = direct_or_scratch(c, "run_tm", o->tm, o->tm ? o->sites_cap : 0, ns);
    uint8_t *pass = direct_or_scratch(c, "run_pass", o->pass, o->pass ? o->sites_cap : 0, ns);
    uint64_t na = 0, nq = 0;
    ah_amplicon *amps = nullptr;
    uint64_t *qoff = nullptr;
    char *seq = nullptr;
    if (ns) {
        // canonical sites, Tm, pair counts (synchronisation: the amplicon count)
        sort_decode(c, gs, n_pairs, keys, ns, sites, st);
        {
            Stage sg(c, "tm", st, 2);
            uint32_t *q = (uint32_t *)scratch(c, "tm_queue", 2 * ns * sizeof(uint32_t));
            launch_tm(sites, ns, nullptr, pd, (int)n_pairs, gs.planes, gs.contig_off, tm, pass, q,
                      (uint32_t *)(c->d_flags + kFlagTmQueue), tm_seg_max(c), tm_few_exact(c), c->d_err, st);
        }
        const uint8_t *filt = o->tm_filter ? pass : nullptr;
        uint64_t *counts = (uint64_t *)scratch(c, "pair_counts", ns * sizeof(uint64_t));
        uint64_t *offs = (uint64_t *)scratch(c, "pair_offsets", ns * sizeof(uint64_t));
        size_t tb = scan_u64_temp_bytes(ns);
        void *temp = scratch(c, "scan_temp", tb);
        {
            Stage sg(c, "pair", st, 2 + scan_u64_launches(ns));
            launch_pair_count(sites, ns, nullptr, filt, pd, counts, st);
            exclusive_scan_u64(temp, tb, counts, offs, ns, st);
            launch_total(offs, counts, ns, nullptr, 0, c->d_aux, 0, nullptr, nullptr, 0, st);
        }
        check_flags(c, st);
        na = c->h_flags[kFlagAux];
        o->n_amplicons = na;
        // amplicons and sequence offsets (synchronisation: the sequence bytes)
        amps = direct_or_scratch(c, "run_amps", o->amplicons, o->amplicons_cap, na);
        qoff = direct_or_scratch(c, "run_qoff", o->seq_offsets, o->seq_offsets ? o->amplicons_cap + 1 : 0, na + 1);
        if (na) {
            Stage sg(c, "pair", st, 1);
            launch_pair_write(sites, ns, nullptr, filt, pd, offs, amps, na, nullptr, 0, st);
        }
        uint64_t *len = (uint64_t *)scratch(c, "fetch_len", (na + 1) * sizeof(uint64_t));
        size_t tb2 = scan_u64_temp_bytes(na + 1);
        void *temp2 = scratch(c, "scan_temp", tb2);
        {
            Stage sg(c, "fetch", st, (na ? 1 : 0) + scan_u64_launches(na + 1));
            AH_CUDA(cudaMemsetAsync(len + na, 0, sizeof(uint64_t), st));
            launch_fetch_lengths(amps, na, nullptr, gs.contig_off, gs.n_contigs, len, c->d_err, st);
            exclusive_scan_u64(temp2, tb2, len, qoff, na + 1, st);
            AH_CUDA(cudaMemcpyAsync(c->d_aux, qoff + na, sizeof(uint64_t), cudaMemcpyDeviceToDevice, st));
        }
        check_flags(c, st);
        nq = c->h_flags[kFlagAux];
        o->n_seq = nq;
        // sequences, then every output that was not written in place
        seq = direct_or_scratch(c, "run_seq", o->seq, o->seq_cap, nq);
        if (na && nq) {
            Stage sg(c, "fetch", st, 1);
            launch_fetch(amps, na, nullptr, qoff, gs.planes, gs.contig_off, seq, nullptr, 0, st);
        }
    }
    // later one-synchronisation runs size their scratch for counts like these
    c->fast_amps = std::min<uint64_t>(kSmallScan - 1, std::max<uint64_t>(c->fast_amps, na + na / 4 + 16));
    c->fast_seq = std::min<uint64_t>(1ull << 30, std::max<uint64_t>(c->fast_seq, nq + nq / 4 + 4096));
    overflow |= !deliver(o->sites, o->sites_cap, sites, ns, st);
    if (o->tm)
        overflow |= !deliver(o->tm, o->sites_cap, tm, ns, st);
    if (o->pass)
        overflow |= !deliver(o->pass, o->sites_cap, pass, ns, st);
    overflow |= !deliver(o->amplicons, o->amplicons_cap, amps, na, st);
    if (o->seq_offsets) {
        if (ns)
            overflow |= !deliver(o->seq_offsets, o->amplicons_cap + 1, qoff, na + 1, st);
        else if (is_device_ptr(c, o->seq_offsets))
            AH_CUDA(cudaMemsetAsync(o->seq_offsets, 0, sizeof(uint64_t), st));
        else
            o->seq_offsets[0] = 0;
    }
    overflow |= !deliver(o->seq, o->seq_cap, seq, nq, st);
    check_flags(c, st);
    if (overflow)
        throw Error(AH_ERR_OVERFLOW, "ah_run: an output buffer is too small (counts are in the out struct)");
}


// ---------------------------------------------------------------------------
// Serving (continuous batching over one resident genome set).
//
// A worker thread owns the context while the server runs.  Requests wait in a
// FIFO queue; each time the GPU is free the worker admits the queued requests
// whose estimated device memory fits the budget (at least one), and runs them
// as one batch: per (primer pair, k), one scan over the union of the
// requests' genomes' tiles, then sort, Tm and all-pairs amplicon calling on
// those sites.  A request's result is then taken out exactly: the sites of its
// genomes and the amplicons between them (both ends passing under its Tm
// filter).  A site and an amplicon depend only on their own windows, so a
// request's result does not depend on what it was batched with.
// ---------------------------------------------------------------------------
struct ServeReq {
    std::vector<uint32_t> genomes;
    uint32_t pair_id = 0;
    int k = 0, tm_filter = 0;
    double t_submit = 0, t_start = 0, t_done = 0;
    bool done = false;
    ah_status status = AH_OK;
    std::string msg;
    uint32_t batch = 0, batch_size = 0;
    uint64_t n_sites = 0, bases = 0;
    std::vector<ah_site> sites;
    std::vector<ah_amplicon> amps;
    std::vector<char> seq;          // amplicon sequences, concatenated
    std::vector<uint64_t> seq_off;  // n_amplicons + 1 offsets into seq
};

} // namespace

struct ah_server {
    ah_ctx *c = nullptr;
    uint32_t set_id = 0;
    ah_serve_config cfg{};
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::map<uint64_t, ServeReq> reqs;
    std::deque<uint64_t> queue;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
    std::vector<uint64_t> genome_bases; // bases per genome id
    // contigs of each genome id (CSR): genome_contig[genome_first[g] .. genome_first[g + 1])
    std::vector<uint64_t> genome_first;
    std::vector<uint32_t> genome_contig;
    // pinned staging of a group's device results (several, so that the host
    // filtering of a group overlaps the next groups' device work)
    static constexpr int kStaging = 6;
    struct Staging {
        void *p = nullptr;
        size_t bytes = 0;
    } staging[kStaging];
    ~ah_server()
    {
        for (auto &st : staging)
            if (st.p)
                cudaFreeHost(st.p);
    }
    double now_ms() const
    {
        return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

// device bytes a request's share of a batch may need (sites and amplicons grow with bases)
size_t serve_request_bytes(const ServeReq &r) { return 4096 + (size_t)(r.bases / 1000) * 64; }

// Device results of one group of requests (one primer pair and one k), in
// pinned host memory.
struct GroupData {
    const ah_site *sites = nullptr;
    const uint8_t *pass = nullptr;
    const ah_amplicon *amps = nullptr;
    uint64_t ns = 0, na = 0;
};

void *staging_at_least(ah_server::Staging &st, size_t bytes)
{
    if (st.bytes < bytes) {
        if (st.p)
            AH_CUDA(cudaFreeHost(st.p));
        st.p = nullptr;
        st.bytes = 0;
        const size_t want = std::max<size_t>(bytes + bytes / 4, 1 << 20);
        AH_CUDA(cudaMallocHost(&st.p, want));
        st.bytes = want;
    }
    return st.p;
}

// Scan of the union of the group's genomes, then sort, Tm and amplicon calling
// without a Tm filter; results to the host staging buffer.
// Tiles holding a start of a contig of the union of the requests' genomes:
// each contig's tile range, ranges sorted and merged, then listed.  Host work
// only (thread-safe: reads the set's host tables).
std::vector<uint64_t> group_tiles(const GenomeSet &gs, const ah_server *S, const std::vector<ServeReq *> &rs)
{
    std::vector<uint32_t> gen;
    for (ServeReq *r : rs)
        gen.insert(gen.end(), r->genomes.begin(), r->genomes.end());
    std::sort(gen.begin(), gen.end());
    gen.erase(std::unique(gen.begin(), gen.end()), gen.end());
    std::vector<std::pair<uint64_t, uint64_t>> ranges; // [first, last] tile of a contig
    for (uint32_t g : gen) {
        if (g + 1 >= S->genome_first.size())
            continue;
        for (uint64_t q = S->genome_first[g]; q < S->genome_first[g + 1]; ++q) {
            const uint32_t ci = S->genome_contig[q];
            const uint64_t a = gs.contig_off_h[ci], b = gs.contig_off_h[ci + 1];
            if (b > a)
                ranges.push_back({a / kTileBases, (b - 1) / kTileBases});
        }
    }
    std::sort(ranges.begin(), ranges.end());
    std::vector<uint64_t> tiles;
    uint64_t next = 0; // first tile not yet listed
    for (const auto &rg : ranges) { // sorted by first tile: the list comes out sorted and unique
        for (uint64_t t = std::max(rg.first, next); t <= rg.second; ++t)
            tiles.push_back(t);
        next = std::max(next, rg.second + 1);
    }
    return tiles;
}

// Scan of the group's tiles at the group's k, then sort, Tm and amplicon
// calling without a Tm filter; results to the host staging buffer.
void group_device(ah_ctx *c, const GenomeSet &gs, uint32_t pid, int k, const std::vector<uint64_t> &tiles,
                  ah_server::Staging &stage, GroupData &d)
{
    cudaStream_t st = c->stream;
    HostSpan span(c, "host.serve.device");
    if (tiles.empty())
        return;
    uint64_t *tl = (uint64_t *)scratch(c, "serve_tiles", tiles.size() * sizeof(uint64_t));
    AH_CUDA(cudaMemcpyAsync(tl, tiles.data(), tiles.size() * sizeof(uint64_t), cudaMemcpyHostToDevice, st));
    std::vector<ScanPattern> pats = patterns_of(c, &pid, 1, k);
    const PairDev *pd = upload_pairs(c, &pid, 1, st);
    uint64_t *keys = nullptr;
    const uint64_t ns = scan_keys(c, gs, pats, &keys, st, tl, tiles.size());
    if (!ns)
        return;
    ah_site *sites = (ah_site *)scratch(c, "serve_sites", ns * sizeof(ah_site));
    sort_decode(c, gs, 1, keys, ns, sites, st);
    float *tm = (float *)scratch(c, "serve_tm", ns * sizeof(float));
    uint8_t *pass = (uint8_t *)scratch(c, "serve_pass", ns);
    uint32_t *q = (uint32_t *)scratch(c, "tm_queue", 2 * ns * sizeof(uint32_t));
    {
        Stage sg(c, "tm", st, 2);
        launch_tm(sites, ns, nullptr, pd, 1, gs.planes, gs.contig_off, tm, pass, q,
                  (uint32_t *)(c->d_flags + kFlagTmQueue), tm_seg_max(c), tm_few_exact(c), c->d_err, st);
    }
    uint64_t *counts = (uint64_t *)scratch(c, "pair_counts", ns * sizeof(uint64_t));
    uint64_t *offs = (uint64_t *)scratch(c, "pair_offsets", ns * sizeof(uint64_t));
    size_t tb = scan_u64_temp_bytes(ns);
    void *temp = scratch(c, "scan_temp", tb);
    {
        Stage sg(c, "pair", st, 2 + scan_u64_launches(ns));
        launch_pair_count(sites, ns, nullptr, nullptr, pd, counts, st);
        exclusive_scan_u64(temp, tb, counts, offs, ns, st);
        launch_total(offs, counts, ns, nullptr, 0, c->d_aux, 0, nullptr, nullptr, 0, st);
    }
    check_flags(c, st);
    const uint64_t na = c->h_flags[kFlagAux];
    ah_amplicon *amps = (ah_amplicon *)scratch(c, "serve_amps", std::max<uint64_t>(na, 1) * sizeof(ah_amplicon));
    if (na) {
        Stage sg(c, "pair", st, 1);
        launch_pair_write(sites, ns, nullptr, nullptr, pd, offs, amps, na, nullptr, 0, st);
    }
    // staging layout: sites, amplicons, pass flags
    const size_t sb = ns * sizeof(ah_site), ab = na * sizeof(ah_amplicon);
    char *h = (char *)staging_at_least(stage, sb + ab + ns);
    AH_CUDA(cudaMemcpyAsync(h, sites, sb, cudaMemcpyDeviceToHost, st));
    if (na)
        AH_CUDA(cudaMemcpyAsync(h + sb, amps, ab, cudaMemcpyDeviceToHost, st));
    AH_CUDA(cudaMemcpyAsync(h + sb + ab, pass, ns, cudaMemcpyDeviceToHost, st));
    check_flags(c, st);
    d.sites = (const ah_site *)h;
    d.amps = (const ah_amplicon *)(h + sb);
    d.pass = (const uint8_t *)(h + sb + ab);
    d.ns = ns;
    d.na = na;
}

// Per request: the group's sites of its genomes (all have mm <= the group's
// k), and the amplicons whose two ends are among them (both passing under the
// Tm filter).  Sites of other genomes are few (they share an edge tile with a
// requested genome), so the kept sites are copied in runs between the dropped
// ones and an index is re-mapped by counting the dropped ones below it.  The
// group's canonical order is kept.  Host work only (runs beside the next
// group's device work).
void group_filter(uint64_t G, const GroupData &d, const std::vector<ServeReq *> &rs)
{
    std::vector<char> mine(G, 0);
    std::vector<uint64_t> dropped;
    for (ServeReq *r : rs) {
        for (uint32_t g : r->genomes)
            if (g < G)
                mine[g] = 1;
        dropped.clear();
        for (uint64_t i = 0; i < d.ns; ++i)
            if (!mine[d.sites[i].genome])
                dropped.push_back(i);
        r->sites.clear();
        r->sites.reserve(d.ns - dropped.size());
        uint64_t from = 0;
        for (size_t j = 0; j <= dropped.size(); ++j) {
            const uint64_t end = j < dropped.size() ? dropped[j] : d.ns;
            if (end > from)
                r->sites.insert(r->sites.end(), d.sites + from, d.sites + end);
            from = end + 1;
        }
        r->n_sites = r->sites.size();
        auto remap = [&](uint64_t i) -> int64_t { // -1: dropped
            const auto it = std::lower_bound(dropped.begin(), dropped.end(), i);
            if (it != dropped.end() && *it == i)
                return -1;
            return (int64_t)(i - (uint64_t)(it - dropped.begin()));
        };
        r->amps.clear();
        for (uint64_t i = 0; i < d.na; ++i) {
            const ah_amplicon &x = d.amps[i];
            if (!mine[x.genome])
                continue;
            if (r->tm_filter && !(d.pass[x.left] && d.pass[x.right]))
                continue;
            const int64_t l = remap(x.left), rr = remap(x.right);
            if (l < 0 || rr < 0)
                continue;
            ah_amplicon b = x;
            b.left = (uint32_t)l; // indices into the request's own site list
            b.right = (uint32_t)rr;
            r->amps.push_back(b);
        }
        for (uint32_t g : r->genomes)
            if (g < G)
                mine[g] = 0;
    }
}

// One batch: fills every request's result fields.  Requests are grouped by
// (primer pair, k); groups run one after another on the device, each group's
// host filtering overlaps the next group's device work, and one fetch at the
// end decodes every distinct amplicon some request keeps.
void serve_batch(ah_server *S, std::vector<ServeReq *> &batch)
{
    ah_ctx *c = S->c;
    GenomeSet &gs = get_set(c, S->set_id);
    cudaStream_t st = c->stream;
    std::map<std::pair<uint32_t, int>, std::vector<ServeReq *>> groups;
    for (ServeReq *r : batch)
        groups[{r->pair_id, r->k}].push_back(r);
    const uint64_t G = (uint64_t)gs.max_genome + 1;
    std::deque<GroupData> data;
    std::vector<std::future<void>> filters;
    // every group's tile list is built on the host cores while the device works
    std::vector<std::future<std::vector<uint64_t>>> plans;
    for (auto &kv : groups) {
        const std::vector<ServeReq *> *rs = &kv.second;
        const GenomeSet *g = &gs;
        plans.push_back(std::async(std::launch::async, [g, S, rs] { return group_tiles(*g, S, *rs); }));
    }
    try {
        size_t gi = 0;
        for (auto &kv : groups) {
            if (gi >= ah_server::kStaging) { // the staging buffer is reused: its earlier group is filtered first
                HostSpan hs(c, "host.serve.filter_wait");
                filters[gi - ah_server::kStaging].get();
            }
            data.emplace_back();
            std::vector<uint64_t> tiles;
            {
                HostSpan hs(c, "host.serve.tiles");
                tiles = plans[gi].get();
            }
            group_device(c, gs, kv.first.first, kv.first.second, tiles, S->staging[gi % ah_server::kStaging],
                         data.back());
            const GroupData *d = &data.back();
            const std::vector<ServeReq *> *rs = &kv.second;
            filters.push_back(std::async(std::launch::async, [G, d, rs] { group_filter(G, *d, *rs); }));
            ++gi;
        }
    } catch (...) {
        for (auto &f : filters)
            if (f.valid())
                f.wait();
        for (auto &f : plans)
            if (f.valid())
                f.wait();
        throw;
    }
    {
        HostSpan hs(c, "host.serve.filter_wait");
        for (auto &f : filters)
            if (f.valid())
                f.get();
    }
    HostSpan hs_fetch(c, "host.serve.fetch");
    // distinct amplicons of the batch (a sequence depends on contig, start, end, orient)
    struct Ref {
        uint64_t k0, k1;
        ServeReq *r;
        uint32_t j;
    };
    std::vector<Ref> refs;
    for (ServeReq *r : batch)
        for (uint32_t j = 0; j < r->amps.size(); ++j) {
            const ah_amplicon &x = r->amps[j];
            refs.push_back({(uint64_t)x.contig << 32 | x.start, (uint64_t)x.end << 8 | x.orient, r, j});
        }
    std::sort(refs.begin(), refs.end(),
              [](const Ref &a, const Ref &b) { return a.k0 != b.k0 ? a.k0 < b.k0 : a.k1 < b.k1; });
    std::vector<ah_amplicon> recs;
    std::vector<uint64_t> slot(refs.size());
    for (size_t i = 0; i < refs.size(); ++i) {
        if (i == 0 || refs[i].k0 != refs[i - 1].k0 || refs[i].k1 != refs[i - 1].k1)
            recs.push_back(refs[i].r->amps[refs[i].j]);
        slot[i] = recs.size() - 1;
    }
    const uint64_t nf = recs.size();
    std::vector<uint64_t> f_off(nf + 1, 0);
    for (uint64_t j = 0; j < nf; ++j)
        f_off[j + 1] = f_off[j] + (recs[j].end - recs[j].start);
    // sequences through the first staging buffer (every filter is done with it)
    char *seq_h = (char *)staging_at_least(S->staging[0], std::max<uint64_t>(f_off.back(), 1));
    if (nf) {
        ah_amplicon *ra = (ah_amplicon *)scratch(c, "serve_fetch_amps", nf * sizeof(ah_amplicon));
        uint64_t *ro = (uint64_t *)scratch(c, "serve_fetch_offs", (nf + 1) * sizeof(uint64_t));
        char *rq = (char *)scratch(c, "serve_fetch_seq", std::max<uint64_t>(f_off.back(), 1));
        AH_CUDA(cudaMemcpyAsync(ra, recs.data(), nf * sizeof(ah_amplicon), cudaMemcpyHostToDevice, st));
        AH_CUDA(cudaMemcpyAsync(ro, f_off.data(), (nf + 1) * sizeof(uint64_t), cudaMemcpyHostToDevice, st));
        {
            Stage sg(c, "fetch", st, 1);
            launch_fetch(ra, nf, nullptr, ro, gs.planes, gs.contig_off, rq, nullptr, 0, st);
        }
        if (f_off.back())
            AH_CUDA(cudaMemcpyAsync(seq_h, rq, f_off.back(), cudaMemcpyDeviceToHost, st));
        check_flags(c, st);
    }
    // per request, sequences in the order of its amplicons
    std::map<ServeReq *, std::vector<uint64_t>> per;
    for (ServeReq *r : batch)
        per[r].assign(r->amps.size(), 0);
    for (size_t i = 0; i < refs.size(); ++i)
        per[refs[i].r][refs[i].j] = slot[i];
    for (ServeReq *r : batch) {
        r->seq_off.assign(1, 0);
        r->seq.clear();
        for (uint64_t j : per[r]) {
            r->seq.insert(r->seq.end(), seq_h + f_off[j], seq_h + f_off[j + 1]);
            r->seq_off.push_back(r->seq.size());
        }
    }
}

void serve_loop(ah_server *S)
{
    cudaSetDevice(S->c->device);
    uint32_t batch_no = 0;
    for (;;) {
        std::vector<uint64_t> tickets;
        std::vector<ServeReq> work;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait(lk, [&] { return S->stop || !S->queue.empty(); });
            if (S->queue.empty())
                return; // stopped with nothing pending
            size_t mem = 0;
            const double t = S->now_ms();
            while (!S->queue.empty() && tickets.size() < S->cfg.max_batch) {
                ServeReq &r = S->reqs[S->queue.front()];
                const size_t need = serve_request_bytes(r);
                if (!tickets.empty() && mem + need > S->cfg.mem_budget)
                    break; // admitted later, when the running work has left
                mem += need;
                r.t_start = t;
                tickets.push_back(S->queue.front());
                work.push_back(r); // a copy: the map may grow while the batch runs
                S->queue.pop_front();
            }
        }
        ++batch_no;
        std::vector<ServeReq *> ptrs;
        for (ServeReq &r : work)
            ptrs.push_back(&r);
        ah_status status = AH_OK;
        std::string msg;
        try {
            HostSpan hs(S->c, "host.serve.batch");
            serve_batch(S, ptrs);
        } catch (const Error &e) {
            status = e.status;
            msg = e.msg;
        } catch (const std::exception &e) {
            status = AH_ERR_ARG;
            msg = e.what();
        }
        {
            std::lock_guard<std::mutex> lk(S->mu);
            const double t = S->now_ms();
            for (size_t i = 0; i < tickets.size(); ++i) {
                ServeReq &r = S->reqs[tickets[i]];
                r.amps = std::move(work[i].amps);
                r.sites = std::move(work[i].sites);
                r.seq = std::move(work[i].seq);
                r.seq_off = std::move(work[i].seq_off);
                r.n_sites = work[i].n_sites;
                r.batch_size = (uint32_t)tickets.size();
                r.status = status;
                r.msg = msg;
                r.batch = batch_no;
                r.t_done = t;
                r.done = true;
            }
        }
        S->cv_done.notify_all();
    }
}
} // namespace

// ===========================================================================
extern "C" {

ah_status ah_create(int device, size_t mem_budget_bytes, ah_ctx **out)
{
    std::lock_guard<std::mutex> lock(g_create_mu);
    if (!out) {
        g_create_err = "ah_create: out is null";
        return AH_ERR_ARG;
    }
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        g_create_err = "ah_create: no such CUDA device";
        return AH_ERR_ARG;
    }
    ah_ctx *c = new (std::nothrow) ah_ctx;
    if (!c) {
        g_create_err = "ah_create: host allocation failed";
        return AH_ERR_OOM;
    }
    c->device = device;
    c->budget = mem_budget_bytes;
    ah_status st = guarded(c, [&] {
        AH_CUDA(cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device));
        // default scan variant; AH_SCAN_TUNING="R,arith_pct,order,stages,warps[,min_blocks[,resident]]" overrides
        // it (profiling aid)
        if (const char *e = getenv("AH_SCAN_TUNING")) {
            int R = 8, ap = 0, order = 1, S = 3, wpc = 4, mb = 1, res = 0;
            if (sscanf(e, "%d,%d,%d,%d,%d,%d,%d", &R, &ap, &order, &S, &wpc, &mb, &res) >= 1 && (R == 4 || R == 8) &&
                ap >= 0 && ap <= 100 && (order == 0 || order == 1) && S >= 2 && S <= 4 && wpc >= 1 && wpc <= 16 &&
                mb >= 1 && mb <= 8 && res >= 0 && res <= 8) {
                c->tuning.resident = res;
                c->tuning.R = R;
                c->tuning.arith_pct = ap;
                c->tuning.order = order;
                c->tuning.stages = S;
                c->tuning.warps = wpc;
                c->tuning.min_blocks = mb;
            }
        }
        AH_CUDA(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
        c->d_flags = (uint64_t *)dev_alloc(c, kFlagWords * sizeof(uint64_t));
        c->d_counter = c->d_flags + kFlagCounter;
        c->d_aux = c->d_flags + kFlagAux;
        c->d_err = (int *)(c->d_flags + kFlagErr);
        AH_CUDA(cudaMemsetAsync(c->d_flags, 0, kFlagWords * sizeof(uint64_t), c->stream));
        AH_CUDA(cudaStreamSynchronize(c->stream));
        AH_CUDA(cudaMallocHost(&c->h_flags, kFlagWords * sizeof(uint64_t)));
        AH_CUDA(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
        {
            int least = 0, greatest = 0;
            AH_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
            AH_CUDA(cudaStreamCreateWithPriority(&c->run_stream, cudaStreamNonBlocking, greatest));
        }
        AH_CUDA(cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming));
        AH_CUDA(cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming));
        for (auto &sl : c->pin)
            AH_CUDA(cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming));
        AH_CUDA(cudaEventCreateWithFlags(&c->ev_run, cudaEventDisableTiming));
        for (int b = 0; b < 2; ++b) {
            AH_CUDA(cudaEventCreateWithFlags(&c->ev_copied[b], cudaEventDisableTiming));
            AH_CUDA(cudaEventCreateWithFlags(&c->ev_packed[b], cudaEventDisableTiming));
        }
        AH_CUDA(cudaEventCreateWithFlags(&c->ev_load_start, cudaEventDisableTiming));
        AH_CUDA(cudaEventCreateWithFlags(&c->ev_last_copy, cudaEventDisableTiming));
    });
    if (st != AH_OK) {
        g_create_err = c->err;
        ah_destroy(c);
        return st;
    }
    *out = c;
    return AH_OK;
}

void ah_destroy(ah_ctx *c)
{
    if (!c)
        return;
    cudaSetDevice(c->device);
    if (c->pend.active && !c->pend.done)
        cudaEventSynchronize(c->ev_run); // a queued run still uses the context's memory
    if (c->stream)
        cudaStreamSynchronize(c->stream);
    // host loads queued without waiting (AH_LOAD_HOST_ASYNC) may still copy into the staging buffers
    if (c->copy_stream)
        cudaStreamSynchronize(c->copy_stream);
    if (c->run_stream)
        cudaStreamSynchronize(c->run_stream);
    for (auto &kv : c->live)
        cudaFree(kv.first);
    for (auto &p : c->pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    for (auto e : c->events)
        cudaEventDestroy(e);
    if (c->h_flags)
        cudaFreeHost(c->h_flags);
    for (auto &sl : c->pin) {
        if (sl.ev)
            cudaEventSynchronize(sl.ev);
        if (sl.p)
            cudaFreeHost(sl.p);
        if (sl.ev)
            cudaEventDestroy(sl.ev);
    }
    if (c->ev_run)
        cudaEventDestroy(c->ev_run);
    for (auto &kv : c->sets)
        if (kv.second->ready)
            cudaEventDestroy(kv.second->ready);
    for (auto e : c->set_events)
        cudaEventDestroy(e);
    if (c->copy_stream) {
        cudaStreamSynchronize(c->copy_stream);
        cudaStreamDestroy(c->copy_stream);
    }
    if (c->run_stream) {
        cudaStreamSynchronize(c->run_stream);
        cudaStreamDestroy(c->run_stream);
    }
    if (c->ev_in)
        cudaEventDestroy(c->ev_in);
    if (c->ev_out)
        cudaEventDestroy(c->ev_out);
    for (int b = 0; b < 2; ++b) {
        if (c->ev_copied[b])
            cudaEventDestroy(c->ev_copied[b]);
        if (c->ev_packed[b])
            cudaEventDestroy(c->ev_packed[b]);
    }
    if (c->ev_load_start)
        cudaEventDestroy(c->ev_load_start);
    if (c->ev_last_copy)
        cudaEventDestroy(c->ev_last_copy);
    if (c->stream)
        cudaStreamDestroy(c->stream);
    delete c;
}

ah_status ah_set_profiling(ah_ctx *c, int enable)
{
    if (!c)
        return AH_ERR_ARG;
    return guarded(c, [&] {
        require_idle(c);
        AH_CUDA(cudaStreamSynchronize(c->stream));
        prof_flush(c);
        c->prof.clear();
        c->launches_total = 0;
        c->profiling = enable == 1 || enable == 3;
        c->prof_streaming_only = enable == 3;
        c->host_timing = enable >= 1 && enable <= 3;
    });
}

ah_status ah_get_profile(const ah_ctx *c, const char *stage, double *ms, uint64_t *launches, uint64_t *calls)
{
    if (!c)
        return AH_ERR_ARG;
    if (!c->pending.empty()) { // read the event timings still pending
        try {
            cudaSetDevice(c->device);
            prof_flush(const_cast<ah_ctx *>(c));
        } catch (...) {
        }
    }
    double m = 0;
    uint64_t l = 0, k = 0;
    if (!stage) {
        for (auto &kv : c->prof) {
            if (kv.first.compare(0, 5, "host.") == 0)
                continue;
            m += kv.second.ms;
            k += kv.second.calls;
        }
        l = c->launches_total;
    } else {
        auto it = c->prof.find(stage);
        if (it != c->prof.end()) {
            m = it->second.ms;
            l = it->second.launches;
            k = it->second.calls;
        }
    }
    if (ms)
        *ms = m;
    if (launches)
        *launches = l;
    if (calls)
        *calls = k;
    return AH_OK;
}

const char *ah_last_error(const ah_ctx *c)
{
    if (!c)
        return g_create_err.c_str();
    return c->err.c_str();
}

size_t ah_device_bytes(const ah_ctx *c) { return c ? c->used : 0; }

ah_status ah_load_genomes(ah_ctx *c, const uint8_t *seq, uint64_t n_bases, const uint64_t *contig_off,
                          uint32_t n_contigs, const uint32_t *contig_genome, uint32_t *set_id_out, void *stream)
{
    return ah_load_genomes_ex(c, seq, n_bases, contig_off, n_contigs, contig_genome, 0, set_id_out, stream);
}

namespace {
// 2-bit input of ah_load_genomes_2bit: codes (host or device), no-base runs (host)
struct TwoBit {
    const uint64_t *gaps = nullptr;
    uint64_t n_gaps = 0;
};
} // namespace

static ah_status load_impl(ah_ctx *c, const uint8_t *seq, uint64_t n_bases, const uint64_t *contig_off,
                           uint32_t n_contigs, const uint32_t *contig_genome, uint32_t flags, uint32_t *set_id_out,
                           void *stream, const TwoBit *two)
{
    if (!c)
        return AH_ERR_ARG;
    return guarded(c, [&] {
        HostSpan hs(c, "host.load");
        require((flags & ~(AH_LOAD_REVERSED | AH_LOAD_HOST_ASYNC)) == 0, AH_ERR_ARG,
                "ah_load_genomes_ex: unknown flag bits");
        const bool reversed = (flags & AH_LOAD_REVERSED) != 0;
        const bool host_async = (flags & AH_LOAD_HOST_ASYNC) != 0;
        require(set_id_out && contig_off && contig_genome && n_contigs >= 1, AH_ERR_ARG,
                "ah_load_genomes: null argument or no contigs");
        require(n_bases == 0 || seq, AH_ERR_ARG, "ah_load_genomes: seq is null");
        require(n_bases < (1ull << 44), AH_ERR_ARG, "ah_load_genomes: more than 2^44 bases in one set");
        require(contig_off[0] == 0 && contig_off[n_contigs] == n_bases, AH_ERR_ARG,
                "ah_load_genomes: contig_off must start at 0 and end at n_bases");
        for (uint32_t i = 0; i < n_contigs; ++i)
            require(contig_off[i] <= contig_off[i + 1], AH_ERR_ARG, "ah_load_genomes: contig_off not monotone");
        for (uint32_t i = 0; i < n_contigs; ++i)
            require(contig_off[i + 1] - contig_off[i] < (1ull << 32), AH_ERR_ARG,
                    "ah_load_genomes: contig longer than 2^32 - 1");
        cudaStream_t st = stream_of(c, stream);
        auto gs = std::make_unique<GenomeSet>();
        gs->n_bases = n_bases;
        gs->n_contigs = n_contigs;
        gs->n_tiles = (n_bases + kTileBases - 1) / kTileBases;
        gs->contig_off_h.assign(contig_off, contig_off + n_contigs + 1);
        gs->contig_genome_h.assign(contig_genome, contig_genome + n_contigs);
        {
            std::vector<uint32_t> ids(contig_genome, contig_genome + n_contigs);
            std::sort(ids.begin(), ids.end());
            gs->max_genome = ids.back();
            gs->n_genomes = (uint64_t)(std::unique(ids.begin(), ids.end()) - ids.begin());
        }
        const size_t plane_bytes = gs->n_tiles * kTileBytes;
        HostSpan hs_alloc(c, "host.load.alloc");
        // the three tables in one block (one copy fills them): contig offsets,
        // genome ids, per-tile contigs
        const size_t ob = (n_contigs + 1) * sizeof(uint64_t), gb = n_contigs * sizeof(uint32_t),
                     tb = 2 * (gs->n_tiles + 1) * sizeof(uint32_t);
        const size_t table_bytes = ob + gb + tb; // a multiple of 4; ob keeps the rest 4-byte aligned
        try {
            gs->planes = (uint32_t *)dev_alloc(c, plane_bytes);
            gs->contig_off = (uint64_t *)dev_alloc(c, table_bytes);
        } catch (...) {
            dev_free(c, gs->planes, plane_bytes);
            dev_free(c, gs->contig_off, table_bytes);
            throw;
        }
        gs->contig_genome = (uint32_t *)((char *)gs->contig_off + ob);
        gs->tile_contig = (uint32_t *)((char *)gs->contig_off + ob + gb);
        gs->tile_room = gs->tile_contig + (gs->n_tiles + 1);
        gs->bytes = plane_bytes + table_bytes;
        const bool dev_seq = n_bases && is_device_ptr(c, seq);
        // a queued run leaves the flag block alone for plain loads (host or device input)
        require(!reversed || !c->pend.active, AH_ERR_ARG, "a run is pending: reversed sets are loaded after ah_run_end");
        require(!two || !reversed, AH_ERR_ARG, "ah_load_genomes_2bit: no reversed form");
        require(!two || !dev_seq || reinterpret_cast<uintptr_t>(seq) % 16 == 0, AH_ERR_ARG,
                "ah_load_genomes_2bit: device codes must be 16-byte aligned");
        // the packing first (it reads no contig table), then the tables' copies
        std::vector<void *> temp; // freed once the packing is done (reversed loads)
        if (gs->n_tiles && reversed) {
            HostSpan hs_pack(c, "host.load.pack");
            // decoy: the input on the device, reversed contig by contig, then packed
            const uint8_t *src = seq;
            if (!dev_seq) {
                uint8_t *d = (uint8_t *)dev_alloc(c, n_bases);
                temp.push_back(d);
                AH_CUDA(cudaMemcpyAsync(d, seq, n_bases, cudaMemcpyHostToDevice, st));
                src = d;
            }
            uint8_t *dst = (uint8_t *)dev_alloc(c, n_bases);
            temp.push_back(dst);
            const uint64_t kStretch = 1ull << 16;
            std::vector<RevChunk> ch;
            ch.reserve(n_bases / kStretch + n_contigs);
            for (uint32_t i = 0; i < n_contigs; ++i) {
                const uint64_t o = contig_off[i], len = contig_off[i + 1] - o;
                for (uint64_t q = 0; q < len; q += kStretch)
                    ch.push_back({o + q, 2 * o + len - 1, std::min(kStretch, len - q)});
            }
            RevChunk *ch_d = (RevChunk *)dev_alloc(c, std::max<size_t>(ch.size(), 1) * sizeof(RevChunk));
            temp.push_back(ch_d);
            AH_CUDA(cudaMemcpyAsync(ch_d, ch.data(), ch.size() * sizeof(RevChunk), cudaMemcpyHostToDevice, st));
            Stage sg(c, "pack", st, 2);
            launch_reverse_contigs(src, dst, ch_d, ch.size(), st);
            launch_pack(dst, 0, n_bases, n_bases, gs->planes, 0, gs->n_tiles, c->d_err, st);
        } else if (gs->n_tiles && two) {
            HostSpan hs_pack(c, "host.load.pack");
            // the no-base runs on the device, owned by the set (another load in flight on
            // another stream must not overwrite them while this packing reads them),
            // followed by each tile's first run that ends after the tile's start (a
            // merge walk here, so the packing searches nothing); through a pinned
            // slot, like the contig tables
            const uint64_t run_bytes = two->n_gaps * 16, tab_bytes = (gs->n_tiles + 1) * 4;
            gs->gaps_bytes = std::max<uint64_t>(run_bytes + tab_bytes, 16);
            gs->gaps = (uint64_t *)dev_alloc(c, gs->gaps_bytes);
            uint64_t *gaps_d = gs->gaps;
            const uint32_t *tile_gap_d = reinterpret_cast<const uint32_t *>(gs->gaps + 2 * two->n_gaps);
            {
                ah_ctx::PinSlot &gsl = pin_slot(c, run_bytes + tab_bytes);
                memcpy(gsl.p, two->gaps, run_bytes);
                uint32_t *tg = reinterpret_cast<uint32_t *>(gsl.p + run_bytes);
                uint64_t gi = 0;
                for (uint64_t t = 0; t <= gs->n_tiles; ++t) {
                    const uint64_t p0 = t * kTileBases;
                    while (gi < two->n_gaps && two->gaps[2 * gi] + two->gaps[2 * gi + 1] <= p0)
                        ++gi;
                    tg[t] = (uint32_t)gi;
                }
                launch_copy_words((const uint32_t *)gsl.dp, (uint32_t *)gaps_d, (run_bytes + tab_bytes) / 4, st);
                AH_CUDA(cudaEventRecord(gsl.ev, st));
            }
            if (dev_seq) {
                Stage sg(c, "pack", st, 1);
                launch_pack2(seq, 0, n_bases, n_bases, gaps_d, two->n_gaps, tile_gap_d, gs->planes, 0, gs->n_tiles,
                             st);
            } else {
                // host codes: tile-aligned chunks through two staging buffers (the whole
                // set in one when it fits), copies on the copy stream beside the packing
                // of the previous chunk; each chunk also carries the next 64 positions
                // (the extension row)
                uint8_t *stage[2];
                const uint64_t cap = host_stage(c, (gs->n_tiles * kTileBases + 64) / 4 + 16, stage);
                const uint64_t chunk_tiles = std::max<uint64_t>(1, (cap * 4 - 128) / kTileBases);
                AH_CUDA(cudaStreamWaitEvent(c->copy_stream, c->ev_packed[0], 0));
                AH_CUDA(cudaStreamWaitEvent(c->copy_stream, c->ev_packed[1], 0));
                AH_CUDA(cudaEventRecord(c->ev_load_start, st));
                AH_CUDA(cudaStreamWaitEvent(c->copy_stream, c->ev_load_start, 0));
                uint64_t i = 0;
                for (uint64_t t0 = 0; t0 < gs->n_tiles; t0 += chunk_tiles, ++i) {
                    const int b = (int)(i & 1);
                    const uint64_t t1 = std::min(gs->n_tiles, t0 + chunk_tiles);
                    const uint64_t b0 = t0 * kTileBases;
                    const uint64_t b1 = std::min(n_bases, t1 * kTileBases + 64);
                    if (i >= 2)
                        AH_CUDA(cudaStreamWaitEvent(c->copy_stream, c->ev_packed[b], 0));
                    AH_CUDA(cudaMemcpyAsync(stage[b], seq + b0 / 4, (b1 - b0 + 3) / 4, cudaMemcpyHostToDevice,
                                            c->copy_stream));
                    AH_CUDA(cudaEventRecord(c->ev_copied[b], c->copy_stream));
                    AH_CUDA(cudaStreamWaitEvent(st, c->ev_copied[b], 0));
                    {
                        Stage sg(c, "pack", st, 1);
                        launch_pack2(stage[b], b0, b1 - b0, n_bases, gaps_d, two->n_gaps, tile_gap_d, gs->planes, t0,
                                     t1, st);
                    }
                    AH_CUDA(cudaEventRecord(c->ev_packed[b], st));
                }
                AH_CUDA(cudaEventRecord(c->ev_last_copy, c->copy_stream));
            }
        } else if (gs->n_tiles) {
            HostSpan hs_pack(c, "host.load.pack");
            if (dev_seq) {
                // stream-ordered: the pack runs after the caller's earlier work on
                // the stream; a device-side failure reaches the next call that
                // synchronises (the error word is kept until the host reads it)
                Stage sg(c, "pack", st, 1);
                launch_pack(seq, 0, n_bases, n_bases, gs->planes, 0, gs->n_tiles, c->d_err, st);
            } else {
                // host sequence: tile-aligned chunks through two staging buffers; the
                // copies run on a second stream so chunk i+1 crosses the link while chunk
                // i is packed.  Each chunk also carries the next tile (extension words).
                uint8_t *stage[2];
                const uint64_t cap = host_stage(c, gs->n_tiles * kTileBases + kTileBases, stage);
                const uint64_t chunk_tiles = std::max<uint64_t>(1, (cap - kTileBases) / kTileBases);
                // the copy stream starts after everything queued so far on st, and after
                // the packing of an earlier load from these staging buffers
                AH_CUDA(cudaStreamWaitEvent(c->copy_stream, c->ev_packed[0], 0));
                AH_CUDA(cudaStreamWaitEvent(c->copy_stream, c->ev_packed[1], 0));
                AH_CUDA(cudaEventRecord(c->ev_load_start, st));
                AH_CUDA(cudaStreamWaitEvent(c->copy_stream, c->ev_load_start, 0));
                uint64_t i = 0;
                for (uint64_t t0 = 0; t0 < gs->n_tiles; t0 += chunk_tiles, ++i) {
                    const int b = (int)(i & 1);
                    const uint64_t t1 = std::min(gs->n_tiles, t0 + chunk_tiles);
                    const uint64_t b0 = t0 * kTileBases;
                    const uint64_t b1 = std::min(n_bases, t1 * kTileBases + kTileBases);
                    if (i >= 2) // staging buffer b is free once the chunk packed from it two rounds ago is done
                        AH_CUDA(cudaStreamWaitEvent(c->copy_stream, c->ev_packed[b], 0));
                    AH_CUDA(cudaMemcpyAsync(stage[b], seq + b0, b1 - b0, cudaMemcpyHostToDevice, c->copy_stream));
                    AH_CUDA(cudaEventRecord(c->ev_copied[b], c->copy_stream));
                    AH_CUDA(cudaStreamWaitEvent(st, c->ev_copied[b], 0));
                    {
                        Stage sg(c, "pack", st, 1);
                        launch_pack(stage[b], b0, b1 - b0, n_bases, gs->planes, t0, t1, c->d_err, st);
                    }
                    AH_CUDA(cudaEventRecord(c->ev_packed[b], st));
                }
                AH_CUDA(cudaEventRecord(c->ev_last_copy, c->copy_stream));
            }
        }
        {
            HostSpan hs_tables(c, "host.load.tables");
            // the tables through a mapped pinned slot, read by one copy kernel; the
            // per-tile contig table is built here by a merge walk over tiles and contigs
            ah_ctx::PinSlot &sl = pin_slot(c, table_bytes);
            memcpy(sl.p, contig_off, ob);
            memcpy(sl.p + ob, contig_genome, gb);
            {
                // tile t: the last contig starting at or before t * kTileBases, and
                // the room from the tile's first position to that contig's end
                uint32_t *tc = (uint32_t *)(sl.p + ob + gb);
                uint32_t *room = tc + (gs->n_tiles + 1);
                uint32_t ci = 0;
                for (uint64_t t = 0; t <= gs->n_tiles; ++t) {
                    const uint64_t P = t * kTileBases;
                    while (ci + 1 < n_contigs && contig_off[ci + 1] <= P)
                        ++ci;
                    tc[t] = ci;
                    const uint64_t end = n_contigs ? contig_off[ci + 1] : 0;
                    room[t] = end > P ? (uint32_t)std::min<uint64_t>(end - P, 0xffffffffull) : 0u;
                }
            }
            Stage sg(c, "tables", st, 1);
            launch_copy_words((const uint32_t *)sl.dp, (uint32_t *)gs->contig_off, table_bytes / 4, st);
            AH_CUDA(cudaEventRecord(sl.ev, st));
        }
        if (c->set_events.empty()) {
            cudaEvent_t e;
            AH_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            c->set_events.push_back(e);
        }
        gs->ready = c->set_events.back();
        c->set_events.pop_back();
        AH_CUDA(cudaEventRecord(gs->ready, st));
        if (!dev_seq && !reversed) {
            // the caller's host buffer may be reused once this call returns: wait for
            // the copies only; the packing stays queued (like a device-input load, a
            // failure reaches the next call that synchronises), so a host load may
            // also overlap a pending run.  AH_LOAD_HOST_ASYNC: the caller keeps the
            // buffer unchanged until the set is ready, so the copies stay queued too
            if (gs->n_tiles && !host_async)
                AH_CUDA(cudaEventSynchronize(c->ev_last_copy));
            c->flags_dirty = true;
        } else if (reversed) { // the temporaries are freed once the packing is done
            try {
                check_flags(c, st);
            } catch (...) {
                for (void *q : temp)
                    dev_free(c, q, 0);
                throw;
            }
            for (void *q : temp) // the packing is done: the temporaries go back to the cache
                dev_free(c, q, 0);
        } else {
            c->flags_dirty = true;
        }
        uint32_t id = c->next_set++;
        c->sets[id] = std::move(gs);
        *set_id_out = id;
    });
}

ah_status ah_load_genomes_ex(ah_ctx *c, const uint8_t *seq, uint64_t n_bases, const uint64_t *contig_off,
                             uint32_t n_contigs, const uint32_t *contig_genome, uint32_t flags, uint32_t *set_id_out,
                             void *stream)
{
    return load_impl(c, seq, n_bases, contig_off, n_contigs, contig_genome, flags, set_id_out, stream, nullptr);
}

ah_status ah_load_genomes_2bit(ah_ctx *c, const uint8_t *codes, uint64_t n_bases, const uint64_t *gaps,
                               uint64_t n_gaps, const uint64_t *contig_off, uint32_t n_contigs,
                               const uint32_t *contig_genome, uint32_t *set_id_out, void *stream)
{
    return ah_load_genomes_2bit_ex(c, codes, n_bases, gaps, n_gaps, contig_off, n_contigs, contig_genome, 0,
                                   set_id_out, stream);
}

ah_status ah_load_genomes_2bit_ex(ah_ctx *c, const uint8_t *codes, uint64_t n_bases, const uint64_t *gaps,
                                  uint64_t n_gaps, const uint64_t *contig_off, uint32_t n_contigs,
                                  const uint32_t *contig_genome, uint32_t flags, uint32_t *set_id_out, void *stream)
{
    if (!c)
        return AH_ERR_ARG;
    if (flags & ~AH_LOAD_HOST_ASYNC) {
        c->err = "ah_load_genomes_2bit_ex: unknown flag bits (AH_LOAD_HOST_ASYNC only)";
        return AH_ERR_ARG;
    }
    if ((n_gaps && !gaps) || (n_bases && !codes)) {
        c->err = "ah_load_genomes_2bit: null codes or gaps";
        return AH_ERR_ARG;
    }
    if (n_gaps > 0xffffffffull) {
        c->err = "ah_load_genomes_2bit: more than 2^32 - 1 no-base runs";
        return AH_ERR_ARG;
    }
    for (uint64_t g = 0; g < n_gaps; ++g) { // sorted, disjoint, inside the set
        const uint64_t a = gaps[2 * g], len = gaps[2 * g + 1];
        if (len == 0 || a + len > n_bases || a + len < a || (g && a < gaps[2 * g - 2] + gaps[2 * g - 1])) {
            c->err = "ah_load_genomes_2bit: gaps must be sorted, disjoint, non-empty runs inside the set";
            return AH_ERR_ARG;
        }
    }
    TwoBit two;
    two.gaps = gaps;
    two.n_gaps = n_gaps;
    return load_impl(c, codes, n_bases, contig_off, n_contigs, contig_genome, flags, set_id_out, stream, &two);
}

ah_status ah_unload_genomes(ah_ctx *c, uint32_t set_id)
{
    if (!c)
        return AH_ERR_ARG;
    return guarded(c, [&] {
        require_idle(c);
        HostSpan hs(c, "host.unload");
        GenomeSet &gs = get_set(c, set_id);
        // the calls that read a set synchronise before they return; its packing may not have
        if (gs.ready)
            AH_CUDA(cudaEventSynchronize(gs.ready));
        // a failure of a packing nothing else synchronised on is reported here
        const int e = c->flags_dirty ? read_flags(c, c->stream) : 0;
        dev_free(c, gs.planes, gs.n_tiles * kTileBytes);
        dev_free(c, gs.contig_off, 0); // the block of the three tables
        dev_free(c, gs.gaps, gs.gaps_bytes);
        if (gs.ready)
            c->set_events.push_back(gs.ready);
        c->sets.erase(set_id);
        raise_device_error(e);
    });
}

ah_status ah_set_primers(ah_ctx *c, const char *fwd, const char *rev, const ah_pcr_params *p, uint32_t *pair_id_out)
{
    if (!c)
        return AH_ERR_ARG;
    return guarded(c, [&] {
        require_idle(c);
        require(fwd && rev && p && pair_id_out, AH_ERR_ARG, "ah_set_primers: null argument");
        PrimerPair pp;
        const char *pr[2] = {fwd, rev};
        for (int x = 0; x < 2; ++x) {
            const size_t L = strlen(pr[x]);
            require(L >= AH_MIN_PRIMER_LEN, AH_ERR_PRIMER, "primer shorter than 5 letters");
            require(L <= AH_MAX_PRIMER_LEN, AH_ERR_PRIMER, "primer longer than 32 letters");
            double deg = 1.0;
            for (size_t i = 0; i < L; ++i) {
                const int m = iupac_mask(pr[x][i]);
                require(m != 0, AH_ERR_PRIMER, std::string("non-IUPAC letter in primer: '") + pr[x][i] + "'");
                pp.mask[x][i] = (uint8_t)m;
                deg *= (double)__builtin_popcount(m);
            }
            require(deg <= AH_MAX_DEGENERACY, AH_ERR_PRIMER, "primer degeneracy above 10000");
            pp.L[x] = (int)L;
        }
        pp.fwd = fwd;
        pp.rev = rev;
        require(p->k >= 0 && p->k <= AH_MAX_MISMATCHES, AH_ERR_PRIMER, "k must be 0..10");
        require(p->clamp >= 0, AH_ERR_ARG, "clamp must be >= 0");
        require(p->min_len >= 0 && p->min_len <= p->max_len, AH_ERR_ARG, "need 0 <= min_len <= max_len");
        require(p->saltcorr == 0 || p->saltcorr == 1 || p->saltcorr == 5, AH_ERR_ARG, "saltcorr must be 0, 1 or 5");
        require(!std::isnan(p->tm_min) && p->tm_min < INFINITY, AH_ERR_ARG, "tm_min must be a number or -inf");
        const double vals[] = {p->dnac1_nM, p->dnac2_nM, p->Na_mM, p->K_mM, p->Tris_mM, p->Mg_mM, p->dNTPs_mM};
        for (double v : vals)
            require(std::isfinite(v) && v >= 0, AH_ERR_ARG, "concentrations must be finite and >= 0");
        require(p->dnac1_nM - p->dnac2_nM / 2.0 > 0, AH_ERR_ARG, "need dnac1 > dnac2 / 2");
        require(p->saltcorr == 0 || na_eq_mM(*p) > 0, AH_ERR_ARG, "salt correction needs [Na_eq] > 0");
        pp.params = *p;
        default_table(&pp.table);
        uint32_t id = c->next_pair++;
        c->pairs[id] = pp;
        ++c->pairs_version;
        *pair_id_out = id;
    });
}

ah_status ah_set_nn_table(ah_ctx *c, uint32_t pair_id, const ah_nn_table *t)
{
    if (!c)
        return AH_ERR_ARG;
    return guarded(c, [&] {
        require_idle(c);
        PrimerPair &pp = get_pair(c, pair_id);
        ++c->pairs_version;
        if (!t) {
            default_table(&pp.table);
            return;
        }
        for (int i = 0; i < 256; ++i)
            require(std::isfinite(t->stack_dH[i]) && std::isfinite(t->stack_dS[i]), AH_ERR_ARG, "non-finite entry");
        for (int i = 0; i < 16; ++i)
            require(std::isfinite(t->term_dH[i]) && std::isfinite(t->term_dS[i]), AH_ERR_ARG, "non-finite entry");
        pp.table = *t;
        ++c->pairs_version;
    });
}

ah_status ah_scan(ah_ctx *c, uint32_t set_id, const uint32_t *pair_ids, uint32_t n_pairs, ah_site *out,
                  uint64_t cap, uint64_t *n_out, void *stream)
{
    if (!c)
        return AH_ERR_ARG;
    return guarded(c, [&] {
        require_idle(c);
        require(n_out != nullptr && (cap == 0 || out != nullptr), AH_ERR_ARG, "ah_scan: null output");
        require(pair_ids && n_pairs >= 1 && n_pairs <= AH_MAX_PAIRS_PER_SCAN, AH_ERR_ARG, "n_pairs must be 1..16");
        *n_out = 0;
        GenomeSet &gs = get_set(c, set_id);
        cudaStream_t st = stream_of(c, stream);
        wait_ready(gs, st);
        std::vector<ScanPattern> pats = patterns_of(c, pair_ids, n_pairs);
        uint64_t *keys = nullptr;
        const uint64_t count = scan_keys(c, gs, pats, &keys, st);
        *n_out = count;
        if (count > cap)
            throw Error(AH_ERR_OVERFLOW, "ah_scan: " + std::to_string(count) + " sites, capacity " +
                                             std::to_string(cap));
        if (count == 0)
            return;
        ah_site *dst = out_buf(c, "sites_out", out, count);
        sort_decode(c, gs, n_pairs, keys, count, dst, st);
        out_finish(out, dst, count, st);
        AH_CUDA(cudaStreamSynchronize(st));
    });
}

ah_status ah_tune_scan(ah_ctx *c, uint32_t set_id, const uint32_t *pair_ids, uint32_t n_pairs, uint64_t sample_tiles,
                       ah_tune_result *best_out, void *stream)
{
    if (!c)
        return AH_ERR_ARG;
    return guarded(c, [&] {
        require_idle(c);
        require(pair_ids && n_pairs >= 1 && n_pairs <= AH_MAX_PAIRS_PER_SCAN, AH_ERR_ARG, "n_pairs must be 1..16");
        GenomeSet &gs = get_set(c, set_id);
        cudaStream_t st = stream_of(c, stream);
        wait_ready(gs, st);
        std::vector<ScanPattern> pats = patterns_of(c, pair_ids, n_pairs);
        const int pbits = std::max(1, bit_length(gs.n_bases));
        uint64_t tiles = std::min<uint64_t>(gs.n_tiles, sample_tiles ? sample_tiles : 4096);
        require(tiles > 0, AH_ERR_ARG, "ah_tune_scan: empty genome set");
        // the sample must cover whole waves of the persistent grid to time it fairly
        // register-capped variants (more resident warps) first: measured fastest on
        // the 960-oligo pair; R = 8 uncapped for pattern sets that spill under the cap
        std::vector<ScanTuning> cand;
        const int shapes[][2] = {{16, 1}, {8, 2}, {4, 4}}; // warps per CTA, minimum CTAs per SM
        for (const auto &sh : shapes)
            for (int order : {0, 1})
                for (int S : {3, 4}) {
                    ScanTuning t;
                    t.R = 4;
                    t.order = order;
                    t.stages = S;
                    t.warps = sh[0];
                    t.min_blocks = sh[1];
                    cand.push_back(t);
                }
        for (int order : {0, 1}) {
            ScanTuning t;
            t.R = 8;
            t.order = order;
            t.stages = 3;
            t.warps = 4;
            t.min_blocks = 1;
            cand.push_back(t);
        }
        cudaEvent_t e0 = get_event(c), e1 = get_event(c);
        // each launch group is tuned on its own (its kernel is compiled and run alone);
        // the result reports the slowest group's variant and the groups' summed time
        double total_us = 0, worst_us = -1;
        ScanTuning worst = c->tuning;
        int worst_regs = -1;
        for (const std::vector<ScanPattern> &gp : split_launches(pats)) {
            double best_us = 1e30;
            ScanTuning best = c->tuning;
            int best_regs = -1;
            for (const ScanTuning &t : cand) {
                ScanKernel *k = nullptr;
                try {
                    k = scan_kernel(gp, t, c->device);
                } catch (const Error &) {
                    continue; // a variant that does not compile is skipped
                }
                uint64_t *keys = (uint64_t *)scratch(c, "scan_keys", c->key_cap * sizeof(uint64_t));
                float ms_min = 1e30f;
                for (int rep = 0; rep < 4; ++rep) {
                    reset_flags(c, st);
                    AH_CUDA(cudaEventRecord(e0, st));
                    launch_scan(c, k, gs, tiles, keys, c->key_cap, pbits, st, nullptr, c->d_flags + kFlagWork);
                    AH_CUDA(cudaEventRecord(e1, st));
                    AH_CUDA(cudaEventSynchronize(e1));
                    float ms = 0;
                    AH_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                    if (rep > 0)
                        ms_min = std::min(ms_min, ms);
                }
                check_flags(c, st);
                const double us = ms_min * 1e3 / (double)tiles;
                if (getenv("AH_TUNE_VERBOSE"))
                    fprintf(stderr,
                            "ah_tune_scan: patterns=%zu R=%d arith=%d order=%d stages=%d warps=%d regs=%d bps=%d  "
                            "%.4f us/tile\n",
                            gp.size(), t.R, t.arith_pct, t.order, t.stages, t.warps, k->regs, k->blocks_per_sm, us);
                if (us < best_us) {
                    best_us = us;
                    best = t;
                    best_regs = k->regs;
                }
            }
            c->tuned[signature(gp)] = best;
            total_us += best_us;
            if (best_us > worst_us) {
                worst_us = best_us;
                worst = best;
                worst_regs = best_regs;
            }
        }
        c->events.push_back(e0);
        c->events.push_back(e1);
        if (best_out) {
            best_out->R = worst.R;
            best_out->arith_pct = worst.arith_pct;
            best_out->min_blocks = worst.min_blocks;
            best_out->order = worst.order;
            best_out->stages = worst.stages;
            best_out->warps_per_cta = worst.warps;
            best_out->regs = worst_regs;
            best_out->us_per_tile = total_us;
            best_out->tiles = tiles;
        }
    });
}

ah_status ah_run_begin(ah_ctx *c, uint32_t set_id, const uint32_t *pair_ids, uint32_t n_pairs, ah_run_out *o,
                       void *stream, void *scan_done)
{
    if (!c)
        return AH_ERR_ARG;
    return guarded(c, [&] {
        require_idle(c);
        require(o != nullptr, AH_ERR_ARG, "ah_run: out is null");
        require(pair_ids && n_pairs >= 1 && n_pairs <= AH_MAX_PAIRS_PER_SCAN, AH_ERR_ARG, "n_pairs must be 1..16");
        require((o->sites_cap == 0 || o->sites) && (o->amplicons_cap == 0 || o->amplicons) &&
                    (o->seq_cap == 0 || o->seq),
                AH_ERR_ARG, "ah_run: null buffer with non-zero capacity");
        o->n_sites = o->n_amplicons = o->n_seq = 0;
        HostSpan hs(c, "host.run");
        GenomeSet &gs = get_set(c, set_id);
        const cudaStream_t caller = stream_of(c, stream);
        cudaStream_t st = enter_run_stream(c, caller);
        wait_ready(gs, st);
        std::vector<ScanPattern> pats = patterns_of(c, pair_ids, n_pairs);
        const PairDev *pd = upload_pairs(c, pair_ids, n_pairs, st);
        ah_ctx::RunPending &P = c->pend;
        P = ah_ctx::RunPending();
        P.set_id = set_id;
        P.pair_ids.assign(pair_ids, pair_ids + n_pairs);
        P.o = o;
        P.st = st;
        P.caller = caller;
        P.pd = pd;
        if (gs.n_tiles && c->last_sites <= kSmallSort) {
            fast_begin(c, gs, pats, pd, n_pairs, o, st, (cudaEvent_t)scan_done, &P.fr);
            leave_run_stream(c, caller);
            P.active = true;
            return;
        }
        // counts above the one-synchronisation sizes (seen in the last run): queue the
        // scan and its count's copy only; ah_run_end reads the count and finishes step
        // by step, so the caller's next packing (after scan_done) runs beside that
        if (!gs.n_tiles) {
            uint64_t *keys = nullptr;
            const uint64_t ns = scan_keys(c, gs, pats, &keys, st);
            try {
                run_steps(c, gs, pd, n_pairs, keys, ns, o, st);
            } catch (const Error &e) {
                if (e.status != AH_ERR_OVERFLOW)
                    throw;
                P.status = e.status; // reported by ah_run_end, like the counts
                P.msg = e.msg;
            }
            if (scan_done)
                AH_CUDA(cudaEventRecord((cudaEvent_t)scan_done, st));
            leave_run_stream(c, caller);
            P.active = P.done = true;
            return;
        }
        const int pbits = std::max(1, bit_length(gs.n_bases));
        uint64_t *keys = (uint64_t *)scratch(c, "scan_keys", c->key_cap * sizeof(uint64_t));
        reset_flags(c, st);
        {
            Stage sg(c, "scan", st, (int)scan_launch_groups(pats).size());
            launch_scans(c, gs, pats, gs.n_tiles, keys, c->key_cap, pbits, st);
        }
        if (scan_done)
            AH_CUDA(cudaEventRecord((cudaEvent_t)scan_done, st));
        AH_CUDA(cudaMemcpyAsync(c->h_flags, c->d_flags, kFlagWords * sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
        AH_CUDA(cudaEventRecord(c->ev_run, st));
        P.fr.keys = keys;
        P.scan_only = true;
        leave_run_stream(c, caller);
        P.active = true;
    });
}

ah_status ah_run_end(ah_ctx *c)
{
    if (!c)
        return AH_ERR_ARG;
    return guarded(c, [&] {
        require(c->pend.active, AH_ERR_ARG, "ah_run_end: no run is pending");
        const ah_ctx::RunPending P = c->pend;
        c->pend.active = false; // completed or failed, it is no longer pending
        HostSpan hs(c, "host.run");
        if (P.done) {
            if (P.status != AH_OK)
                throw Error(P.status, P.msg);
            return;
        }
        GenomeSet &gs = get_set(c, P.set_id);
        const uint32_t n_pairs = (uint32_t)P.pair_ids.size();
        uint64_t *keys = nullptr;
        uint64_t ns = 0;
        if (P.scan_only) { // the scan ran alone: its count, then step by step
            {
                HostSpan span(c, "host.run.wait");
                AH_CUDA(cudaEventSynchronize(c->ev_run));
            }
            c->flags_dirty = false;
            const int e = (int)(c->h_flags[kFlagErr] & 0xffffffffu);
            if (e != 0) {
                AH_CUDA(cudaMemsetAsync(c->d_flags + kFlagErr, 0, sizeof(uint64_t), P.st));
                raise_device_error(e);
            }
            ns = c->h_flags[kFlagCounter];
            keys = P.fr.keys;
            if (ns > c->key_cap) { // the key buffer was too small: grow it and scan again
                c->key_cap = ns;
                std::vector<ScanPattern> pats = patterns_of(c, P.pair_ids.data(), n_pairs);
                ns = scan_keys(c, gs, pats, &keys, P.st);
            }
            run_steps(c, gs, P.pd, n_pairs, keys, ns, P.o, P.st);
            leave_run_stream(c, P.caller);
            return;
        }
        const FastResult r = fast_end(c, P.o, P.st, P.fr, &keys, &ns);
        if (r == kFastDone) {
            leave_run_stream(c, P.caller); // delivery copies may have been queued
            return;
        }
        if (r == kFastRescan) {
            std::vector<ScanPattern> pats = patterns_of(c, P.pair_ids.data(), n_pairs);
            ns = scan_keys(c, gs, pats, &keys, P.st);
        }
        run_steps(c, gs, P.pd, n_pairs, keys, ns, P.o, P.st);
        leave_run_stream(c, P.caller);
    });
}

ah_status ah_run(ah_ctx *c, uint32_t set_id, const uint32_t *pair_ids, uint32_t n_pairs, ah_run_out *o, void *stream)
{
    const ah_status st = ah_run_begin(c, set_id, pair_ids, n_pairs, o, stream, nullptr);
    if (st != AH_OK)
        return st;
    return ah_run_end(c);
}

ah_status ah_tm_sweep(ah_ctx *c, uint32_t set_id, const uint32_t *pair_ids, uint32_t n_pairs, const ah_site *sites,
                      uint64_t n_sites, const ah_amplicon *amplicons, uint64_t n_amplicons, const double *thresholds,
                      uint32_t n_thresholds, ah_sweep_row *rows, uint64_t *n_genomes_out, void *stream)
{
    if (!c)
        return AH_ERR_ARG;
    return guarded(c, [&] {
        require_idle(c);
        require(thresholds && rows && n_genomes_out && (n_sites == 0 || sites) && (n_amplicons == 0 || amplicons),
                AH_ERR_ARG, "ah_tm_sweep: null argument");
        require(n_thresholds >= 1 && n_thresholds <= (uint32_t)kSweepThresholds, AH_ERR_ARG,
                "ah_tm_sweep: 1..64 thresholds");
        for (uint32_t j = 0; j < n_thresholds; ++j)
            require(std::isfinite(thresholds[j]), AH_ERR_ARG, "ah_tm_sweep: thresholds must be finite");
        GenomeSet &gs = get_set(c, set_id);
        cudaStream_t st = stream_of(c, stream);
        wait_ready(gs, st);
        const PairDev *pd = upload_pairs(c, pair_ids, n_pairs, st);
        *n_genomes_out = gs.n_genomes;
        reset_flags(c, st);
        const ah_site *s = stage_in(c, "sweep_sites_in", sites, n_sites, st);
        const ah_amplicon *a = stage_in(c, "sweep_amps_in", amplicons, n_amplicons, st);
        if (n_sites) {
            Stage sg(c, "validate", st, 1);
            launch_validate_sites(s, n_sites, pd, (int)n_pairs, gs.contig_off, gs.n_contigs, c->d_err, st);
        }
        check_flags(c, st);
        float *tm = (float *)scratch(c, "sweep_tm", std::max<uint64_t>(n_sites, 1) * sizeof(float));
        if (n_sites) {
            Stage sg(c, "tm", st, 2);
            uint32_t *q = (uint32_t *)scratch(c, "tm_queue", 2 * n_sites * sizeof(uint32_t));
            launch_tm(s, n_sites, nullptr, pd, (int)n_pairs, gs.planes, gs.contig_off, tm, nullptr, q,
                      (uint32_t *)(c->d_flags + kFlagTmQueue), tm_seg_max(c), tm_few_exact(c), c->d_err, st);
        }
        double *thr_d = (double *)scratch(c, "sweep_thr", kSweepThresholds * sizeof(double));
        AH_CUDA(cudaMemcpyAsync(thr_d, thresholds, n_thresholds * sizeof(double), cudaMemcpyHostToDevice, st));
        long long *W = (long long *)scratch(c, "sweep_w", (size_t)n_pairs * n_thresholds * 272 * sizeof(long long));
        uint64_t *mask = (uint64_t *)scratch(c, "sweep_mask", std::max<uint64_t>(n_sites, 1) * sizeof(uint64_t));
        auto *gmask = (unsigned long long *)scratch(c, "sweep_gmask", ((uint64_t)gs.max_genome + 1) * 8);
        auto *counts = (unsigned long long *)scratch(c, "sweep_counts", 3 * kSweepThresholds * 8);
        {
            Stage sg(c, "sweep", st, 4);
            launch_tm_sweep(s, n_sites, a, n_amplicons, pd, (int)n_pairs, gs.planes, gs.contig_off, tm, thr_d,
                            (int)n_thresholds, W, tm_few_exact(c), mask, gmask, gs.max_genome, counts, c->d_err, st);
        }
        std::vector<unsigned long long> h(3 * kSweepThresholds);
        AH_CUDA(cudaMemcpyAsync(h.data(), counts, h.size() * 8, cudaMemcpyDeviceToHost, st));
        check_flags(c, st); // also waits for the copy
        std::vector<ah_sweep_row> r(n_thresholds);
        for (uint32_t j = 0; j < n_thresholds; ++j)
            r[j] = {h[j], h[kSweepThresholds + j], h[2 * kSweepThresholds + j]};
        AH_CUDA(cudaMemcpyAsync(rows, r.data(), n_thresholds * sizeof(ah_sweep_row), cudaMemcpyDefault, st));
        AH_CUDA(cudaStreamSynchronize(st));
    });
}

ah_status ah_amplitypes(ah_ctx *c, uint32_t set_id, const ah_amplicon *amplicons, uint64_t n, uint32_t *variant_out,
                        ah_genome_amplitype *rows, uint64_t cap, uint64_t *n_rows_out, uint64_t *n_variants_out,
                        uint64_t *n_amplitypes_out, void *stream)
{
    if (!c)
        return AH_ERR_ARG;
    return guarded(c, [&] {
        require_idle(c);
        require(n_rows_out && n_variants_out && n_amplitypes_out && (n == 0 || amplicons) && (cap == 0 || rows),
                AH_ERR_ARG, "ah_amplitypes: null argument");
        require(n < (1ull << 32), AH_ERR_ARG, "ah_amplitypes: at most 2^32 - 1 amplicons");
        *n_rows_out = *n_variants_out = *n_amplitypes_out = 0;
        GenomeSet &gs = get_set(c, set_id);
        cudaStream_t st = stream_of(c, stream);
        wait_ready(gs, st);
        if (n == 0)
            return;
        reset_flags(c, st);
        const ah_amplicon *a = stage_in(c, "amplitype_in", amplicons, n, st);
        const uint64_t G = (uint64_t)gs.max_genome + 1;  // genome id range
        const uint64_t N = std::max<uint64_t>(n, G);     // the largest count a scratch array serves
        {   // the records lie in the set (checked before any kernel reads planes with them)
            uint64_t *len = (uint64_t *)scratch(c, "fetch_len", (n + 1) * sizeof(uint64_t));
            Stage sg(c, "validate", st, 1);
            launch_fetch_lengths(a, n, nullptr, gs.contig_off, gs.n_contigs, len, c->d_err, st);
        }
        check_flags(c, st);
        AmpliTypeScratch S;
        S.idx = (uint32_t *)scratch(c, "at_idx", N * 4);
        S.idx_b = (uint32_t *)scratch(c, "at_idx_b", N * 4);
        S.run_pos = (uint32_t *)scratch(c, "at_run_pos", N * 4);
        S.keys_a = (uint64_t *)scratch(c, "at_keys_a", N * 8);
        S.keys_b = (uint64_t *)scratch(c, "at_keys_b", N * 8);
        S.keys_s = (uint64_t *)scratch(c, "at_keys_s", N * 8);
        S.head = (uint64_t *)scratch(c, "at_head", N * 8);
        S.head_excl = (uint64_t *)scratch(c, "at_head_excl", N * 8);
        S.is_first = (uint64_t *)scratch(c, "at_is_first", N * 8);
        S.rank = (uint64_t *)scratch(c, "at_rank", N * 8);
        S.temp_bytes = AmpliTypeScratch::cub_bytes(N);
        S.temp = scratch(c, "at_cub", S.temp_bytes);
        S.scan_bytes = scan_u64_temp_bytes(N);
        S.scan_temp = scratch(c, "scan_temp", S.scan_bytes);
        uint64_t *h1 = (uint64_t *)scratch(c, "at_h1", n * 8), *h2 = (uint64_t *)scratch(c, "at_h2", n * 8);
        uint32_t *variant = (uint32_t *)scratch(c, "at_variant", n * 4);
        uint64_t *counts = c->d_flags + kFlagSites; // three device words: variants, genome runs, rows
        {
            Stage sg(c, "amplitype", st, 1);
            launch_amp_hash(a, n, gs.planes, gs.contig_off, h1, h2, st);
            S.sort_by(h1, h2, n, st);
            S.ids(n, variant, counts + 0, st); // sequence variants
            launch_genome_key(a, variant, n, gs.contig_genome, h1, c->d_err, st); // h1 reused for the keys
            S.sort_by(h1, nullptr, n, st);
            S.ids(n, nullptr, counts + 1, st); // (genome, variant) runs
            auto *g1 = (unsigned long long *)scratch(c, "at_g1", G * 8);
            auto *g2 = (unsigned long long *)scratch(c, "at_g2", G * 8);
            auto *gamp = (unsigned int *)scratch(c, "at_gamp", G * 4);
            auto *gvar = (unsigned int *)scratch(c, "at_gvar", G * 4);
            AH_CUDA(cudaMemsetAsync(g1, 0, G * 8, st));
            AH_CUDA(cudaMemsetAsync(g2, 0, G * 8, st));
            AH_CUDA(cudaMemsetAsync(gamp, 0, G * 4, st));
            AH_CUDA(cudaMemsetAsync(gvar, 0, G * 4, st));
            S.genome_sums(n, counts + 1, g1, g2, gamp, gvar, st);
            uint32_t *gid = (uint32_t *)scratch(c, "at_gid", G * 4);
            uint64_t *k1 = (uint64_t *)scratch(c, "at_k1", G * 8), *k2 = (uint64_t *)scratch(c, "at_k2", G * 8);
            uint64_t *has = (uint64_t *)scratch(c, "at_has", G * 8), *pos = (uint64_t *)scratch(c, "at_pos", G * 8);
            launch_genome_compact(gamp, G, has, pos, S.scan_temp, S.scan_bytes, g1, g2, gid, k1, k2, counts + 2, st);
            check_flags(c, st);
            const uint64_t m = c->h_flags[kFlagSites + 2];
            const uint64_t nv = c->h_flags[kFlagSites + 0];
            *n_rows_out = m;
            *n_variants_out = nv;
            uint32_t *type = (uint32_t *)scratch(c, "at_type", std::max<uint64_t>(m, 1) * 4);
            S.sort_by(k1, k2, m, st);
            S.ids(m, type, counts + 1, st); // amplitypes, first occurrence in ascending genome order
            ah_genome_amplitype *r = out_buf(c, "at_rows", rows, m <= cap ? m : 0);
            if (m <= cap)
                launch_amplitype_rows(gid, type, m, gamp, gvar, r, st);
            if (variant_out)
                AH_CUDA(cudaMemcpyAsync(variant_out, variant, n * 4, cudaMemcpyDefault, st));
            check_flags(c, st);
            *n_amplitypes_out = c->h_flags[kFlagSites + 1];
            if (m > cap)
                throw Error(AH_ERR_OVERFLOW, "ah_amplitypes: " + std::to_string(m) + " genomes with amplicons, capacity " +
                                                 std::to_string(cap));
            out_finish(rows, r, m, st);
            AH_CUDA(cudaStreamSynchronize(st));
        }
    });
}

ah_status ah_generate_bases(ah_ctx *c, uint64_t seed, const ah_gen_segment *segments, uint64_t n_segments,
                            const uint64_t *patch_pos, const uint8_t *patch_bytes, uint64_t n_patches, uint64_t base0,
                            uint64_t n, uint8_t *out, void *stream)
{
    if (!c)
        return AH_ERR_ARG;
    return guarded(c, [&] {
        require_idle(c);
        require(segments && n_segments >= 1 && (n_patches == 0 || (patch_pos && patch_bytes)), AH_ERR_ARG,
                "ah_generate_bases: null argument");
        require(base0 % 4 == 0, AH_ERR_ARG, "ah_generate_bases: base0 must be a multiple of 4");
        if (n == 0)
            return;
        require(out && is_device_ptr(c, out), AH_ERR_ARG, "ah_generate_bases: out must be device memory");
        cudaStream_t st = stream_of(c, stream);
        const bool dev_tables = is_device_ptr(c, segments);
        if (dev_tables) {
            // device tables: stream-ordered, no host pass over them; a range the
            // segments do not cover is written as N and reported by the next call
            // that synchronises
            require(n_patches == 0 || (is_device_ptr(c, patch_pos) && is_device_ptr(c, patch_bytes)), AH_ERR_ARG,
                    "ah_generate_bases: device segments take device patches");
            {
                Stage sg(c, "generate", st, n_patches ? 2 : 1);
                launch_generate_bases(segments, n_segments, seed, patch_pos, patch_bytes, n_patches, base0, n, out,
                                      c->d_err, st);
            }
            c->flags_dirty = true;
            return;
        }
        require(n_patches == 0 || (!is_device_ptr(c, patch_pos) && !is_device_ptr(c, patch_bytes)), AH_ERR_ARG,
                "ah_generate_bases: host segments take host patches");
        for (uint64_t i = 0; i < n_segments; ++i)
            require(i == 0 || segments[i].end >= segments[i - 1].end, AH_ERR_ARG,
                    "ah_generate_bases: segment ends must not decrease");
        require(segments[n_segments - 1].end >= base0 + n, AH_ERR_ARG,
                "ah_generate_bases: the segments end before the range does");
        auto *segs = (ah_gen_segment *)scratch(c, "gen_segs", n_segments * sizeof(ah_gen_segment));
        AH_CUDA(cudaMemcpyAsync(segs, segments, n_segments * sizeof(ah_gen_segment), cudaMemcpyHostToDevice, st));
        uint64_t *pp = nullptr;
        uint8_t *pb = nullptr;
        if (n_patches) {
            pp = (uint64_t *)scratch(c, "gen_patch_pos", n_patches * sizeof(uint64_t));
            pb = (uint8_t *)scratch(c, "gen_patch_bytes", n_patches);
            AH_CUDA(cudaMemcpyAsync(pp, patch_pos, n_patches * sizeof(uint64_t), cudaMemcpyHostToDevice, st));
            AH_CUDA(cudaMemcpyAsync(pb, patch_bytes, n_patches, cudaMemcpyHostToDevice, st));
        }
        reset_flags(c, st);
        {
            Stage sg(c, "generate", st, n_patches ? 2 : 1);
            launch_generate_bases(segs, n_segments, seed, pp, pb, n_patches, base0, n, out, c->d_err, st);
        }
        check_flags(c, st);
        AH_CUDA(cudaStreamSynchronize(st));
    });
}

ah_status ah_tm(ah_ctx *c, uint32_t set_id, const uint32_t *pair_ids, uint32_t n_pairs, const ah_site *sites,
                uint64_t n, float *tm_out, uint8_t *pass_out, void *stream)
{
    if (!c)
        return AH_ERR_ARG;
    return guarded(c, [&] {
        require_idle(c);
        require(n == 0 || (sites && tm_out), AH_ERR_ARG, "ah_tm: null argument");
        GenomeSet &gs = get_set(c, set_id);
        cudaStream_t st = stream_of(c, stream);
        wait_ready(gs, st);
        const PairDev *pd = upload_pairs(c, pair_ids, n_pairs, st);
        if (n == 0)
            return;
        reset_flags(c, st);
        const ah_site *s = stage_in(c, "tm_sites_in", sites, n, st);
        {
            Stage sg(c, "validate", st, 1);
            launch_validate_sites(s, n, pd, (int)n_pairs, gs.contig_off, gs.n_contigs, c->d_err, st);
        }
        check_flags(c, st);
        float *tm = out_buf(c, "tm_out", tm_out, n);
        uint8_t *ps = pass_out ? out_buf(c, "pass_out", pass_out, n) : nullptr;
        {
            Stage sg(c, "tm", st, 2);
            uint32_t *q = (uint32_t *)scratch(c, "tm_queue", 2 * n * sizeof(uint32_t));
            launch_tm(s, n, nullptr, pd, (int)n_pairs, gs.planes, gs.contig_off, tm, ps, q,
                      (uint32_t *)(c->d_flags + kFlagTmQueue), tm_seg_max(c),
                      tm_few_exact(c), c->d_err, st);
        }
        out_finish(tm_out, tm, n, st);
        if (pass_out)
            out_finish(pass_out, ps, n, st);
        check_flags(c, st);
    });
}

ah_status ah_pair(ah_ctx *c, uint32_t set_id, const uint32_t *pair_ids, uint32_t n_pairs, const ah_site *sites,
                  const uint8_t *pass, uint64_t n, ah_amplicon *out, uint64_t cap, uint64_t *n_out, void *stream)
{
    if (!c)
        return AH_ERR_ARG;
    return guarded(c, [&] {
        require_idle(c);
        require(n_out && (cap == 0 || out) && (n == 0 || sites), AH_ERR_ARG, "ah_pair: null argument");
        *n_out = 0;
        GenomeSet &gs = get_set(c, set_id);
        cudaStream_t st = stream_of(c, stream);
        wait_ready(gs, st);
        const PairDev *pd = upload_pairs(c, pair_ids, n_pairs, st);
        if (n == 0)
            return;
        reset_flags(c, st);
        const ah_site *s = stage_in(c, "pair_sites_in", sites, n, st);
        const uint8_t *ps = pass ? stage_in(c, "pair_pass_in", pass, n, st) : nullptr;
        {
            Stage sg(c, "validate", st, 1);
            launch_validate_sites(s, n, pd, (int)n_pairs, gs.contig_off, gs.n_contigs, c->d_err, st);
        }
        check_flags(c, st);
        uint64_t *counts = (uint64_t *)scratch(c, "pair_counts", n * sizeof(uint64_t));
        uint64_t *offs = (uint64_t *)scratch(c, "pair_offsets", n * sizeof(uint64_t));
        size_t tb = scan_u64_temp_bytes(n);
        void *temp = scratch(c, "scan_temp", tb);
        {
            Stage sg(c, "pair", st, 1 + scan_u64_launches(n));
            launch_pair_count(s, n, nullptr, ps, pd, counts, st);
            exclusive_scan_u64(temp, tb, counts, offs, n, st);
        }
        uint64_t last[2] = {0, 0};
        AH_CUDA(cudaMemcpyAsync(&last[0], offs + n - 1, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
        AH_CUDA(cudaMemcpyAsync(&last[1], counts + n - 1, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
        AH_CUDA(cudaStreamSynchronize(st));
        const uint64_t total = last[0] + last[1];
        *n_out = total;
        if (total > cap)
            throw Error(AH_ERR_OVERFLOW, "ah_pair: " + std::to_string(total) + " amplicons, capacity " +
                                             std::to_string(cap));
        if (total == 0)
            return;
        ah_amplicon *dst = out_buf(c, "amp_out", out, total);
        {
            Stage sg(c, "pair", st, 1);
            launch_pair_write(s, n, nullptr, ps, pd, offs, dst, total, nullptr, 0, st);
        }
        out_finish(out, dst, total, st);
        AH_CUDA(cudaStreamSynchronize(st));
    });
}

ah_status ah_fetch(ah_ctx *c, uint32_t set_id, const ah_amplicon *amplicons, uint64_t n, char *seq_out,
                   uint64_t cap, uint64_t *offsets_out, void *stream)
{
    if (!c)
        return AH_ERR_ARG;
    return guarded(c, [&] {
        require_idle(c);
        require(offsets_out && (n == 0 || amplicons) && (cap == 0 || seq_out), AH_ERR_ARG, "ah_fetch: null argument");
        GenomeSet &gs = get_set(c, set_id);
        cudaStream_t st = stream_of(c, stream);
        wait_ready(gs, st);
        reset_flags(c, st);
        const ah_amplicon *a = stage_in(c, "fetch_in", amplicons, n, st);
        uint64_t *len = (uint64_t *)scratch(c, "fetch_len", (n + 1) * sizeof(uint64_t));
        uint64_t *offs = out_buf(c, "fetch_offsets", offsets_out, n + 1);
        AH_CUDA(cudaMemsetAsync(len + n, 0, sizeof(uint64_t), st));
        size_t tb = scan_u64_temp_bytes(n + 1);
        void *temp = scratch(c, "scan_temp", tb);
        {
            Stage sg(c, "fetch", st, (n ? 1 : 0) + scan_u64_launches(n + 1));
            launch_fetch_lengths(a, n, nullptr, gs.contig_off, gs.n_contigs, len, c->d_err, st);
            exclusive_scan_u64(temp, tb, len, offs, n + 1, st);
        }
        check_flags(c, st);
        uint64_t total = 0;
        AH_CUDA(cudaMemcpyAsync(&total, offs + n, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
        out_finish(offsets_out, offs, n + 1, st);
        AH_CUDA(cudaStreamSynchronize(st));
        if (total > cap)
            throw Error(AH_ERR_OVERFLOW, "ah_fetch: " + std::to_string(total) + " bytes needed, capacity " +
                                             std::to_string(cap));
        if (total == 0)
            return;
        char *dst = out_buf(c, "fetch_out", seq_out, total);
        {
            Stage sg(c, "fetch", st, 1);
            launch_fetch(a, n, nullptr, offs, gs.planes, gs.contig_off, dst, nullptr, 0, st);
        }
        out_finish(seq_out, dst, total, st);
        AH_CUDA(cudaStreamSynchronize(st));
    });
}


ah_status ah_serve_start(ah_ctx *c, uint32_t set_id, const ah_serve_config *cfg, ah_server **out)
{
    if (!c)
        return AH_ERR_ARG;
    return guarded(c, [&] {
        require_idle(c);
        require(out && cfg && cfg->max_batch >= 1 && cfg->mem_budget > 0, AH_ERR_ARG, "ah_serve_start: bad argument");
        *out = nullptr;
        GenomeSet &gs = get_set(c, set_id);
        AH_CUDA(cudaStreamSynchronize(c->stream));
        auto S = std::make_unique<ah_server>();
        S->c = c;
        S->set_id = set_id;
        S->cfg = *cfg;
        const size_t G = (size_t)gs.max_genome + 1;
        S->genome_bases.assign(G, 0);
        S->genome_first.assign(G + 1, 0);
        for (uint32_t ci = 0; ci < gs.n_contigs; ++ci) {
            S->genome_bases[gs.contig_genome_h[ci]] += gs.contig_off_h[ci + 1] - gs.contig_off_h[ci];
            ++S->genome_first[gs.contig_genome_h[ci] + 1];
        }
        for (size_t g = 0; g < G; ++g)
            S->genome_first[g + 1] += S->genome_first[g];
        S->genome_contig.resize(gs.n_contigs);
        {
            std::vector<uint64_t> fill(S->genome_first.begin(), S->genome_first.end() - 1);
            for (uint32_t ci = 0; ci < gs.n_contigs; ++ci)
                S->genome_contig[fill[gs.contig_genome_h[ci]]++] = ci;
        }
        c->serving = true;
        S->worker = std::thread(serve_loop, S.get());
        *out = S.release();
    });
}

ah_status ah_serve_submit(ah_server *S, const ah_request *req, uint64_t *ticket_out)
{
    if (!S || !req || !ticket_out || (req->n_genomes && !req->genomes))
        return AH_ERR_ARG;
    if (req->k < 0 || req->k > AH_MAX_MISMATCHES)
        return AH_ERR_ARG;
    ServeReq r;
    r.genomes.assign(req->genomes, req->genomes + req->n_genomes);
    std::sort(r.genomes.begin(), r.genomes.end());
    r.genomes.erase(std::unique(r.genomes.begin(), r.genomes.end()), r.genomes.end());
    r.pair_id = req->pair_id;
    r.k = req->k;
    r.tm_filter = req->tm_filter;
    for (uint32_t g : r.genomes)
        if (g < S->genome_bases.size())
            r.bases += S->genome_bases[g];
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop || !S->c->pairs.count(req->pair_id))
            return AH_ERR_ARG;
        r.t_submit = S->now_ms();
        const uint64_t t = S->next_ticket++;
        S->reqs.emplace(t, std::move(r));
        S->queue.push_back(t);
        *ticket_out = t;
    }
    S->cv_work.notify_one();
    return AH_OK;
}

ah_status ah_serve_wait(ah_server *S, uint64_t ticket, ah_request_info *info, ah_site *sites_out, uint64_t sites_cap,
                        ah_amplicon *amps_out, uint64_t amps_cap, char *seq_out, uint64_t seq_cap,
                        uint64_t *seq_offsets_out)
{
    if (!S || !info)
        return AH_ERR_ARG;
    ServeReq r;
    {
        std::unique_lock<std::mutex> lk(S->mu);
        auto it = S->reqs.find(ticket);
        if (it == S->reqs.end())
            return AH_ERR_ARG;
        S->cv_done.wait(lk, [&] { return it->second.done; });
        const ServeReq &q = it->second;
        info->status = q.status;
        info->batch = q.batch;
        info->batch_size = q.batch_size;
        info->reserved = 0;
        info->n_sites = q.sites.size();
        info->n_amplicons = q.amps.size();
        info->n_seq = q.seq.size();
        info->bases = q.bases;
        info->submit_ms = q.t_submit;
        info->start_ms = q.t_start;
        info->done_ms = q.t_done;
        if (q.status == AH_OK) {
            if (q.sites.size() > sites_cap || q.amps.size() > amps_cap || (seq_offsets_out && q.seq.size() > seq_cap))
                return AH_ERR_OVERFLOW; // kept: ask again with room
            if ((!q.sites.empty() && !sites_out) || (!q.amps.empty() && !amps_out) ||
                (seq_offsets_out && !q.seq.empty() && !seq_out))
                return AH_ERR_ARG;
        }
        r = std::move(it->second); // released: the copies below run without the lock
        S->reqs.erase(it);
    }
    if (r.status != AH_OK)
        return r.status;
    if (!r.sites.empty())
        memcpy(sites_out, r.sites.data(), r.sites.size() * sizeof(ah_site));
    if (!r.amps.empty())
        memcpy(amps_out, r.amps.data(), r.amps.size() * sizeof(ah_amplicon));
    if (seq_offsets_out) {
        memcpy(seq_offsets_out, r.seq_off.data(), r.seq_off.size() * sizeof(uint64_t));
        if (!r.seq.empty())
            memcpy(seq_out, r.seq.data(), r.seq.size());
    }
    return AH_OK;
}

ah_status ah_serve_stop(ah_server *S)
{
    if (!S)
        return AH_ERR_ARG;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->worker.joinable())
        S->worker.join();
    S->c->serving = false;
    delete S;
    return AH_OK;
}


ah_status ah_hmm_build(ah_ctx *c, const char *seqs, const uint64_t *offsets, uint64_t n, uint32_t *hmm_id_out)
{
    if (!c)
        return AH_ERR_ARG;
    return guarded(c, [&] {
        require_idle(c);
        require(hmm_id_out && offsets && n >= 1, AH_ERR_ARG, "ah_hmm_build: null argument or no sequence");
        require(!is_device_ptr(c, offsets) && (offsets[n] == 0 || (seqs && !is_device_ptr(c, seqs))), AH_ERR_ARG,
                "ah_hmm_build: sequences and offsets are host arrays");
        require(offsets[0] == 0, AH_ERR_ARG, "ah_hmm_build: offsets must start at 0");
        for (uint64_t q = 0; q < n; ++q)
            require(offsets[q] <= offsets[q + 1], AH_ERR_ARG, "ah_hmm_build: offsets not monotone");
        HmmProfile p;
        build_profile(seqs, offsets, n, p);
        require(p.m >= 1 && p.m + 1 <= kHmmMaxColumns, AH_ERR_ARG,
                "ah_hmm_build: the reference must hold 1.." + std::to_string(kHmmMaxColumns - 1) + " letters");
        p.d_t = (float *)dev_alloc(c, p.t.size() * sizeof(float));
        p.d_e = (float *)dev_alloc(c, p.e.size() * sizeof(float));
        AH_CUDA(cudaMemcpyAsync(p.d_t, p.t.data(), p.t.size() * sizeof(float), cudaMemcpyHostToDevice, c->stream));
        AH_CUDA(cudaMemcpyAsync(p.d_e, p.e.data(), p.e.size() * sizeof(float), cudaMemcpyHostToDevice, c->stream));
        AH_CUDA(cudaStreamSynchronize(c->stream));
        const uint32_t id = c->next_hmm++;
        c->hmms[id] = std::move(p);
        *hmm_id_out = id;
    });
}

ah_status ah_hmm_tables(ah_ctx *c, uint32_t hmm_id, uint64_t *m_out, uint64_t *reference_out, float *t_out,
                        float *e_out)
{
    if (!c)
        return AH_ERR_ARG;
    return guarded(c, [&] {
        auto it = c->hmms.find(hmm_id);
        require(it != c->hmms.end(), AH_ERR_ARG, "ah_hmm_tables: unknown profile id");
        const HmmProfile &p = it->second;
        if (m_out)
            *m_out = (uint64_t)p.m;
        if (reference_out)
            *reference_out = p.reference;
        if (t_out)
            memcpy(t_out, p.t.data(), p.t.size() * sizeof(float));
        if (e_out)
            memcpy(e_out, p.e.data(), p.e.size() * sizeof(float));
    });
}

namespace {

// ah_hmm_score (Viterbi) and ah_hmm_forward (Forward): the same checks, grouping and launch
ah_status hmm_scores(ah_ctx *c, uint32_t set_id, uint32_t hmm_id, const ah_amplicon *amplicons, uint64_t n,
                     float *score_out, void *stream, bool forward)
{
    if (!c)
        return AH_ERR_ARG;
    return guarded(c, [&] {
        require_idle(c);
        require(n == 0 || (amplicons && score_out), AH_ERR_ARG, "ah_hmm_score: null argument");
        auto it = c->hmms.find(hmm_id);
        require(it != c->hmms.end(), AH_ERR_ARG, "ah_hmm_score: unknown profile id");
        const HmmProfile &p = it->second;
        GenomeSet &gs = get_set(c, set_id);
        if (n == 0)
            return;
        cudaStream_t st = stream_of(c, stream);
        wait_ready(gs, st);
        // the records on the host: bounds and the longest amplicon (shared memory of the kernel)
        std::vector<ah_amplicon> h(n);
        if (is_device_ptr(c, amplicons)) {
            AH_CUDA(cudaMemcpyAsync(h.data(), amplicons, n * sizeof(ah_amplicon), cudaMemcpyDeviceToHost, st));
            AH_CUDA(cudaStreamSynchronize(st));
        } else {
            memcpy(h.data(), amplicons, n * sizeof(ah_amplicon));
        }
        uint32_t max_len = 1;
        for (const ah_amplicon &a : h) {
            require(a.contig < gs.n_contigs && a.start <= a.end &&
                        (uint64_t)a.end <= gs.contig_off_h[a.contig + 1] - gs.contig_off_h[a.contig],
                    AH_ERR_ARG, "ah_hmm_score: an amplicon lies outside its contig");
            max_len = std::max(max_len, a.end - a.start);
        }
        require(max_len <= kHmmMaxLetters / 4, AH_ERR_ARG,
                "ah_hmm_score: amplicons longer than " + std::to_string(kHmmMaxLetters / 4) + " letters");
        require(n <= 0xffffffffull, AH_ERR_ARG, "ah_hmm_score: at most 2^32 - 1 amplicons per call");
        // amplicons of similar length side by side (the kernel scores several in lockstep)
        std::vector<uint32_t> ord(n);
        for (uint64_t q = 0; q < n; ++q)
            ord[q] = (uint32_t)q;
        std::stable_sort(ord.begin(), ord.end(), [&](uint32_t x, uint32_t y) {
            return h[x].end - h[x].start > h[y].end - h[y].start;
        });
        reset_flags(c, st);
        const ah_amplicon *a = stage_in(c, "hmm_in", amplicons, n, st);
        uint32_t *d_ord = (uint32_t *)scratch(c, "hmm_order", n * sizeof(uint32_t));
        AH_CUDA(cudaMemcpyAsync(d_ord, ord.data(), n * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
        float *out = out_buf(c, "hmm_out", score_out, n);
        if (hmm_use_wave(forward)) {
            float *bnd = (float *)scratch(c, "hmm_bnd", hmm_scratch_bytes(n, (int)max_len, c->sms));
            Stage sg(c, "hmm", st, 1);
            launch_hmm_wave(a, d_ord, n, gs.planes, gs.contig_off, gs.n_contigs, p.d_t, p.d_e, p.m, (int)max_len,
                            forward, bnd, out, c->d_err, c->sms, st);
        } else {
            Stage sg(c, "hmm", st, 1);
            launch_hmm_score(a, d_ord, n, gs.planes, gs.contig_off, gs.n_contigs, p.d_t, p.d_e, p.m, (int)max_len,
                             forward, out, c->d_err, c->sms, st);
        }
        check_flags(c, st);
        out_finish(score_out, out, n, st);
        AH_CUDA(cudaStreamSynchronize(st));
    });
}

} // namespace

ah_status ah_hmm_score(ah_ctx *c, uint32_t set_id, uint32_t hmm_id, const ah_amplicon *amplicons, uint64_t n,
                       float *score_out, void *stream)
{
    return hmm_scores(c, set_id, hmm_id, amplicons, n, score_out, stream, false);
}

ah_status ah_hmm_forward(ah_ctx *c, uint32_t set_id, uint32_t hmm_id, const ah_amplicon *amplicons, uint64_t n,
                         float *score_out, void *stream)
{
    return hmm_scores(c, set_id, hmm_id, amplicons, n, score_out, stream, true);
}

// Test aid (not in the public header).  on != 0: in later scans the first
// slice of every warp is armed on its barrier with no copy behind it (a wait
// that nothing will end) and the per-slice wait limit is 20 us, so the scan
// takes its timeout path -- error word, bounded wait for the warp's copies
// still in flight, exit -- and the call returns AH_ERR_TIMEOUT.  Nothing
// faults or hangs.  on == 0 restores normal scans.
ah_status ah_debug_scan_stall(ah_ctx *c, int on)
{
    if (!c)
        return AH_ERR_ARG;
    c->scan_stall_first = on != 0;
    return AH_OK;
}

ah_status ah_hmm_free(ah_ctx *c, uint32_t hmm_id)
{
    if (!c)
        return AH_ERR_ARG;
    return guarded(c, [&] {
        require_idle(c);
        auto it = c->hmms.find(hmm_id);
        require(it != c->hmms.end(), AH_ERR_ARG, "ah_hmm_free: unknown profile id");
        AH_CUDA(cudaStreamSynchronize(c->stream));
        dev_free(c, it->second.d_t, 0);
        dev_free(c, it->second.d_e, 0);
        c->hmms.erase(it);
    });
}

} // extern "C"
