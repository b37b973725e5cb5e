// Scan kernel generator (primer matching, Sec. 2.1) and its run-time compiler.
//
// Why generate: the mismatch count of a window against a degenerate primer is
// a sum of L one-bit terms, and on this GPU its cost is set by integer issue
// slots.  With the primer's IUPAC codes known when the kernel is compiled,
// the match word of a single-base position is a plane word itself (0 ops), a
// two- or three-base position is a sum of disjoint plane words (integer adds,
// which do not use the logic pipe), and the count runs through a carry-save
// network whose shape depends on L and k.  So each set of patterns gets its
// own straight-line kernel, built here as CUDA source and compiled with NVRTC
// for sm_103a; compiled kernels are cached per process.
//
// Bit-sliced counting.  A thread owns R consecutive words of a tile; word j
// holds starts p = b * W + j for b = 0..31 (tile-strided layout), so the
// window base at offset i of all 32 starts is word j + i.  For each pattern
// and word the kernel forms the L match words M_i (bit b = 1 when the base at
// p_b + i is in the pattern's set) and reduces them column by column with
// full adders.  It works in the "match" domain: a full adder on match words
// yields the complements of the sum and carry of the mismatch bits, so no
// inversion is ever needed, and padding uses all-ones words (a match).  With
// K2 the smallest power of two above k, columns of weight < K2 are reduced
// to one bit each; a mismatch count >= K2 shows as a zero bit in any carry
// word of weight K2, so those are AND-ed; the low bits are compared with k by
// one or two LOP3s.  Full adders are either two LOP3s (xor3, majority) or one
// majority LOP3 plus integer adds for the sum (s = a + b + c - 2 maj), a mix
// chosen by the tuner to balance the logic and integer pipes.
//
// A warp with any hit runs a slower path in rounds, one hit per lane per
// round: each lane checks its hit against the contig table (windows never
// cross a contig end; the search is confined to the contigs of the tile by a
// per-tile table), recounts its mismatches exactly from shared memory (a
// device check that the network agrees) and applies the 3' clamp; the warp
// appends the surviving 64-bit keys with one atomic per round.  Key =
// ((pair << pbits | flat position) << 10) | primer << 9 | strand << 8 | mm,
// so sorting keys gives the canonical site order.
#include <nvrtc.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <sstream>

#include "ah_internal.h"

namespace ah {
namespace {

const char *kPrelude = R"CUDA(
typedef unsigned int u32;
typedef unsigned long long u64;
typedef unsigned char u8;
template <int IMM> __device__ __forceinline__ u32 lop3(u32 a, u32 b, u32 c)
{
    u32 d;
    asm("lop3.b32 %0, %1, %2, %3, %4;" : "=r"(d) : "r"(a), "r"(b), "r"(c), "n"(IMM));
    return d;
}
__device__ __forceinline__ u32 smem_addr(const void *p) { return (u32)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(u64 *bar, u32 count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
// one thread: start a bulk copy (TMA) whose bytes complete on `bar`; the
// generic-proxy reads of the buffer are ordered before the async write
__device__ __forceinline__ void tma_copy(void *dst, const void *src, u32 bytes, u64 *bar)
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try(u64 *bar, u32 parity)
{
    u32 ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok) : "r"(smem_addr(bar)), "r"(parity) : "memory");
    return ok != 0;
}
__device__ __forceinline__ u64 global_ns()
{
    u64 t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
// bounded wait for a barrier phase: gives up after ~2 s instead of hanging
__device__ __forceinline__ bool mbar_wait(u64 *bar, u32 parity)
{
    if (mbar_try(bar, parity))
        return true;
    const u64 t0 = global_ns();
    while (!mbar_try(bar, parity))
        if (global_ns() - t0 > 2000000000ull)
            return false;
    return true;
}
)CUDA";

// Body of the kernel after the generated hit words.  Uses: h[NPAT*R] (hit
// words), any, lane, sm (the warp's slice planes, stride SLW), tile, wbase
// (first tile word of the slice), j0 (the thread's first slice word) and the
// pattern tables.
const char *kEmit = R"CUDA(
    if (__any_sync(0xffffffffu, any != 0u)) {
        // Hits, one per lane per round: every lane takes its next hit bit, all
        // check theirs at once (contig end, exact recount, clamp), and the warp
        // appends the survivors with one atomic per round.
        u32 hl[NPAT * R];
#pragma unroll
        for (int i = 0; i < NPAT * R; ++i) hl[i] = h[i];
        // the contigs this tile's starts can fall in: [clo, chi)
        const u32 clo = tile_contig[tile];
        const u32 chi = min(n_contigs, tile_contig[tile + 1] + 1u);
        int qr = 0;
        u32 m = hl[0];
        for (;;) {
            while (m == 0u && qr + 1 < NPAT * R) m = hl[++qr];
            const bool have = m != 0u;
            if (!__any_sync(0xffffffffu, have)) break;
            bool valid = false;
            u64 key = 0;
            if (have) {
                const int b = __ffs(m) - 1;
                m &= m - 1;
                const int q = qr / R, r = qr % R;
                const int jr = j0 + r;
                const u64 P = tile * TB + (u64)b * W + wbase + jr;
                const int L = c_L[q];
                u32 lo = clo, hi = chi;
                while (hi - lo > 1) {
                    u32 mid = (lo + hi) >> 1;
                    if (contig_off[mid] <= P) lo = mid; else hi = mid;
                }
                if (P + L <= contig_off[lo + 1]) {
                    int mm = 0, clamp_bad = 0;
                    const int c = c_clamp[q];
                    for (int i = 0; i < L; ++i) {
                        const int wj = jr + i;
                        const u32 code = ((sm[wj] >> b) & 1u) | (((sm[SLW + wj] >> b) & 1u) << 1) |
                                         (((sm[2 * SLW + wj] >> b) & 1u) << 2) | (((sm[3 * SLW + wj] >> b) & 1u) << 3);
                        const int mis = (code & c_mask[q][i]) == 0u;
                        mm += mis;
                        const int in_clamp = c_strand[q] == 0 ? (i >= L - c) : (i < c);
                        clamp_bad |= mis & in_clamp;
                    }
                    if (mm > c_k[q]) atomicExch(err, 3); // the network disagrees with the recount
                    else if (!clamp_bad) {
                        valid = true;
                        key = ((((u64)c_pair[q] << pbits) | P) << 10) | ((u64)c_primer[q] << 9) |
                              ((u64)c_strand[q] << 8) | (u64)mm;
                    }
                }
            }
            const u32 vb = __ballot_sync(0xffffffffu, valid);
            if (vb) {
                u64 base = 0;
                if (lane == 0) base = atomicAdd(counter, (u64)__popc(vb));
                base = __shfl_sync(0xffffffffu, base, 0);
                const u64 idx = base + __popc(vb & ((1u << lane) - 1u));
                if (valid && idx < cap) keys[idx] = key;
            }
        }
    }
)CUDA";

struct Gen {
    std::ostringstream os;
    int n = 0;
    int fa_total = 0, fa_arith = 0;
    int arith_pct = 0;

    std::string tmp() { return "v" + std::to_string(n++); }
    std::string lop(const std::string &a, const std::string &b, const std::string &c, int imm)
    {
        std::string v = tmp();
        os << "    const u32 " << v << " = lop3<0x" << std::hex << imm << std::dec << ">(" << a << ", " << b << ", "
           << c << ");\n";
        return v;
    }
    // full adder on match-domain words -> (sum, carry)
    void fa(const std::string &a, const std::string &b, const std::string &c, std::string &s, std::string &cy)
    {
        ++fa_total;
        cy = lop(a, b, c, 0xE8);
        // Bresenham-style spread of the arithmetic full adders
        bool arith = (fa_arith * 100 < arith_pct * fa_total);
        if (arith) {
            ++fa_arith;
            s = tmp();
            os << "    const u32 " << s << " = " << a << " + " << b << " + " << c << " - " << cy << " - " << cy
               << ";\n";
        } else {
            s = lop(a, b, c, 0x96);
        }
    }
};

int popc4(int m) { return (m & 1) + ((m >> 1) & 1) + ((m >> 2) & 1) + ((m >> 3) & 1); }

// match word of an IUPAC mask at window index w
std::string match_word(Gen &g, int mask, int w, std::map<std::pair<int, int>, std::string> &cache)
{
    auto key = std::make_pair(mask, w);
    auto it = cache.find(key);
    if (it != cache.end())
        return it->second;
    static const char *P[4] = {"pA", "pC", "pG", "pT"};
    std::string r;
    int n = popc4(mask);
    if (n == 4) {
        r = "pV[" + std::to_string(w) + "]";
    } else if (n == 1) {
        for (int x = 0; x < 4; ++x)
            if (mask & (1 << x))
                r = std::string(P[x]) + "[" + std::to_string(w) + "]";
    } else {
        r = g.tmp();
        g.os << "    const u32 " << r << " = ";
        bool first = true;
        for (int x = 0; x < 4; ++x)
            if (mask & (1 << x)) {
                g.os << (first ? "" : " + ") << P[x] << "[" << w << "]";
                first = false;
            }
        g.os << ";\n";
    }
    cache[key] = r;
    return r;
}

// LOP3 immediate of f over (a, b, c): bit index (a << 2) | (b << 1) | c.
template <class F> int lut3(F f)
{
    int imm = 0;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            for (int c = 0; c < 2; ++c)
                if (f(a, b, c))
                    imm |= 1 << ((a << 2) | (b << 1) | c);
    return imm;
}

std::string and_reduce(Gen &g, std::deque<std::string> v)
{
    if (v.empty())
        return "0xffffffffu";
    while (v.size() > 1) {
        std::string a = v.front();
        v.pop_front();
        std::string b = v.front();
        v.pop_front();
        std::string c = "0xffffffffu";
        if (!v.empty()) {
            c = v.front();
            v.pop_front();
        }
        v.push_back(g.lop(a, b, c, 0x80));
    }
    return v.front();
}

// Hit word of pattern p for the thread's word r: bit b set iff the window at
// start p_b has <= k mismatches.
std::string gen_hit(Gen &g, const ScanPattern &p, int r, std::map<std::pair<int, int>, std::string> &cache)
{
    if (p.k >= p.L)
        return "0xffffffffu";
    int klog = 0;
    while ((1 << klog) <= p.k)
        ++klog; // K2 = 2^klog > k
    std::deque<std::string> col[6];
    for (int i = 0; i < p.L; ++i)
        col[0].push_back(match_word(g, p.mask[i], r + i, cache));
    for (int w = 0; w < klog; ++w) {
        while (col[w].size() > 1) {
            std::string a = col[w].front();
            col[w].pop_front();
            std::string b = col[w].front();
            col[w].pop_front();
            std::string c = "0xffffffffu";
            if (!col[w].empty()) {
                c = col[w].front();
                col[w].pop_front();
            }
            std::string s, cy;
            g.fa(a, b, c, s, cy);
            col[w].push_back(s);
            col[w + 1].push_back(cy);
        }
    }
    std::string hi = and_reduce(g, col[klog]);
    if (p.k == (1 << klog) - 1)
        return hi;
    // low part: match-domain bits s_w (mismatch bit = ~s_w), value v = sum 2^w (1 - s_w) <= k
    std::string s[4];
    for (int w = 0; w < klog; ++w)
        s[w] = col[w].empty() ? std::string("0xffffffffu") : col[w].front();
    const int k = p.k;
    if (klog == 2) { // k == 2 (k == 3 handled above)
        int imm = lut3([&](int a, int b, int c) { return a && ((1 - b) + 2 * (1 - c) <= k); });
        return g.lop(hi, s[0], s[1], imm);
    }
    if (klog == 3) { // k in 4..6
        int imm = lut3([&](int a, int b, int c) { return ((1 - a) + 2 * (1 - b) + 4 * (1 - c)) <= k; });
        std::string lo = g.lop(s[0], s[1], s[2], imm);
        return g.lop(hi, lo, "0xffffffffu", 0x80);
    }
    // klog == 4, k in 8..10: v = low3 + 8 (1 - s3); low3 <= 7 <= k, so v <= k iff s3 or low3 <= k - 8
    int imm = lut3([&](int a, int b, int c) { return ((1 - a) + 2 * (1 - b) + 4 * (1 - c)) <= k - 8; });
    std::string lo = g.lop(s[0], s[1], s[2], imm);
    int imm2 = lut3([](int a, int b, int c) { return a && (b || c); });
    return g.lop(hi, s[3], lo, imm2);
}

} // namespace

std::string scan_source(const std::vector<ScanPattern> &pats, const ScanTuning &t)
{
    const int npat = (int)pats.size();
    int Lmax = 1;
    for (auto &p : pats)
        Lmax = std::max(Lmax, p.L);
    const int R = t.R;
    if (R != 4 && R != 8) // the loader reads 16-byte vectors at word lane * R of the slice
        throw Error(AH_ERR_ARG, "scan kernel: R must be 4 or 8");
    const int nwin = 4 * ((R + Lmax - 1 + 3) / 4);
    const int NT = 32 * t.warps;
    Gen g;
    g.arith_pct = t.arith_pct;
    std::ostringstream &os = g.os;
    os << kPrelude;
    os << "#define W " << kTileW << "\n#define WX " << kTileWX << "\n#define TB " << kTileBases << "ull\n";
    os << "#define R " << R << "\n#define NPAT " << npat << "\n#define NWIN " << nwin << "\n#define NT " << NT
       << "\n";
    auto table = [&](const char *name, auto get) {
        os << "__device__ const u8 " << name << "[" << npat << "] = {";
        for (int q = 0; q < npat; ++q)
            os << (q ? ", " : "") << get(pats[q]);
        os << "};\n";
    };
    table("c_L", [](const ScanPattern &p) { return p.L; });
    table("c_k", [](const ScanPattern &p) { return p.k; });
    table("c_clamp", [](const ScanPattern &p) { return p.clamp; });
    table("c_pair", [](const ScanPattern &p) { return p.pair; });
    table("c_primer", [](const ScanPattern &p) { return p.primer; });
    table("c_strand", [](const ScanPattern &p) { return p.strand; });
    os << "__device__ const u8 c_mask[" << npat << "][32] = {";
    for (int q = 0; q < npat; ++q) {
        os << (q ? ", " : "") << "{";
        for (int i = 0; i < 32; ++i)
            os << (i ? "," : "") << (i < pats[q].L ? (int)pats[q].mask[i] : 15);
        os << "}";
    }
    os << "};\n";
    os << "#define S " << t.stages << "\n#define WPC " << t.warps << "\n#define SLICES (W / (32 * R))\n"
       << "#define SLW (32 * R + 32)\n";
    os << "extern \"C\" __global__ void __launch_bounds__(NT, " << t.min_blocks << ")\n"
       << "ah_scan_kernel(const u32 *__restrict__ planes, u64 n_tiles, const u64 *__restrict__ contig_off,\n"
       << "               u32 n_contigs, u64 *__restrict__ keys, u64 cap, u64 *__restrict__ counter, int pbits,\n"
       << "               int *__restrict__ err, u64 *__restrict__ work, const u64 *__restrict__ tile_list,\n"
       << "               const u32 *__restrict__ tile_contig)\n{\n"
       << "  // Every warp claims slices of tiles (32*R words of each plane plus a 32-word\n"
       << "  // overhang) from the shared counter `work` (zeroed before the launch), so SMs\n"
       << "  // that run faster take more, and runs its own S-stage pipeline: lane 0 claims\n"
       << "  // and starts bulk async copies (TMA) into the warp's buffers, one mbarrier\n"
       << "  // per stage; no CTA-wide barrier is ever taken.  A warp's claims only grow,\n"
       << "  // so the first claim past the end means that none of its stages holds work.\n"
       << "  // With tile_list, the n_tiles tiles scanned are tile_list[0 .. n_tiles).\n"
       << "  extern __shared__ __align__(128) u32 smbuf[];\n"
       << "  __shared__ __align__(8) u64 bars[WPC * S];\n"
       << "  __shared__ u64 claims[WPC * S];\n"
       << "  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;\n"
       << "  u32 *wbuf = smbuf + warp * (S * 4 * SLW);\n"
       << "  u64 *wbar = bars + warp * S;\n"
       << "  u64 *witem = claims + warp * S;\n"
       << "  const u64 n_items = n_tiles * SLICES;\n"
       << "  if (lane == 0) {\n"
       << "    for (int q = 0; q < S; ++q) mbar_init(&wbar[q], 1);\n"
       << "    asm volatile(\"fence.mbarrier_init.release.cluster;\" ::: \"memory\");\n"
       << "  }\n"
       << "  __syncwarp();\n"
       << "  auto issue = [&](u64 wi, int stg) {\n"
       << "    const u64 tl = tile_list ? tile_list[wi / SLICES] : wi / SLICES;\n"
       << "    const int sl = (int)(wi % SLICES);\n"
       << "    asm volatile(\"mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\" ::\"r\"(smem_addr(&wbar[stg])),\n"
       << "                 \"r\"((u32)(4 * SLW * 4)) : \"memory\");\n"
       << "    for (int x = 0; x < 4; ++x)\n"
       << "      tma_copy(wbuf + (stg * 4 + x) * SLW, planes + (tl * 4 + x) * WX + sl * 32 * R, SLW * 4, &wbar[stg]);\n"
       << "  };\n"
       << "  if (lane == 0)\n"
       << "    for (int q = 0; q < S; ++q) {\n"
       << "      const u64 w = atomicAdd(work, 1ull);\n"
       << "      witem[q] = w;\n"
       << "      if (w < n_items) issue(w, q);\n"
       << "    }\n"
       << "  __syncwarp();\n"
       << "  for (int k = 0;; ++k) {\n"
       << "    const int stg = k % S;\n"
       << "    const u64 wi = witem[stg];\n"
       << "    if (wi >= n_items)\n"
       << "      break;\n"
       << "    const bool ok = mbar_wait(&wbar[stg], (u32)((k / S) & 1));\n"
       << "    if (!__all_sync(0xffffffffu, ok)) {\n"
       << "      // a copy never landed: report, wait (bounded) for the copies still in flight, leave\n"
       << "      if (lane == 0) {\n"
       << "        atomicExch(err, 1);\n"
       << "        for (int d = 1; d < S; ++d)\n"
       << "          if (witem[(k + d) % S] < n_items) mbar_wait(&wbar[(k + d) % S], (u32)(((k + d) / S) & 1));\n"
       << "      }\n"
       << "      break;\n"
       << "    }\n"
       << "    const u64 tile = tile_list ? tile_list[wi / SLICES] : wi / SLICES;\n"
       << "    const int wbase = (int)(wi % SLICES) * 32 * R;\n"
       << "    const u32 *sm = wbuf + stg * 4 * SLW;\n"
       << "    const int j0 = lane * R;\n"
       << "    u32 pA[NWIN], pC[NWIN], pG[NWIN], pT[NWIN], pV[NWIN];\n"
       << "#pragma unroll\n"
       << "    for (int c = 0; c < NWIN / 4; ++c) {\n"
       << "      uint4 a = reinterpret_cast<const uint4 *>(sm + 0 * SLW + j0)[c];\n"
       << "      uint4 cc = reinterpret_cast<const uint4 *>(sm + 1 * SLW + j0)[c];\n"
       << "      uint4 gg = reinterpret_cast<const uint4 *>(sm + 2 * SLW + j0)[c];\n"
       << "      uint4 tt = reinterpret_cast<const uint4 *>(sm + 3 * SLW + j0)[c];\n"
       << "      pA[4*c] = a.x; pA[4*c+1] = a.y; pA[4*c+2] = a.z; pA[4*c+3] = a.w;\n"
       << "      pC[4*c] = cc.x; pC[4*c+1] = cc.y; pC[4*c+2] = cc.z; pC[4*c+3] = cc.w;\n"
       << "      pG[4*c] = gg.x; pG[4*c+1] = gg.y; pG[4*c+2] = gg.z; pG[4*c+3] = gg.w;\n"
       << "      pT[4*c] = tt.x; pT[4*c+1] = tt.y; pT[4*c+2] = tt.z; pT[4*c+3] = tt.w;\n"
       << "    }\n"
       << "#pragma unroll\n"
       << "    for (int w = 0; w < NWIN; ++w) pV[w] = pA[w] + pC[w] + pG[w] + pT[w];\n"
       << "    u32 h[NPAT * R];\n"
       << "    u32 any = 0;\n";
    std::map<std::pair<int, int>, std::string> cache;
    auto one = [&](int q, int r) {
        os << "    // pattern " << q << ", word " << r << "\n";
        std::string hw = gen_hit(g, pats[q], r, cache);
        os << "    h[" << q * R + r << "] = " << hw << ";\n    any |= h[" << q * R + r << "];\n";
    };
    if (t.order == 0) {
        for (int r = 0; r < R; ++r)
            for (int q = 0; q < npat; ++q)
                one(q, r);
    } else {
        for (int q = 0; q < npat; ++q)
            for (int r = 0; r < R; ++r)
                one(q, r);
    }
    os << kEmit;
    os << "    __syncwarp();\n"
       << "    if (lane == 0) { // refill this stage with the next claim\n"
       << "      const u64 w = atomicAdd(work, 1ull);\n"
       << "      witem[stg] = w;\n"
       << "      if (w < n_items) issue(w, stg);\n"
       << "    }\n"
       << "    __syncwarp();\n"
       << "  }\n}\n";
    return os.str();
}

namespace {
std::mutex g_mu;
std::map<std::string, std::unique_ptr<ScanKernel>> g_cache; // key: device + source

std::string nvrtc_err(nvrtcResult r) { return nvrtcGetErrorString(r); }
} // namespace

namespace {
std::string compile_cubin(const std::string &src, std::vector<char> *cubin, bool *ok)
{
    nvrtcProgram prog;
    nvrtcResult r = nvrtcCreateProgram(&prog, src.c_str(), "ah_scan_generated.cu", 0, nullptr, nullptr);
    if (r != NVRTC_SUCCESS)
        throw Error(AH_ERR_JIT, "nvrtcCreateProgram: " + nvrtc_err(r));
    const char *opts[] = {"-arch=sm_103a", "-std=c++17", "-lineinfo", "--ptxas-options=-v", "-DNDEBUG"};
    r = nvrtcCompileProgram(prog, 5, opts);
    size_t log_size = 0;
    nvrtcGetProgramLogSize(prog, &log_size);
    std::string log(log_size, '\0');
    if (log_size)
        nvrtcGetProgramLog(prog, &log[0]);
    *ok = (r == NVRTC_SUCCESS);
    if (*ok && cubin) {
        size_t cubin_size = 0;
        nvrtcGetCUBINSize(prog, &cubin_size);
        cubin->resize(cubin_size);
        nvrtcGetCUBIN(prog, cubin->data());
    }
    nvrtcDestroyProgram(&prog);
    return log;
}
} // namespace

std::string scan_compile_only(const std::vector<ScanPattern> &pats, const ScanTuning &t, bool *ok)
{
    return compile_cubin(scan_source(pats, t), nullptr, ok);
}

ScanKernel *scan_kernel(const std::vector<ScanPattern> &pats, const ScanTuning &t, int device)
{
    // cache key: device, tuning and the patterns (cheap; the source is only generated on a miss)
    std::string key = std::to_string(device) + "|" + std::to_string(t.R) + "," + std::to_string(t.arith_pct) + "," +
                      std::to_string(t.min_blocks) + "," + std::to_string(t.order) + "," + std::to_string(t.stages) +
                      "," + std::to_string(t.warps) + "," + std::to_string(t.resident) + "|";
    for (auto &p : pats) {
        key += std::to_string(p.L) + "," + std::to_string(p.k) + "," + std::to_string(p.clamp) + "," +
               std::to_string(p.pair) + "," + std::to_string(p.primer) + "," + std::to_string(p.strand) + ":";
        for (int i = 0; i < p.L; ++i)
            key += (char)('a' + p.mask[i]);
        key += ";";
    }
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_cache.find(key);
    if (it != g_cache.end())
        return it->second.get();
    const std::string src = scan_source(pats, t);
    bool ok = false;
    std::vector<char> cubin;
    std::string log = compile_cubin(src, &cubin, &ok);
    if (!ok)
        throw Error(AH_ERR_JIT, "scan kernel compilation failed: " + log.substr(0, 2000));

    auto k = std::make_unique<ScanKernel>();
    k->log = log;
    AH_CUDA(cudaLibraryLoadData(&k->lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0));
    AH_CUDA(cudaLibraryGetKernel(&k->fn, k->lib, "ah_scan_kernel"));
    k->threads = 32 * t.warps;
    k->smem = (size_t)t.warps * t.stages * 4 * (32 * t.R + 32) * sizeof(uint32_t); // per-warp stage buffers
    if (k->smem > 48 * 1024)
        AH_CUDA(cudaKernelSetAttributeForDevice(k->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k->smem,
                                                device));
    auto pos = log.find("Used ");
    if (pos != std::string::npos)
        k->regs = atoi(log.c_str() + pos + 5);
    int bps = 0;
    AH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, (const void *)k->fn, k->threads, k->smem));
    k->blocks_per_sm = std::max(1, bps);
    if (t.resident > 0)
        k->blocks_per_sm = std::min(k->blocks_per_sm, t.resident);
    ScanKernel *raw = k.get();
    g_cache[key] = std::move(k);
    return raw;
}

} // namespace ah

// Generate and compile (no GPU needed) the scan kernel of one primer pair;
// writes the NVRTC/ptxas log (register use) into log[0..log_cap).  Returns 0
// on success.  A development aid; not part of the public header.
static int debug_scan(const char *fwd, const char *rev, int k, int R, int arith_pct, int order, char *log,
                      size_t log_cap, bool compile)
{
    try {
        std::vector<ah::ScanPattern> pats;
        const char *pr[2] = {fwd, rev};
        for (int primer = 0; primer < 2; ++primer)
            for (int strand = 0; strand < 2; ++strand) {
                ah::ScanPattern p;
                p.L = (int)strlen(pr[primer]);
                if (p.L < 1 || p.L > AH_MAX_PRIMER_LEN)
                    return 2;
                p.k = k;
                p.primer = primer;
                p.strand = strand;
                for (int i = 0; i < p.L; ++i) {
                    int m = strand == 0 ? ah::iupac_mask(pr[primer][i]) : ah::comp_mask(ah::iupac_mask(pr[primer][p.L - 1 - i]));
                    if (!m)
                        return 2;
                    p.mask[i] = (uint8_t)m;
                }
                pats.push_back(p);
            }
        ah::ScanTuning t; // no register cap: the log reports the generator's own register use
        t.R = R;
        t.arith_pct = arith_pct;
        t.order = order;
        t.warps = 4;
        t.min_blocks = 1;
        bool ok = false;
        std::string l = compile ? ah::scan_compile_only(pats, t, &ok) : ah::scan_source(pats, t);
        if (!compile)
            ok = true;
        if (log && log_cap) {
            size_t n = std::min(log_cap - 1, l.size());
            memcpy(log, l.data(), n);
            log[n] = 0;
        }
        return ok ? 0 : 1;
    } catch (const std::exception &e) {
        if (log && log_cap)
            snprintf(log, log_cap, "%s", e.what());
        return 3;
    }
}

extern "C" int ah_debug_compile_scan(const char *fwd, const char *rev, int k, int R, int arith_pct, int order,
                                     char *log, size_t log_cap)
{
    return debug_scan(fwd, rev, k, R, arith_pct, order, log, log_cap, true);
}

// The generated source of one pair's scan kernel (development aid).
extern "C" int ah_debug_scan_source(const char *fwd, const char *rev, int k, int R, int arith_pct, int order,
                                    char *out, size_t cap)
{
    return debug_scan(fwd, rev, k, R, arith_pct, order, out, cap, false);
}
