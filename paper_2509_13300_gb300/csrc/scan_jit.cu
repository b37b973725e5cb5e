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
// Hits.  The network's hit words of the patterns of one primer pair are
// OR-ed into one word per pair and thread word (few live registers however
// many patterns one launch scans).  A warp with any hit visits the hit
// starts together: the lanes that hold hits publish their words to shared
// memory one lane at a time, and for each hit start the warp gathers the 32
// window bases as four ballots of the plane bits (bit i = base at window
// position i), so that every pattern of the pair is re-counted exactly by
// warp-uniform AND/OR/popc against per-pattern position masks (the network
// only filters; the recount yields the mismatch count and the 3' clamp test,
// and a network hit that no pattern confirms is reported as a device-check
// error).  Windows never cross a contig end: a hit within the first contig
// of its tile takes that contig's end from a per-tile table loaded while the
// network runs; any other takes it from a cooperative search of the tile's
// contigs (one load per lane, cached per warp).  Surviving keys collect in a per-warp stash in shared memory and
// are appended 32 at a time with one atomic (the rest when the warp ends).
// Key = ((pair << pbits | flat position) << 10) | primer << 9 | strand << 8
// | mm, so sorting keys gives the canonical site order.
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
__device__ __forceinline__ bool mbar_test(u64 *bar, u32 parity)
{
    u32 ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok) : "r"(smem_addr(bar)), "r"(parity) : "memory");
    return ok != 0;
}
// bounded wait for a barrier phase: gives up after limit_ns instead of hanging.
// Limits of a millisecond and more poll with try_wait (the thread may be
// suspended between tests); shorter ones poll with the non-blocking test, so
// that the limit itself decides.
__device__ __forceinline__ bool mbar_wait(u64 *bar, u32 parity, u64 limit_ns)
{
    if (mbar_test(bar, parity))
        return true;
    const u64 t0 = global_ns();
    if (limit_ns >= 1000000ull) {
        while (!mbar_try(bar, parity))
            if (global_ns() - t0 > limit_ns)
                return false;
    } else {
        while (!mbar_test(bar, parity))
            if (global_ns() - t0 > limit_ns)
                return false;
    }
    return true;
}
)CUDA";

// Body of the kernel after the generated hit words.  Uses: hg[NGRP*R] (hit
// words per pattern group and thread word), any, lane, warp, sm (the warp's
// slice planes, stride SLW), tile, wbase and the per-warp state in shared
// memory (hsbuf, stash, w_nv, w_cs, w_ce); @VISIT@ is replaced by the cases of
// the pattern groups.
const char *kEmit = R"CUDA(
    if (__any_sync(0xffffffffu, any != 0u)) {
        u32 *hs = hsbuf + warp * HSW;
        u32 nzw[NZW]; // bit i: hg[i] != 0
#pragma unroll
        for (int z = 0; z < NZW; ++z) nzw[z] = 0u;
#pragma unroll
        for (int i = 0; i < NGRP * R; ++i) nzw[i >> 5] |= (hg[i] != 0u ? 1u : 0u) << (i & 31);
        u32 nv = w_nv[warp];
        u64 cs = w_cs[warp], ce = w_ce[warp];
        u32 lanes = __ballot_sync(0xffffffffu, any != 0u);
        while (lanes) {
            const int src = __ffs(lanes) - 1;
            lanes &= lanes - 1;
            if (lane == src) {
#pragma unroll
                for (int i = 0; i < NGRP * R; ++i) hs[i] = hg[i];
#pragma unroll
                for (int z = 0; z < NZW; ++z) hs[NGRP * R + z] = nzw[z];
            }
            __syncwarp();
            for (int z = 0; z < NZW; ++z) {
                u32 nz = hs[NGRP * R + z];
                while (nz) {
                    const int i = z * 32 + __ffs(nz) - 1;
                    nz &= nz - 1;
                    const int g = i / R;
                    const int jr = src * R + i % R; // slice word of the starts
                    u32 m = hs[i];
                    while (m) {
                        const int b = __ffs(m) - 1;
                        m &= m - 1;
                        const u64 P = tile * TB + (u64)b * W + wbase + jr;
                        // window bases, bit i = base at position i of the window
                        const u32 cA = __ballot_sync(0xffffffffu, (sm[jr + lane] >> b) & 1u);
                        const u32 cC = __ballot_sync(0xffffffffu, (sm[SLW + jr + lane] >> b) & 1u);
                        const u32 cG = __ballot_sync(0xffffffffu, (sm[2 * SLW + jr + lane] >> b) & 1u);
                        const u32 cT = __ballot_sync(0xffffffffu, (sm[3 * SLW + jr + lane] >> b) & 1u);
                        // end (flat) of the contig holding P: the tile's first contig when P lies
                        // within `room` of the tile's start, else the first contig end above P
                        // among the tile's contigs [clo, chi) (cached per warp)
                        const u32 o = (u32)(b * W + wbase + jr);
                        if (o >= room && (P < cs || P >= ce)) {
                            const u32 clo = tile_contig[tile];
                            const u32 chi = min(n_contigs, tile_contig[tile + 1] + 1u);
                            cs = 0;
                            ce = 0;
                            for (u32 x0 = clo + 1u; x0 <= chi; x0 += 32u) {
                                const u32 x = x0 + (u32)lane;
                                const bool in = x <= chi;
                                const u64 e = in ? contig_off[x] : 0ull;
                                const u32 f = __ballot_sync(0xffffffffu, in && e > P);
                                if (f) {
                                    const int fl = __ffs(f) - 1;
                                    ce = __shfl_sync(0xffffffffu, e, fl);
                                    cs = contig_off[x0 + fl - 1u];
                                    break;
                                }
                            }
                        }
                        const u64 cend = o < room ? tile * TB + room : ce;
                        bool some = false;
                        // exact count of every pattern of the group (masks compiled in)
                        switch (g) {
@VISIT@                        }
                        if (!some && lane == 0)
                            atomicExch(err, 3); // the network disagrees with the exact count
                    }
                }
            }
            __syncwarp();
        }
        w_nv[warp] = nv;
        w_cs[warp] = cs;
        w_ce[warp] = ce;
        __syncwarp();
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
    // pattern groups: runs of consecutive patterns of one primer pair
    std::vector<int> g0;
    std::vector<int> group_of(npat);
    for (int q = 0; q < npat; ++q) {
        if (q == 0 || pats[q].pair != pats[q - 1].pair)
            g0.push_back(q);
        group_of[q] = (int)g0.size() - 1;
    }
    const int ngrp = (int)g0.size();
    g0.push_back(npat);
    const int nzw = (ngrp * R + 31) / 32;
    os << "#define NGRP " << ngrp << "\n#define NZW " << nzw << "\n#define HSW (NGRP * R + NZW)\n";
    // per pattern group: the exact recount of each of its patterns at one start
    // from the window columns cA..cT, with the pattern's position masks compiled in
    std::ostringstream vs;
    for (int gi = 0; gi < ngrp; ++gi) {
        vs << "                        case " << gi << ":\n";
        for (int q = g0[gi]; q < g0[gi + 1]; ++q) {
            const ScanPattern &p = pats[q];
            uint32_t m[4] = {0, 0, 0, 0}, lm = 0, cm = 0;
            for (int i = 0; i < p.L; ++i) {
                for (int x = 0; x < 4; ++x)
                    if (p.mask[i] & (1 << x))
                        m[x] |= 1u << i;
                lm |= 1u << i;
                if (p.strand == 0 ? (i >= p.L - p.clamp) : (i < p.clamp)) // the c 3'-most positions
                    cm |= 1u << i;
            }
            vs << "                        {\n"
               << "                            const u32 mis = ~((cA & " << m[0] << "u) | (cC & " << m[1]
               << "u) | (cG & " << m[2] << "u) | (cT & " << m[3] << "u)) & " << lm << "u;\n"
               << "                            const u32 mm = __popc(mis);\n"
               << "                            if (mm <= " << p.k << "u) {\n"
               << "                                some = true;\n"
               << "                                if (" << (cm ? "(mis & " + std::to_string(cm) + "u) == 0u && " : "")
               << "P + " << p.L << "u <= cend) {\n"
               << "                                    if (lane == (int)(nv & 31u))\n"
               << "                                        stash[warp * 32 + lane] = ((((u64)" << p.pair
               << "u << pbits) | P) << 10) | " << ((p.primer << 9) | (p.strand << 8)) << "ull | (u64)mm;\n"
               << "                                    if ((++nv & 31u) == 0u)\n"
               << "                                        flush(32u);\n"
               << "                                }\n"
               << "                            }\n"
               << "                        }\n";
        }
        vs << "                        break;\n";
    }
    os << "#define S " << t.stages << "\n#define WPC " << t.warps << "\n#define SLICES (W / (32 * R))\n"
       << "#define SLW (32 * R + 32)\n";
    os << "extern \"C\" __global__ void __launch_bounds__(NT, " << t.min_blocks << ")\n"
       << "ah_scan_kernel(const u32 *__restrict__ planes, u64 n_tiles, const u64 *__restrict__ contig_off,\n"
       << "               u32 n_contigs, u64 *__restrict__ keys, u64 cap, u64 *__restrict__ counter, int pbits,\n"
       << "               int *__restrict__ err, u64 *__restrict__ work, const u64 *__restrict__ tile_list,\n"
       << "               const u32 *__restrict__ tile_contig, const u32 *__restrict__ tile_room, u64 wait_ns,\n"
       << "               int stall_first)\n{\n"
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
       << "  // per warp: hit words of one lane being visited, the key stash, its fill\n"
       << "  // count, and the last contig found ([w_cs, w_ce) in flat positions)\n"
       << "  __shared__ u32 hsbuf[WPC * HSW];\n"
       << "  __shared__ u64 stash[WPC * 32];\n"
       << "  __shared__ u64 w_cs[WPC], w_ce[WPC];\n"
       << "  __shared__ u32 w_nv[WPC];\n"
       << "  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;\n"
       << "  u32 *wbuf = smbuf + warp * (S * 4 * SLW);\n"
       << "  u64 *wbar = bars + warp * S;\n"
       << "  u64 *witem = claims + warp * S;\n"
       << "  const u64 n_items = n_tiles * SLICES;\n"
       << "  if (lane == 0) {\n"
       << "    w_nv[warp] = 0u;\n"
       << "    w_cs[warp] = 0ull;\n"
       << "    w_ce[warp] = 0ull;\n"
       << "    for (int q = 0; q < S; ++q) mbar_init(&wbar[q], 1);\n"
       << "    asm volatile(\"fence.mbarrier_init.release.cluster;\" ::: \"memory\");\n"
       << "  }\n"
       << "  __syncwarp();\n"
       << "  // stall_first (a test of the timeout path): the first slice of each warp is\n"
       << "  // armed on its barrier without a copy, so its wait can only run out\n"
       << "  auto issue = [&](u64 wi, int stg, bool copy) {\n"
       << "    const u64 tl = tile_list ? tile_list[wi / SLICES] : wi / SLICES;\n"
       << "    const int sl = (int)(wi % SLICES);\n"
       << "    asm volatile(\"mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\" ::\"r\"(smem_addr(&wbar[stg])),\n"
       << "                 \"r\"((u32)(4 * SLW * 4)) : \"memory\");\n"
       << "    if (copy)\n"
       << "      for (int x = 0; x < 4; ++x)\n"
       << "        tma_copy(wbuf + (stg * 4 + x) * SLW, planes + (tl * 4 + x) * WX + sl * 32 * R, SLW * 4, &wbar[stg]);\n"
       << "  };\n"
       << "  // append the n keys stash[warp * 32 + 0 .. n) with one atomic\n"
       << "  auto flush = [&](u32 n) {\n"
       << "    u64 base = 0;\n"
       << "    if (lane == 0) base = atomicAdd(counter, (u64)n);\n"
       << "    base = __shfl_sync(0xffffffffu, base, 0);\n"
       << "    if ((u32)lane < n && base + lane < cap) keys[base + lane] = stash[warp * 32 + lane];\n"
       << "  };\n"
       << "  if (lane == 0)\n"
       << "    for (int q = 0; q < S; ++q) {\n"
       << "      const u64 w = atomicAdd(work, 1ull);\n"
       << "      witem[q] = w;\n"
       << "      if (w < n_items) issue(w, q, !(stall_first && q == 0));\n"
       << "    }\n"
       << "  __syncwarp();\n"
       << "  for (int k = 0;; ++k) {\n"
       << "    const int stg = k % S;\n"
       << "    const u64 wi = witem[stg];\n"
       << "    if (wi >= n_items)\n"
       << "      break;\n"
       << "    const bool ok = mbar_wait(&wbar[stg], (u32)((k / S) & 1), wait_ns);\n"
       << "    if (!__all_sync(0xffffffffu, ok)) {\n"
       << "      // a copy did not land in time: report, wait (bounded, ~2 s) for every copy\n"
       << "      // of this warp still in flight, this stage's included, then leave\n"
       << "      if (lane == 0) {\n"
       << "        atomicExch(err, 1);\n"
       << "        for (int d = 0; d < S; ++d)\n"
       << "          if (witem[(k + d) % S] < n_items && !(stall_first && k + d == 0)) // no copy was issued there\n"
       << "            mbar_wait(&wbar[(k + d) % S], (u32)(((k + d) / S) & 1), 2000000000ull);\n"
       << "      }\n"
       << "      break;\n"
       << "    }\n"
       << "    const u64 tile = tile_list ? tile_list[wi / SLICES] : wi / SLICES;\n"
       << "    const int wbase = (int)(wi % SLICES) * 32 * R;\n"
       << "    const u32 room = tile_room[tile]; // used only on hits; the load overlaps the network\n"
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
       << "    u32 hg[NGRP * R];\n";
    std::map<std::pair<int, int>, std::string> cache;
    std::vector<bool> assigned(ngrp * R, false);
    auto one = [&](int q, int r) {
        os << "    // pattern " << q << ", word " << r << "\n";
        std::string hw = gen_hit(g, pats[q], r, cache);
        const int i = group_of[q] * R + r;
        os << "    hg[" << i << "] " << (assigned[i] ? "|=" : "=") << " " << hw << ";\n";
        assigned[i] = true;
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
    os << "    u32 any = 0u;\n";
    for (int i = 0; i < ngrp * R; ++i)
        os << "    any |= hg[" << i << "];\n";
    std::string emit = kEmit;
    emit.replace(emit.find("@VISIT@"), 7, vs.str());
    os << emit;
    os << "    __syncwarp();\n"
       << "    if (lane == 0) { // refill this stage with the next claim\n"
       << "      const u64 w = atomicAdd(work, 1ull);\n"
       << "      witem[stg] = w;\n"
       << "      if (w < n_items) issue(w, stg, true);\n"
       << "    }\n"
       << "    __syncwarp();\n"
       << "  }\n"
       << "  __syncwarp();\n"
       << "  const u32 rest = w_nv[warp] & 31u; // keys still in the stash\n"
       << "  if (rest) flush(rest);\n"
       << "}\n";
    return os.str();
}

// Logic and integer operations of one pattern's network per thread word (the
// generator's own statement count).
static int pattern_ops(const ScanPattern &p)
{
    Gen g;
    std::map<std::pair<int, int>, std::string> cache;
    gen_hit(g, p, 0, cache);
    const std::string src = g.os.str();
    return (int)std::count(src.begin(), src.end(), ';');
}

std::vector<std::pair<int, int>> scan_launch_groups(const std::vector<ScanPattern> &pats)
{
    // measured on GB300: one pair of a 960-oligo primer set at k = 4 (~150-190 operations
    // per word) runs spill-free; three such pairs in one kernel spilled under the
    // register cap and stalled on instruction fetch
    int budget = 240;
    if (const char *e = getenv("AH_SCAN_GROUP_OPS"))
        budget = std::max(1, atoi(e));
    static std::mutex mu;
    static std::map<std::string, std::vector<std::pair<int, int>>> cache;
    std::string key = std::to_string(budget) + "|";
    for (const auto &p : pats) {
        key += std::to_string(p.L) + "," + std::to_string(p.k) + "," + std::to_string(p.pair) + ":";
        for (int i = 0; i < p.L; ++i)
            key += (char)('a' + p.mask[i]);
        key += ";";
    }
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it != cache.end())
        return it->second;
    std::vector<std::pair<int, int>> out;
    int q = 0, start = 0, ops = 0;
    const int n = (int)pats.size();
    while (q < n) {
        int e = q, pops = 0; // the pair starting at q: [q, e)
        while (e < n && pats[e].pair == pats[q].pair)
            pops += pattern_ops(pats[e++]);
        if (q > start && ops + pops > budget) {
            out.push_back({start, q});
            start = q;
            ops = 0;
        }
        ops += pops;
        q = e;
    }
    if (n > start)
        out.push_back({start, n});
    cache[key] = out;
    return out;
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
