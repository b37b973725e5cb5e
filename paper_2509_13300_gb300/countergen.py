"""Counter-based synthetic genome collections (large and served workloads).

Large collections are generated on the device (ah_generate_bases) rather than
on the host: every base is a function of its flat position alone, so any
range can be produced independently, in any chunking, on either side.  This
module holds the host side: the Philox4x32-10 counter-based generator
(Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as easy as 1, 2,
3", SC 2011) written from its published definition, the collection layout
(genome lengths, contigs, GC, N runs, planted primer sites) drawn from it,
and a CPU twin of the device's base generation used by the tests.

The layout follows the collection generator of synth.py (log-uniform genome
lengths, geometric contig counts capped at 200, GC uniform in 0.3-0.7, 0.1 %
of bases in N runs of 1-100, operon-like planted regions whose primer sites
carry 0..k substitutions).  Bases: position P draws output P mod 4 of
Philox(counter = (P div 4 low, P div 4 high, 0, 0), key = (seed low, seed
high)) and maps it through the genome's integer thresholds (A below t_a, C
below t_c, G below t_g, else T).  Like synth.py, this module computes no
mismatch count, pairing, melting temperature or packing.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import synth

_M0, _M1 = np.uint64(0xD2511F53), np.uint64(0xCD9E8D57)
_W0, _W1 = 0x9E3779B9, 0xBB67AE85
_MASK = np.uint64(0xFFFFFFFF)

SEGMENT_DTYPE = np.dtype([("end", "<u8"), ("t_a", "<u4"), ("t_c", "<u4"), ("t_g", "<u4"), ("letter", "<u4")])


def philox4x32(ctr: np.ndarray, key) -> np.ndarray:
    """Philox4x32-10: ctr (N, 4) uint32 counters, key (2,) uint32 -> (N, 4) uint32."""
    c = [np.asarray(ctr[:, i], dtype=np.uint64) for i in range(4)]
    k0, k1 = int(key[0]) & 0xFFFFFFFF, int(key[1]) & 0xFFFFFFFF
    for r in range(10):
        if r:
            k0 = (k0 + _W0) & 0xFFFFFFFF
            k1 = (k1 + _W1) & 0xFFFFFFFF
        p0 = _M0 * c[0]
        p1 = _M1 * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c = [hi1 ^ c[1] ^ np.uint64(k0), lo1, hi0 ^ c[3] ^ np.uint64(k1), lo0]
    return np.stack([x.astype(np.uint32) for x in c], axis=1)


def _uniform(seed: int, stream: int, i: np.ndarray, j: int = 0) -> np.ndarray:
    """(N, 4) uniforms in [0, 1) from counters (i, j, stream, 0), key = seed."""
    i = np.asarray(i, dtype=np.uint64)
    ctr = np.stack([i & _MASK, i >> np.uint64(32), np.full_like(i, j), np.full_like(i, stream)], axis=1)
    return philox4x32(ctr.astype(np.uint32), (seed & 0xFFFFFFFF, seed >> 32)) / 4294967296.0


def gc_thresholds(gc: float):
    """Integer thresholds on a 32-bit draw: P(A) = P(T) = (1 - gc) / 2, P(C) = P(G) = gc / 2."""
    at = int((1.0 - gc) / 2.0 * 4294967296.0)
    cg = int(gc / 2.0 * 4294967296.0)
    return at, at + cg, at + 2 * cg


def bases(seed: int, segments: np.ndarray, p0: int, p1: int, patches=None) -> np.ndarray:
    """CPU twin of the device generator: ASCII bases of flat positions [p0, p1)."""
    pos = np.arange(p0, p1, dtype=np.uint64)
    if len(pos) == 0:
        return np.zeros(0, dtype=np.uint8)
    q = pos >> np.uint64(2)
    uq, inv = np.unique(q, return_inverse=True)
    ctr = np.stack([uq & _MASK, uq >> np.uint64(32), np.zeros_like(uq), np.zeros_like(uq)], axis=1).astype(np.uint32)
    out4 = philox4x32(ctr, (seed & 0xFFFFFFFF, seed >> 32))
    draw = out4[inv, (pos & np.uint64(3)).astype(np.int64)].astype(np.uint64)
    seg = np.searchsorted(segments["end"], pos, side="right")
    ta, tc, tg = (segments[f][seg].astype(np.uint64) for f in ("t_a", "t_c", "t_g"))
    letter = segments["letter"][seg]
    b = np.where(draw < ta, ord("A"), np.where(draw < tc, ord("C"), np.where(draw < tg, ord("G"), ord("T"))))
    b = np.where(letter != 0, letter, b).astype(np.uint8)
    if patches is not None and len(patches[0]):
        pp, pb = patches
        sel = (pp >= p0) & (pp < p1)
        b[(pp[sel] - p0).astype(np.int64)] = pb[sel]
    return b


@dataclass
class CounterCollection:
    seed: int
    contig_off: np.ndarray     # uint64, n_contigs + 1
    contig_genome: np.ndarray  # uint32
    genome_off: np.ndarray     # uint64, n_genomes + 1
    segments: np.ndarray       # SEGMENT_DTYPE, tiling [0, n_bases)
    patch_pos: np.ndarray      # uint64 flat positions overwritten after the bulk bases
    patch_bytes: np.ndarray    # uint8
    pairs: list

    @property
    def n_bases(self) -> int:
        return int(self.contig_off[-1])

    def bases(self, p0: int = 0, p1: int | None = None) -> np.ndarray:
        return bases(self.seed, self.segments, p0, self.n_bases if p1 is None else p1,
                     (self.patch_pos, self.patch_bytes))

    def workload(self, genomes=None) -> synth.Workload:
        """The collection (or some genomes of it) as a host Workload, bases from the CPU twin."""
        if genomes is None:
            genomes = range(len(self.genome_off) - 1)
        seqs, offs, gens = [], [0], []
        for g in genomes:
            a, b = int(self.genome_off[g]), int(self.genome_off[g + 1])
            seqs.append(self.bases(a, b))
            c0 = int(np.searchsorted(self.contig_off, a, side="left"))
            c1 = int(np.searchsorted(self.contig_off, b, side="left"))
            for c in range(c0, c1):
                offs.append(offs[-1] + int(self.contig_off[c + 1] - self.contig_off[c]))
                gens.append(g)
        seq = np.concatenate(seqs) if seqs else np.zeros(0, np.uint8)
        return synth.Workload(name="counter", seq=seq, contig_off=np.array(offs, dtype=np.uint64),
                              contig_genome=np.array(gens, dtype=np.uint32), pairs=self.pairs,
                              planted=np.zeros(0, dtype=synth.PLANT_DTYPE))


def _draw_oligos(rng, primer: str, n_subs: np.ndarray) -> np.ndarray:
    """len(n_subs) oligos of `primer` (uint8 rows): each position drawn from its
    IUPAC set, then n_subs[i] distinct non-N positions replaced by a base outside
    their set."""
    n, L = len(n_subs), len(primer)
    sets = [synth._IUPAC_BASES[ch] for ch in primer]
    out = np.empty((n, L), dtype=np.uint8)
    for j, st in enumerate(sets):
        alpha = np.frombuffer("".join(sorted(st)).encode(), dtype=np.uint8)
        out[:, j] = alpha[rng.integers(len(alpha), size=n)]
    cand = np.array([j for j, ch in enumerate(primer) if ch != "N"], dtype=np.int64)
    if len(cand) and n:
        order = np.argsort(rng.random((n, len(cand))), axis=1)  # a random permutation per row
        k = np.minimum(n_subs, len(cand))
        for r in range(int(k.max()) if len(k) else 0):
            rows = np.nonzero(k > r)[0]
            cols = cand[order[rows, r]]
            for j in np.unique(cols):
                outside = np.frombuffer("".join(b for b in "ACGT" if b not in sets[j]).encode(), dtype=np.uint8)
                sel = rows[cols == j]
                out[sel, j] = outside[rng.integers(len(outside), size=len(sel))]
    return out


_COMP = np.zeros(256, dtype=np.uint8)
for _a, _b in zip(b"ACGT", b"TGCA"):
    _COMP[_a] = _b


def collection(seed: int = 7, n_genomes: int = 50_000, len_lo: float = 1e6, len_hi: float = 8e6, pairs=None,
               k: int = 4, min_len: int = 100, max_len: int = 3000, plants=(1, 15)) -> CounterCollection:
    """Layout of a counter-generated collection (the large workload: 50,000 genomes of
    1-8 Mbp, seed 7).  pairs: list of pcr_params dicts (default: one pair of 960 oligos).
    Every draw is vectorised over genomes, so 50,000 genomes lay out in seconds."""
    rng = np.random.default_rng(seed)  # primer and patch content only
    if pairs is None:
        pairs = [synth.pcr_params("AGRRTTYGATYHTDGYTYAG", "YCNTTCCYTYDYRGTACT", k=k, min_len=min_len,
                                  max_len=max_len)]
    G = n_genomes
    g = np.arange(G, dtype=np.uint64)
    u = _uniform(seed, 1, g)
    lengths = np.round(len_lo * (len_hi / len_lo) ** u[:, 0]).astype(np.int64)
    gcs = 0.3 + 0.4 * u[:, 1]
    n_contigs = np.minimum(200, 1 + np.floor(np.log1p(-u[:, 2]) / np.log(0.95))).astype(np.int64)
    base = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    # contigs: n_c - 1 sorted cuts per genome (counter (genome << 8) + j)
    nc1 = n_contigs - 1
    owner = np.repeat(np.arange(G), nc1)
    j = np.arange(len(owner)) - np.repeat(np.cumsum(nc1) - nc1, nc1)
    cu = _uniform(seed, 2, (owner.astype(np.uint64) << np.uint64(8)) + j.astype(np.uint64))[:, 0]
    cuts = (cu * lengths[owner]).astype(np.int64)
    o = np.lexsort((cuts, owner))
    cuts, owner_s = cuts[o], owner[o]
    # contig starts: genome start, then the genome's cuts
    starts = np.concatenate([base[:-1], base[owner_s] + cuts])
    sg = np.concatenate([np.arange(G), owner_s])
    o = np.lexsort((starts, sg))
    contig_off = np.append(starts[o], base[-1]).astype(np.uint64)
    contig_genome = sg[o].astype(np.uint32)
    # N runs, about 0.1 % of the bases: runs of 1..100 at sorted starts, each cut
    # short at the next run's start (counter (genome << 20) + j)
    n_runs = np.round(lengths * 0.001 / 50.5).astype(np.int64)
    rown = np.repeat(np.arange(G), n_runs)
    j = np.arange(len(rown)) - np.repeat(np.cumsum(n_runs) - n_runs, n_runs)
    ur = _uniform(seed, 3, (rown.astype(np.uint64) << np.uint64(20)) + j.astype(np.uint64))
    rs = (ur[:, 0] * lengths[rown]).astype(np.int64)
    rl = 1 + (ur[:, 1] * 100).astype(np.int64)
    o = np.lexsort((rs, rown))
    rs, rl, rown = rs[o], rl[o], rown[o]
    nxt = np.append(rs[1:], 0)
    last = np.append(rown[1:] != rown[:-1], True)
    re = np.minimum(rs + rl, np.where(last, lengths[rown], nxt))
    keep = re > rs
    rs, re, rown = rs[keep], re[keep], rown[keep]
    # segments: per genome, base stretches between the N runs, the N runs, the tail
    at, cg = ((1.0 - gcs) / 2.0 * 4294967296.0).astype(np.int64), (gcs / 2.0 * 4294967296.0).astype(np.int64)
    thr = np.stack([at, at + cg, at + 2 * cg], axis=1)
    prev_end = np.where(np.append(True, rown[1:] != rown[:-1]), 0, np.append(0, re[:-1]))
    gap = rs > prev_end
    seg_end = np.concatenate([base[rown[gap]] + rs[gap], base[rown] + re, base[1:]])
    seg_g = np.concatenate([rown[gap], rown, np.arange(G)])
    seg_n = np.concatenate([np.zeros(gap.sum(), bool), np.ones(len(rown), bool), np.zeros(G, bool)])
    o = np.argsort(seg_end, kind="stable")
    seg = np.zeros(len(seg_end), dtype=SEGMENT_DTYPE)
    seg["end"] = seg_end[o]
    for f, col in zip(("t_a", "t_c", "t_g"), range(3)):
        seg[f] = np.where(seg_n[o], 0, thr[seg_g[o], col])
    seg["letter"] = np.where(seg_n[o], ord("N"), 0)
    # planted operon-like regions: forward oligo ... reverse-complemented reverse oligo
    npl = np.where(lengths > 4000, rng.integers(plants[0], plants[1] + 1, size=G), 0)
    pg = np.repeat(np.arange(G), npl)
    P = len(pg)
    which = rng.integers(len(pairs), size=P)
    lo = np.array([max(p["min_len"], 300) for p in pairs])[which]
    hi = np.array([min(p["max_len"], 1500) for p in pairs])[which]
    span = lo + (rng.random(P) * (hi - lo + 1)).astype(np.int64)
    ps = (rng.random(P) * (lengths[pg] - span)).astype(np.int64)
    kk = np.array([p["k"] for p in pairs])[which]
    pos_l, byt_l = [], []
    for i, p in enumerate(pairs):
        sel = np.nonzero(which == i)[0]
        if not len(sel):
            continue
        f = _draw_oligos(rng, p["fwd"], (rng.random(len(sel)) * (kk[sel] + 1)).astype(np.int64))
        r = _draw_oligos(rng, p["rev"], (rng.random(len(sel)) * (kk[sel] + 1)).astype(np.int64))
        r = _COMP[r[:, ::-1]]  # reverse complement
        s0 = base[pg[sel]] + ps[sel]
        s1 = s0 + span[sel] - r.shape[1]
        pos_l += [(s0[:, None] + np.arange(f.shape[1])).ravel(), (s1[:, None] + np.arange(r.shape[1])).ravel()]
        byt_l += [f.ravel(), r.ravel()]
    pp = np.concatenate(pos_l).astype(np.uint64) if pos_l else np.zeros(0, np.uint64)
    pb = np.concatenate(byt_l).astype(np.uint8) if byt_l else np.zeros(0, np.uint8)
    if len(pp):  # where two plants overlap, the later one wins; one write per position
        order = np.argsort(pp, kind="stable")
        pp, pb = pp[order], pb[order]
        keep = np.append(pp[1:] != pp[:-1], True)
        pp, pb = pp[keep], pb[keep]
    return CounterCollection(seed, contig_off, contig_genome, base.astype(np.uint64), seg, pp, pb, pairs)
