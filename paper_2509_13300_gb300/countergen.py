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


def collection(seed: int = 7, n_genomes: int = 50_000, len_lo: float = 1e6, len_hi: float = 8e6, pairs=None,
               k: int = 4, min_len: int = 100, max_len: int = 3000, plants=(1, 15)) -> CounterCollection:
    """Layout of a counter-generated collection (the large workload: 50,000 genomes of
    1-8 Mbp, seed 7).  pairs: list of pcr_params dicts (default: one pair of 960 oligos)."""
    rng = np.random.default_rng(seed)  # primer and patch content only
    if pairs is None:
        pairs = [synth.pcr_params("AGRRTTYGATYHTDGYTYAG", "YCNTTCCYTYDYRGTACT", k=k, min_len=min_len,
                                  max_len=max_len)]
    g = np.arange(n_genomes, dtype=np.uint64)
    u = _uniform(seed, 1, g)
    lengths = np.round(len_lo * (len_hi / len_lo) ** u[:, 0]).astype(np.int64)
    gcs = 0.3 + 0.4 * u[:, 1]
    n_contigs = np.minimum(200, 1 + np.floor(np.log1p(-u[:, 2]) / np.log(0.95))).astype(np.int64)
    contig_off, contig_genome, genome_off = [0], [], [0]
    seg_end, seg_t, seg_letter = [], [], []
    patch_pos, patch_bytes = [], []
    base = 0
    for i in range(n_genomes):
        L = int(lengths[i])
        cuts = np.sort((_uniform(seed, 2, np.arange(max(1, n_contigs[i] - 1)) + (i << 8))[:, 0] * L)
                       .astype(np.int64))[: n_contigs[i] - 1]
        bounds = np.concatenate([[0], cuts, [L]])
        for c in range(len(bounds) - 1):
            contig_off.append(base + int(bounds[c + 1]))
            contig_genome.append(i)
        # N runs: about 0.1 % of the bases, runs of 1..100
        n_runs = max(0, int(round(L * 0.001 / 50.5)))
        ur = _uniform(seed, 3, np.arange(max(n_runs, 1)) + (i << 20))[:n_runs]
        runs = sorted((int(x[0] * L), 1 + int(x[1] * 100)) for x in ur)
        t = gc_thresholds(float(gcs[i]))
        pos = 0
        for s, ln in runs:
            s = max(s, pos)
            e = min(L, s + ln)
            if s >= e:
                continue
            if s > pos:
                seg_end.append(base + s); seg_t.append(t); seg_letter.append(0)
            seg_end.append(base + e); seg_t.append((0, 0, 0)); seg_letter.append(ord("N"))
            pos = e
        seg_end.append(base + L); seg_t.append(t); seg_letter.append(0)
        # planted operon-like regions: forward oligo ... reverse-complemented reverse oligo
        for _ in range(int(rng.integers(plants[0], plants[1] + 1)) if L > 4000 else 0):
            pair = pairs[int(rng.integers(len(pairs)))]
            span = int(rng.integers(max(pair["min_len"], 300), min(pair["max_len"], 1500) + 1))
            s = int(rng.integers(0, L - span))
            kk = pair["k"]
            f = synth._draw_oligo(rng, pair["fwd"], int(rng.integers(0, kk + 1)))
            r = synth._revcomp(synth._draw_oligo(rng, pair["rev"], int(rng.integers(0, kk + 1))))
            for off, text in ((s, f), (s + span - len(r), r)):
                patch_pos.extend(range(base + off, base + off + len(text)))
                patch_bytes.extend(text.encode())
        genome_off.append(base + L)
        base += L
    seg = np.zeros(len(seg_end), dtype=SEGMENT_DTYPE)
    seg["end"] = seg_end
    seg["t_a"], seg["t_c"], seg["t_g"] = (np.array([t[j] for t in seg_t], dtype=np.uint64) for j in range(3))
    seg["letter"] = seg_letter
    pp = np.array(patch_pos, dtype=np.uint64)
    pb = np.frombuffer(bytes(patch_bytes), dtype=np.uint8).copy()
    if len(pp):  # later patches win where two overlap; keep one write per position
        order = np.argsort(pp, kind="stable")
        pp, pb = pp[order], pb[order]
        keep = np.append(pp[1:] != pp[:-1], True)
        pp, pb = pp[keep], pb[keep]
    return CounterCollection(seed, np.array(contig_off, dtype=np.uint64), np.array(contig_genome, dtype=np.uint32),
                             np.array(genome_off, dtype=np.uint64), seg, pp, pb, pairs)
