"""Seeded synthetic inputs shaped like the paper's workloads.

The paper evaluates on bacterial genome collections (RefSeq, GTDB, PATRIC,
AllTheBacteria; Sec. 2.3) that are not available here.  These generators
stand in for them with the same structure: multi-contig bacterial-size
genomes, varying GC content, short runs of N, and rRNA-operon-like regions
where a primer pair binds with a known number of substitutions, together
with degenerate (IUPAC) primer pairs of the degeneracies the paper uses
(the Titan pair has 960 oligonucleotides in total, Sec. 1).

This module only builds inputs.  It computes no mismatch count, no pairing,
no melting temperature and no packing: the planted truth it returns is the
record of what it wrote.  The IUPAC letter table below is used only to draw
planted oligonucleotides and the substitutions placed in them.

Both the GPU path (tests, bench) and the CPU oracle consume these inputs.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# IUPAC letter -> admitted bases; used only to draw planted oligos.
_IUPAC_BASES = {
    "A": "A", "C": "C", "G": "G", "T": "T", "R": "AG", "Y": "CT", "S": "CG", "W": "AT",
    "K": "GT", "M": "AC", "B": "CGT", "D": "AGT", "H": "ACT", "V": "ACG", "N": "ACGT",
}
_BASE_COMP = {"A": "T", "C": "G", "G": "C", "T": "A"}
TWO_WAY = "RYSWKM"
THREE_WAY = "BDHV"

# Primer pairs printed in the paper (Sec. 2.3, benchmarking primer list).
PAPER_PAIRS = {
    "V3V4": ("CCTACGGGNGGCNGCAG", "GACTACNNGGGTATCTAATCC"),
    "V1V9": ("AGRGTTYGATYMTGGCTCAG", "RGYTACCTTGTTACGACTT"),
    "Titan": ("AGRRTTYGATYHTDGYTYAG", "YCNTTCCYTYDYRGTACT"),
    "mecA": ("GTAGAAATGACTGAACGTCCGATAA", "CCAATTCCACATTGTTTCGGTCTAA"),
}

PLANT_DTYPE = np.dtype([("genome", "<u4"), ("contig", "<u4"), ("start", "<u4"), ("end", "<u4"),
                        ("orient", "u1"), ("subs_left", "u1"), ("subs_right", "u1"), ("pair", "u1")])


@dataclass
class Workload:
    """A genome collection plus primer pairs.

    seq            uint8 ASCII, all contigs concatenated
    contig_off     uint64[n_contigs + 1], contig c is seq[contig_off[c]:contig_off[c+1]]
    contig_genome  uint32[n_contigs], genome id of each contig
    pairs          list of dicts: fwd, rev, k, clamp, min_len, max_len, tm_min, dnac1_nM,
                   dnac2_nM, Na_mM, K_mM, Tris_mM, Mg_mM, dNTPs_mM, saltcorr
    planted        PLANT_DTYPE records of the planted amplicons (orient 0 = FR, 1 = RF)
    """
    name: str
    seq: np.ndarray
    contig_off: np.ndarray
    contig_genome: np.ndarray
    pairs: list
    planted: np.ndarray
    genome_off: np.ndarray = field(default=None)  # uint64[n_genomes+1] in seq coordinates

    @property
    def n_bases(self) -> int:
        return int(self.contig_off[-1])

    @property
    def n_contigs(self) -> int:
        return len(self.contig_off) - 1


def pcr_params(fwd, rev, k, min_len, max_len, tm_min=float("-inf"), clamp=0, dnac1_nM=250.0,
               dnac2_nM=25.0, Na_mM=50.0, K_mM=0.0, Tris_mM=0.0, Mg_mM=0.0, dNTPs_mM=0.0, saltcorr=5):
    return dict(fwd=fwd, rev=rev, k=k, clamp=clamp, min_len=min_len, max_len=max_len, tm_min=tm_min,
                dnac1_nM=dnac1_nM, dnac2_nM=dnac2_nM, Na_mM=Na_mM, K_mM=K_mM, Tris_mM=Tris_mM,
                Mg_mM=Mg_mM, dNTPs_mM=dNTPs_mM, saltcorr=saltcorr)


def random_primer(rng: np.random.Generator, length: int, codes: str) -> str:
    """Random ACGT primer with the given degenerate letters at random positions."""
    p = list(rng.choice(list("ACGT"), size=length))
    pos = rng.choice(length, size=len(codes), replace=False)
    for i, c in zip(pos, codes):
        p[int(i)] = c
    return "".join(p)


def random_bases(rng: np.random.Generator, n: int, gc: float) -> np.ndarray:
    """i.i.d. bases with P(G) = P(C) = gc/2 and P(A) = P(T) = (1-gc)/2."""
    u = rng.random(n, dtype=np.float32)
    idx = ((u >= gc / 2).astype(np.uint8) + (u >= gc) + (u >= gc + (1 - gc) / 2))
    return np.frombuffer(b"GCAT", dtype=np.uint8)[idx]


def _draw_oligo(rng, primer: str, n_subs: int) -> str:
    """One oligo of `primer` with `n_subs` substitutions at non-N positions, each
    by a base outside that position's IUPAC set."""
    o = [rng.choice(list(_IUPAC_BASES[c])) for c in primer]
    cand = [i for i, c in enumerate(primer) if c != "N"]
    n_subs = min(n_subs, len(cand))
    for i in rng.choice(cand, size=n_subs, replace=False):
        outside = [b for b in "ACGT" if b not in _IUPAC_BASES[primer[int(i)]]]
        o[int(i)] = rng.choice(outside)
    return "".join(o)


def _revcomp(s: str) -> str:
    return "".join(_BASE_COMP[b] for b in reversed(s))


def _contig_lengths(rng, total: int, n_contigs: int) -> np.ndarray:
    n_contigs = max(1, min(n_contigs, total))
    if n_contigs == 1:
        return np.array([total], dtype=np.int64)
    cuts = np.sort(rng.choice(np.arange(1, total), size=n_contigs - 1, replace=False))
    edges = np.concatenate([[0], cuts, [total]])
    return np.diff(edges).astype(np.int64)


def _add_n_runs(rng, g: np.ndarray, frac: float, max_run: int = 100):
    if frac <= 0:
        return
    n_runs = int(round(frac * len(g) / ((1 + max_run) / 2)))
    for _ in range(n_runs):
        ln = int(rng.integers(1, max_run + 1))
        s = int(rng.integers(0, max(1, len(g) - ln)))
        g[s:s + ln] = ord("N")


def _plant(rng, g: np.ndarray, contig_bounds, pair: dict, lengths, subs_fn, genome_id, contig_base, pair_idx,
           out: list, max_tries: int = 200):
    """Write amplicons (forward oligo + filler + revcomp(reverse oligo)), FR or
    (reverse-complemented as a whole) RF, into distinct stretches of single contigs."""
    taken = []
    for length in lengths:
        for _ in range(max_tries):
            ci = int(rng.integers(0, len(contig_bounds)))
            lo, hi = contig_bounds[ci]
            if hi - lo < length + 2:
                continue
            s = int(rng.integers(lo, hi - length + 1))
            if any(not (s + length <= a or b <= s) for a, b in taken):
                continue
            sl, sr = subs_fn()
            fo = _draw_oligo(rng, pair["fwd"], sl)
            ro = _draw_oligo(rng, pair["rev"], sr)
            filler_len = length - len(fo) - len(ro)
            if filler_len < 0:
                continue
            filler = random_bases(rng, filler_len, 0.5).tobytes().decode()
            region = fo + filler + _revcomp(ro)
            orient = int(rng.integers(0, 2))
            if orient == 1:
                region = _revcomp(region)
            g[s:s + length] = np.frombuffer(region.encode(), dtype=np.uint8)
            taken.append((s, s + length))
            out.append((genome_id, contig_base + ci, s - lo, s - lo + length, orient, sl, sr, pair_idx))
            break


def _assemble(name, genomes, pairs, planted):
    seq = np.concatenate([g for g, _ in genomes]) if genomes else np.zeros(0, np.uint8)
    offs, cg, goff = [0], [], [0]
    base = 0
    for gi, (g, lens) in enumerate(genomes):
        for ln in lens:
            base += int(ln)
            offs.append(base)
            cg.append(gi)
        goff.append(base)
    pl = np.array(planted, dtype=PLANT_DTYPE) if planted else np.zeros(0, PLANT_DTYPE)
    return Workload(name, seq, np.array(offs, np.uint64), np.array(cg, np.uint32), pairs, pl,
                    np.array(goff, np.uint64))


def tiny(seed: int = 0) -> Workload:
    """Plain method, tiny: one 200 kbp genome in 3 contigs, GC 0.5, no N runs,
    10 planted amplicons of 300-1500 bp whose sites carry 0/1/2/3 substitutions
    (cycling); F 19 nt (3 two-way + 1 N = 32 oligos), R 20 nt (2 two-way + 1 N
    = 16 oligos); k = 2; window 200-2000; Na 50 mM, primer 0.25 uM."""
    rng = np.random.default_rng(seed)
    fwd = random_primer(rng, 19, "".join(rng.choice(list(TWO_WAY), 3)) + "N")
    rev = random_primer(rng, 20, "".join(rng.choice(list(TWO_WAY), 2)) + "N")
    pair = pcr_params(fwd, rev, k=2, min_len=200, max_len=2000, dnac1_nM=250.0, Na_mM=50.0)
    n = 200_000
    g = random_bases(rng, n, 0.5)
    lens = _contig_lengths(rng, n, 3)
    bounds, o = [], 0
    for ln in lens:
        bounds.append((o, o + int(ln)))
        o += int(ln)
    planted = []
    cyc = iter(range(1000))

    def subs():
        i = next(cyc)
        return (2 * i) % 4, (2 * i + 1) % 4

    _plant(rng, g, bounds, pair, [int(x) for x in rng.integers(300, 1501, size=10)], subs, 0, 0, 0, planted)
    return _assemble("tiny", [(g, lens)], [pair], planted)


def collection(seed: int = 1, n_genomes: int = 100, len_lo: float = 2e6, len_hi: float = 7e6,
               max_contigs: int = 200, n_frac: float = 0.001, k: int = 3, min_len: int = 100,
               max_len: int = 2500, pairs=None, plant_len: int = 1500, plant_max: int = 15,
               max_subs: int = 4, name: str = "collection") -> Workload:
    """Genome collection: lengths log-uniform in [len_lo, len_hi], contig count
    geometric (p = 0.05) truncated to 1..max_contigs, GC per genome U(0.3, 0.7),
    a fraction n_frac of bases in N runs of 1-100, 1..plant_max planted 1.5 kbp
    operon-like regions per genome with site substitutions U{0..max_subs}.
    Default pair: F 20 nt with six 2-way + two 3-way codes (576 oligos), R 22 nt
    with one N + five 2-way + one 3-way (384 oligos): 960 in total."""
    rng = np.random.default_rng(seed)
    if pairs is None:
        fwd = random_primer(rng, 20, "".join(rng.choice(list(TWO_WAY), 6)) + "".join(rng.choice(list(THREE_WAY), 2)))
        rev = random_primer(rng, 22, "N" + "".join(rng.choice(list(TWO_WAY), 5)) + "".join(rng.choice(list(THREE_WAY), 1)))
        pairs = [pcr_params(fwd, rev, k=k, min_len=min_len, max_len=max_len)]
    genomes, planted = [], []
    contig_base = 0
    for gi in range(n_genomes):
        L = int(np.exp(rng.uniform(np.log(len_lo), np.log(len_hi))))
        gc = float(rng.uniform(0.3, 0.7))
        g = random_bases(rng, L, gc)
        _add_n_runs(rng, g, n_frac)
        nc = int(min(max_contigs, rng.geometric(0.05)))
        lens = _contig_lengths(rng, L, nc)
        bounds, o = [], 0
        for ln in lens:
            bounds.append((o, o + int(ln)))
            o += int(ln)
        pj = int(rng.integers(0, len(pairs)))
        n_pl = int(rng.integers(1, plant_max + 1))
        _plant(rng, g, bounds, pairs[pj], [plant_len] * n_pl,
               lambda: (int(rng.integers(0, max_subs + 1)), int(rng.integers(0, max_subs + 1))),
               gi, contig_base, pj, planted)
        genomes.append((g, lens))
        contig_base += len(lens)
    return _assemble(name, genomes, pairs, planted)


def random_small(seed: int, n_bases: int = 2000, n_contigs: int = 3, L_f: int = 8, L_r: int = 7,
                 k: int = 2, codes_f: str = "RN", codes_r: str = "Y", lower_frac: float = 0.0,
                 iupac_frac: float = 0.0, min_len: int = 20, max_len: int = 400, gc: float = 0.5) -> Workload:
    """Small random case for property and edge-case tests: short primers (so
    chance hits are frequent), optional lower-case letters and non-ACGT IUPAC
    letters inside the genome."""
    rng = np.random.default_rng(seed)
    fwd = random_primer(rng, L_f, codes_f)
    rev = random_primer(rng, L_r, codes_r)
    pair = pcr_params(fwd, rev, k=k, min_len=min_len, max_len=max_len)
    g = random_bases(rng, n_bases, gc)
    if iupac_frac > 0:
        m = rng.random(n_bases) < iupac_frac
        g[m] = np.frombuffer(b"NRYKMSWBDHV-", dtype=np.uint8)[rng.integers(0, 12, size=int(m.sum()))]
    if lower_frac > 0:
        m = (rng.random(n_bases) < lower_frac) & (g >= ord("A")) & (g <= ord("Z"))
        g[m] += ord("a") - ord("A")
    lens = _contig_lengths(rng, n_bases, n_contigs)
    return _assemble("random_small", [(g, lens)], [pair], [])


def _mutate(rng, s: str, sub: float, indel: float) -> str:
    """Copy of s with per-letter substitutions (rate sub) and single-letter
    insertions and deletions (rate indel each)."""
    out = []
    for c in s:
        u = rng.random()
        if u < indel:  # deletion
            continue
        if u < 2 * indel:  # insertion before the letter
            out.append("ACGT"[int(rng.integers(4))])
        if rng.random() < sub:
            c = "ACGT".replace(c, "")[int(rng.integers(3))] if c in "ACGT" else c
        out.append(c)
    return "".join(out)


def operon_family(seed: int = 21, n_genomes: int = 12, genome_len: int = 150_000, template_len: int = 600,
                  copies=(1, 4), sub: float = 0.02, indel: float = 0.005, k: int = 2) -> Workload:
    """Genomes carrying copies of one operon-like template (a gene family): each
    copy is the forward primer (an oligo with 0-2 substitutions, 70 % exact),
    the template with per-copy substitutions and small indels, and the reverse
    complement of the reverse primer, inserted in either orientation into a
    random genome of one contig.  Amplicons whose two sites match exactly are
    the training set of a profile HMM; the others are scored against it."""
    rng = np.random.default_rng(seed)
    fwd = random_primer(rng, 20, "".join(rng.choice(list(TWO_WAY), 2)))
    rev = random_primer(rng, 20, "".join(rng.choice(list(TWO_WAY), 2)))
    pair = pcr_params(fwd, rev, k=k, min_len=100, max_len=template_len + 400)
    template = random_bases(rng, template_len, 0.5).tobytes().decode()
    genomes = []
    for gi in range(n_genomes):
        g = random_bases(rng, genome_len, float(rng.uniform(0.4, 0.6)))
        n_cp = int(rng.integers(copies[0], copies[1] + 1))
        slots = np.sort(rng.choice(genome_len // (template_len + 500) - 1, size=n_cp, replace=False))
        for sl in slots:
            nf = 0 if rng.random() < 0.7 else int(rng.integers(1, 3))
            nr = 0 if rng.random() < 0.7 else int(rng.integers(1, 3))
            body = _draw_oligo(rng, fwd, nf) + _mutate(rng, template, sub, indel) + _revcomp(_draw_oligo(rng, rev, nr))
            if rng.random() < 0.5:
                body = _revcomp(body)
            p0 = int(sl) * (template_len + 500) + int(rng.integers(0, 100))
            g[p0:p0 + len(body)] = np.frombuffer(body.encode(), dtype=np.uint8)
        genomes.append((g, [genome_len]))
    return _assemble("operon_family", genomes, [pair], [])
