"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Nothing here compares the oracle with itself: every check uses an
independent definition (minimum Hamming distance over the expanded
oligonucleotides, strand symmetry, planted truth, closed forms, hand sums
from the published NN table, brute-force enumeration).
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
from paper_2509_13300_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# NC-IUB (1984) nucleotide code table: the standard the paper's degenerate
# primers are written in (Sec. 1).
IUPAC = {"A": "A", "C": "C", "G": "G", "T": "T", "R": "AG", "Y": "CT", "S": "CG", "W": "AT", "K": "GT",
         "M": "AC", "B": "CGT", "D": "AGT", "H": "ACT", "V": "ACG", "N": "ACGT"}
COMP = {"A": "T", "C": "G", "G": "C", "T": "A"}


def expand(primer):
    return ["".join(t) for t in itertools.product(*[IUPAC[c] for c in primer])]


def revcomp(s):
    return "".join(COMP[b] for b in reversed(s))


def hamming(a, b):
    return sum(1 for x, y in zip(a, b) if x != y)


def brute_sites(seq: bytes, contig_off, pair):
    """Sites by the definition 'min Hamming distance over every oligo of the
    primer' (Sec. 2.1 Primer matching; reading S1): '+' compares the oligo with
    the window, '-' compares the oligo's reverse complement with the window.
    A non-ACGT genome letter never equals an oligo base."""
    out = []
    oligos = {0: expand(pair["fwd"]), 1: expand(pair["rev"])}
    up = seq.upper()
    for c in range(len(contig_off) - 1):
        lo, hi = int(contig_off[c]), int(contig_off[c + 1])
        g = up[lo:hi].decode()
        for p in range(hi - lo):
            for primer in (0, 1):
                L = len(pair["fwd"] if primer == 0 else pair["rev"])
                if p + L > hi - lo:
                    continue
                w = g[p:p + L]
                for strand in (0, 1):
                    mm = min(hamming(w, o if strand == 0 else revcomp(o)) for o in oligos[primer])
                    if mm <= pair["k"]:
                        out.append((c, p, primer, strand, mm))
    return out


def site_tuples(sites):
    return [(int(s["contig"]), int(s["pos"]), int(s["primer"]), int(s["strand"]), int(s["mm"])) for s in sites]


# ----------------------------------------------------------------------------- scan

def test_iupac_sets_match_standard():
    for code, bases in IUPAC.items():
        for b in "ACGT":
            mm = oracle.window_mismatches(b.encode(), code, 0)
            assert mm == (0 if b in bases else 1), (code, b)
        # non-ACGT genome letters mismatch every code, N included (reading S2)
        for g in b"NRY-.":
            assert oracle.window_mismatches(bytes([g]), code, 0) == 1
        # lower-case genome letters are the same bases
        for b in "acgt":
            assert oracle.window_mismatches(b.encode(), code, 0) == (0 if b.upper() in bases else 1)


def test_reverse_complement_of_codes():
    # the '-' pattern of a single letter admits exactly the complements of its bases
    for code, bases in IUPAC.items():
        for b in "ACGT":
            mm = oracle.window_mismatches(b.encode(), code, 1)
            assert mm == (0 if COMP[b] in bases else 1), (code, b)


@pytest.mark.parametrize("L", [1, 2, 3])
def test_exhaustive_short_primers_every_code(L):
    """Every primer of length L over all 15 codes against every ACGT window:
    mask count == min Hamming over expanded oligos, both strands."""
    codes = list(IUPAC)
    rng = np.random.default_rng(L)
    primers = ["".join(t) for t in itertools.product(codes, repeat=L)]
    if len(primers) > 400:
        primers = [primers[i] for i in rng.choice(len(primers), 400, replace=False)]
    windows = ["".join(t) for t in itertools.product("ACGT", repeat=L)]
    for pr in primers:
        ol = expand(pr)
        for w in windows:
            for strand in (0, 1):
                want = min(hamming(w, o if strand == 0 else revcomp(o)) for o in ol)
                assert oracle.window_mismatches(w.encode(), pr, strand) == want


@pytest.mark.parametrize("seed", range(6))
def test_scan_equals_min_hamming_bruteforce(seed):
    w = synth.random_small(seed, n_bases=700, n_contigs=3, L_f=6 + seed % 3, L_r=5 + seed % 4, k=seed % 3 + 1,
                           codes_f="RNH"[: 1 + seed % 3], codes_r="YS"[: 1 + seed % 2],
                           iupac_frac=0.02, lower_frac=0.1)
    got = site_tuples(oracle.scan(w.seq, w.contig_off, w.contig_genome, w.pairs))
    want = brute_sites(w.seq.tobytes(), w.contig_off, w.pairs[0])
    assert got == want
    assert len(want) > 0


def test_scan_reverse_complement_symmetry():
    """Scanning the reverse-complemented contig turns a site (X, +, p) into
    (X, -, len - L - p) with the same mismatch count, and vice versa."""
    w = synth.random_small(11, n_bases=3000, n_contigs=1, L_f=7, L_r=6, k=2)
    g = w.seq.tobytes().decode()
    rc = revcomp(g).encode()
    a = oracle.scan(w.seq, w.contig_off, w.contig_genome, w.pairs)
    b = oracle.scan(np.frombuffer(rc, np.uint8), w.contig_off, w.contig_genome, w.pairs)
    n = len(g)
    La = {0: len(w.pairs[0]["fwd"]), 1: len(w.pairs[0]["rev"])}
    mapped = sorted((n - La[pr] - p, pr, 1 - st, mm) for (_, p, pr, st, mm) in site_tuples(a))
    other = sorted((p, pr, st, mm) for (_, p, pr, st, mm) in site_tuples(b))
    assert mapped == other and len(mapped) > 10


def test_tiny_planted_sites_recovered():
    """The planted sites of the tiny workload carry 0/1/2/3 substitutions:
    those with <= k = 2 are found with exactly that count, the 3s are not."""
    w = synth.tiny(0)
    sites = oracle.scan(w.seq, w.contig_off, w.contig_genome, w.pairs)
    idx = {(int(s["contig"]), int(s["pos"]), int(s["primer"]), int(s["strand"])): int(s["mm"]) for s in sites}
    Lf, Lr = len(w.pairs[0]["fwd"]), len(w.pairs[0]["rev"])
    k = w.pairs[0]["k"]
    assert len(w.planted) == 10
    for p in w.planted:
        c, s, e = int(p["contig"]), int(p["start"]), int(p["end"])
        if p["orient"] == 0:   # F+ at start, R- ending at end
            left, right = (c, s, 0, 0), (c, e - Lr, 1, 1)
        else:                  # R+ at start, F- ending at end
            left, right = (c, s, 1, 0), (c, e - Lf, 0, 1)
        for key, subs in ((left, int(p["subs_left"] if p["orient"] == 0 else p["subs_right"])),
                          (right, int(p["subs_right"] if p["orient"] == 0 else p["subs_left"]))):
            if subs <= k:
                assert idx.get(key) == subs, (key, subs)
            else:
                assert key not in idx


def test_scan_special_cases():
    w = synth.random_small(3, n_bases=500, n_contigs=4, L_f=6, L_r=5, k=0)
    lens = np.diff(w.contig_off.astype(np.int64))
    # k >= L: every valid start, both primers, both strands, mm = window mismatches
    pairs = [dict(w.pairs[0], k=6)]
    s = oracle.scan(w.seq, w.contig_off, w.contig_genome, pairs)
    want = sum(2 * max(0, int(n) - 6 + 1) + 2 * max(0, int(n) - 5 + 1) for n in lens)
    assert len(s) == want
    # an all-N primer with k = 0 matches every all-ACGT window
    allN = [dict(w.pairs[0], fwd="NNNN", rev="NNNN", k=0)]
    s = oracle.scan(w.seq, w.contig_off, w.contig_genome, allN)
    assert len(s) == sum(4 * max(0, int(n) - 3) for n in lens)
    w2 = synth.random_small(3, n_bases=500, n_contigs=1, iupac_frac=0.05)
    s2 = oracle.scan(w2.seq, w2.contig_off, w2.contig_genome, allN)
    g = w2.seq.tobytes()
    ok = [p for p in range(len(g) - 3) if all(ch in b"ACGT" for ch in g[p:p + 4])]
    assert len(s2) == 4 * len(ok)


def test_clamp():
    """Clamp c: no mismatch in the c 3'-most primer bases (Sec. 2.1)."""
    w = synth.random_small(5, n_bases=2000, n_contigs=2, L_f=7, L_r=6, k=2)
    base = oracle.scan(w.seq, w.contig_off, w.contig_genome, w.pairs)
    cl = oracle.scan(w.seq, w.contig_off, w.contig_genome, [dict(w.pairs[0], clamp=2)])
    g = w.seq.tobytes().upper()
    oligos = {0: expand(w.pairs[0]["fwd"]), 1: expand(w.pairs[0]["rev"])}
    kept = []
    for s in base:
        L = len(w.pairs[0]["fwd"] if s["primer"] == 0 else w.pairs[0]["rev"])
        lo = int(w.contig_off[s["contig"]]) + int(s["pos"])
        win = g[lo:lo + L].decode()
        # 3' end of the primer = right end of a '+' window, left end of a '-' window
        idx = [L - 1, L - 2] if s["strand"] == 0 else [0, 1]
        ok = any(all(win[i] == (o if s["strand"] == 0 else revcomp(o))[i] for i in idx) for o in oligos[s["primer"]])
        if ok:
            kept.append(s)
    assert site_tuples(cl) == site_tuples(kept)
    assert 0 < len(cl) < len(base)


# ----------------------------------------------------------------------------- pair

def test_pair_bruteforce_and_invariants():
    w = synth.random_small(7, n_bases=3000, n_contigs=3, L_f=7, L_r=6, k=2, min_len=30, max_len=300)
    sites = oracle.scan(w.seq, w.contig_off, w.contig_genome, w.pairs)
    amps = oracle.pair(sites, w.pairs)
    pr = w.pairs[0]
    L = {0: len(pr["fwd"]), 1: len(pr["rev"])}
    want = set()
    for i, a in enumerate(sites):
        for j, b in enumerate(sites):
            if a["contig"] == b["contig"] and a["strand"] == 0 and b["strand"] == 1 and b["pos"] >= a["pos"]:
                end = int(b["pos"]) + L[int(b["primer"])]
                if pr["min_len"] <= end - int(a["pos"]) <= pr["max_len"]:
                    want.add((int(a["contig"]), int(a["pos"]), end, {(0, 1): 0, (1, 0): 1, (0, 0): 2, (1, 1): 3}[
                        (int(a["primer"]), int(b["primer"]))], i, j))
    got = [(int(x["contig"]), int(x["start"]), int(x["end"]), int(x["orient"]), int(x["left"]), int(x["right"]))
           for x in amps]
    assert sorted(got) == got and set(got) == want and len(got) > 5
    # the Tm pass flags remove exactly the amplicons with a failing end
    passed = (np.arange(len(sites)) % 3 != 0).astype(np.uint8)
    amps2 = oracle.pair(sites, w.pairs, passed)
    assert {(a[0], a[1], a[2], a[3]) for a in got if passed[a[4]] and passed[a[5]]} == \
        {(int(x["contig"]), int(x["start"]), int(x["end"]), int(x["orient"])) for x in amps2}


def test_tiny_planted_amplicons_called():
    w = synth.tiny(0)
    sites = oracle.scan(w.seq, w.contig_off, w.contig_genome, w.pairs)
    amps = oracle.pair(sites, w.pairs)
    got = {(int(a["contig"]), int(a["start"]), int(a["end"]), int(a["orient"])) for a in amps}
    k = w.pairs[0]["k"]
    n_exp = 0
    for p in w.planted:
        key = (int(p["contig"]), int(p["start"]), int(p["end"]), int(p["orient"]))
        if p["subs_left"] <= k and p["subs_right"] <= k:
            assert key in got
            n_exp += 1
        else:
            assert key not in got
    assert n_exp >= 4


# ----------------------------------------------------------------------------- fetch

def test_fetch_slices_and_reverse_complement():
    w = synth.random_small(9, n_bases=1500, n_contigs=2, lower_frac=0.2, iupac_frac=0.03)
    amps = np.zeros(4, dtype=oracle.AMPLICON_DTYPE)
    amps["contig"] = [0, 0, 1, 1]
    amps["start"] = [0, 10, 5, 0]
    amps["end"] = [50, 200, 300, 1]
    amps["orient"] = [0, 1, 2, 1]
    seqs, offs = oracle.fetch(w.seq, w.contig_off, amps)
    g = w.seq.tobytes()
    for i, a in enumerate(amps):
        lo = int(w.contig_off[a["contig"]])
        raw = g[lo + int(a["start"]):lo + int(a["end"])].decode().upper()
        raw = "".join(ch if ch in "ACGT" else "N" for ch in raw)
        if a["orient"] == 1:
            raw = "".join({"A": "T", "C": "G", "G": "C", "T": "A", "N": "N"}[ch] for ch in reversed(raw))
        assert seqs[int(offs[i]):int(offs[i + 1])].decode() == raw


# ----------------------------------------------------------------------------- Tm

def _read_golden():
    cases, cur = [], None
    for line in open(os.path.join(GOLDEN, "tm_hand.txt")):
        line = line.split("#")[0].strip()
        if not line:
            continue
        f = line.split()
        if f[0] == "case":
            cur = dict(name=f[1], oligo=f[2], bottom=f[3], terms=[])
            cases.append(cur)
        elif f[0] == "term":
            cur["terms"].append((float(f[2]), float(f[3])))
        elif f[0] == "total":
            cur["total"] = (float(f[1]), float(f[2]))
    return cases


P0 = dict(dnac1_nM=250.0, dnac2_nM=25.0, Na_mM=50.0, saltcorr=0)


def _tm_from_terms(H, S, L, p):
    """Two-state NN Tm, Tm = 1000 dH / (dS + R ln x) - 273.15 with
    x = (dnac1 - dnac2/2) 1e-9 and, for salt method 5, the entropy term
    0.368 (N-1) ln[Na+] (SantaLucia 1998)."""
    if p["saltcorr"] == 5:
        S += 0.368 * (L - 1) * math.log(p["Na_mM"] / 1000)
    return 1000 * H / (S + 1.987 * math.log((p["dnac1_nM"] - p["dnac2_nM"] / 2) * 1e-9)) - 273.15


@pytest.mark.parametrize("salt", [0, 5])
def test_tm_hand_computed_cases(salt):
    cases = _read_golden()
    assert len(cases) == 4
    for c in cases:
        H = sum(t[0] for t in c["terms"])
        S = sum(t[1] for t in c["terms"])
        assert abs(H - c["total"][0]) < 1e-9 and abs(S - c["total"][1]) < 1e-9, c["name"]
        p = dict(P0, saltcorr=salt)
        want = _tm_from_terms(H, S, len(c["oligo"]), p)
        got = oracle.duplex_tm(c["oligo"], c["bottom"], p)
        assert abs(got - want) < 1e-9, (c["name"], got, want)


@pytest.mark.parametrize("L", [5, 12, 25])
def test_tm_homopolymer_closed_form(L):
    """A_L / T_L: dH = 2 init(A.T) + (L-1) dH(AA/TT), likewise dS."""
    H = 2 * 2.3 + (L - 1) * -7.9
    S = 2 * 4.1 + (L - 1) * -22.2
    for salt in (0, 5):
        p = dict(P0, saltcorr=salt)
        assert abs(oracle.duplex_tm("A" * L, "T" * L, p) - _tm_from_terms(H, S, L, p)) < 1e-9
        # the same duplex read from the other strand
        assert abs(oracle.duplex_tm("T" * L, "A" * L, p) - _tm_from_terms(H, S, L, p)) < 1e-9


def test_tm_reading_duplex_from_either_end():
    """The NN sum does not depend on which strand is called the top: the duplex
    o / b equals the duplex read from the other strand, rev(b) / rev(o).  Internal
    mismatches are allowed; the ends are Watson-Crick because a terminal
    mismatch is scored by the primer base's class, which is strand-specific."""
    rng = np.random.default_rng(2)
    for _ in range(200):
        L = int(rng.integers(5, 30))
        o = "".join(rng.choice(list("ACGT"), L))
        b = "".join(COMP[x] if rng.random() > 0.2 else rng.choice(list("ACGT")) for x in o)
        b = COMP[o[0]] + b[1:-1] + COMP[o[-1]]
        p = dict(P0, saltcorr=5)
        assert abs(oracle.duplex_tm(o, b, p) - oracle.duplex_tm(b[::-1], o[::-1], p)) < 1e-9


def test_tm_default_table_array_matches_lookup():
    t = oracle.default_table()
    rng = np.random.default_rng(4)
    for _ in range(100):
        L = int(rng.integers(5, 30))
        o = "".join(rng.choice(list("ACGT"), L))
        b = "".join(rng.choice(list("ACGT"), L))
        p = dict(P0, saltcorr=5)
        assert abs(oracle.duplex_tm(o, b, p) - oracle.duplex_tm(o, b, p, t)) < 1e-12
    # stack rotation symmetry of the table: t0 t1 / b0 b1 == b1 b0 / t1 t0
    H = np.array(t.stack_dH).reshape(4, 4, 4, 4)
    S = np.array(t.stack_dS).reshape(4, 4, 4, 4)
    assert np.array_equal(H, H.transpose(3, 2, 1, 0)) and np.array_equal(S, S.transpose(3, 2, 1, 0))
    # ten distinct Watson-Crick stacks, all other stacks zero (reading S12)
    wc = [(a, b, 3 - a, 3 - b) for a in range(4) for b in range(4)]
    assert len({(H[x], S[x]) for x in wc}) == 10
    mask = np.ones((4, 4, 4, 4), bool)
    for x in wc:
        mask[x] = False
    assert not H[mask].any() and not S[mask].any()


def _site_workload(window: str, primer_f: str, primer_r: str):
    seq = np.frombuffer(window.encode(), np.uint8).copy()
    off = np.array([0, len(window)], np.uint64)
    return seq, off


def test_tm_site_max_over_oligos_bruteforce():
    """Site Tm = max over every oligo of the primer of the duplex Tm against
    the template (Sec. 2.1); '-' sites use the + strand bases as the bottom."""
    rng = np.random.default_rng(6)
    p = dict(P0, saltcorr=5, fwd="ACRYTGNCAG", rev="GTKAMCTG", k=10, min_len=0, max_len=0)
    for trial in range(10):
        win = "".join(rng.choice(list("ACGT"), 40))
        seq, off = _site_workload(win, p["fwd"], p["rev"])
        sites = np.zeros(4, dtype=oracle.SITE_DTYPE)
        sites["pos"] = [3, 7, 11, 20]
        sites["primer"] = [0, 1, 0, 1]
        sites["strand"] = [0, 0, 1, 1]
        tm, _ = oracle.tm(seq, off, sites, [p])
        for s, t in zip(sites, tm):
            X = p["fwd"] if s["primer"] == 0 else p["rev"]
            L = len(X)
            w = win[int(s["pos"]):int(s["pos"]) + L]
            bottom = "".join(COMP[x] for x in w) if s["strand"] == 0 else w[::-1]
            want = max(oracle.duplex_tm(o, bottom, p) for o in expand(X))
            assert abs(t - want) < 1e-12


def test_tm_plus_minus_site_symmetry():
    """A '+' site on window w and a '-' site on revcomp(w) are the same duplex."""
    rng = np.random.default_rng(8)
    p = dict(P0, saltcorr=5, fwd="AGRRTTYGATYHTDGYTYAG", rev="ACGT" * 5, k=20, min_len=0, max_len=0)
    for _ in range(5):
        w = "".join(rng.choice(list("ACGT"), 20))
        seq = np.frombuffer((w + "TTTT" + revcomp(w)).encode(), np.uint8).copy()
        off = np.array([0, len(seq)], np.uint64)
        sites = np.zeros(2, dtype=oracle.SITE_DTYPE)
        sites["pos"] = [0, 24]
        sites["strand"] = [0, 1]
        tm, _ = oracle.tm(seq, off, sites, [p])
        assert abs(tm[0] - tm[1]) < 1e-12


def test_tm_nondegenerate_equals_single_oligo_and_monotone():
    p = dict(P0, saltcorr=5, fwd="GATCCAAGTACGT", rev="ACGTACGTAC", k=20, min_len=0, max_len=0)
    w = "GATCCAAGTACGT"
    seq = np.frombuffer(w.encode(), np.uint8).copy()
    off = np.array([0, len(w)], np.uint64)
    sites = np.zeros(1, dtype=oracle.SITE_DTYPE)
    tm, _ = oracle.tm(seq, off, sites, [p])
    assert abs(tm[0] - oracle.duplex_tm(w, "".join(COMP[x] for x in w), p)) < 1e-12
    prev = -1e9
    for na in (5, 20, 50, 100, 500):
        t, _ = oracle.tm(seq, off, sites, [dict(p, Na_mM=na)])
        assert t[0] > prev
        prev = t[0]
    prev = -1e9
    for c1 in (50, 100, 250, 1000, 5000):
        t, _ = oracle.tm(seq, off, sites, [dict(p, dnac1_nM=c1)])
        assert t[0] > prev
        prev = t[0]


def test_tm_mismatch_lowers_tm_and_nonacgt_is_nan():
    p = dict(P0, saltcorr=5, fwd="GATCCAAGTACGTAC", rev="ACGTACGTAC", k=20, min_len=0, max_len=0, tm_min=0.0)
    w = "GATCCAAGTACGTAC"
    bad = w[:6] + ("A" if w[6] != "A" else "C") + w[7:]
    nn = w[:4] + "N" + w[5:]
    seq = np.frombuffer((w + bad + nn).encode(), np.uint8).copy()
    off = np.array([0, len(seq)], np.uint64)
    sites = np.zeros(3, dtype=oracle.SITE_DTYPE)
    sites["pos"] = [0, 15, 30]
    tm, ps = oracle.tm(seq, off, sites, [p])
    assert tm[1] < tm[0] and math.isnan(tm[2])
    assert list(ps) == [1, 1, 0]


def test_salt_equivalent_concentration():
    """von Ahsen (2001): [Na_eq] = Na + K + Tris/2 + 120 sqrt(Mg - dNTPs); the Mg
    term vanishes when dNTPs >= Mg."""
    o, b = "GATCCAAGTACGTAC", "CTAGGTTCATGCATG"
    a = oracle.duplex_tm(o, b, dict(P0, saltcorr=5, Na_mM=50.0))
    assert abs(a - oracle.duplex_tm(o, b, dict(P0, saltcorr=5, Na_mM=20.0, K_mM=10.0, Tris_mM=40.0))) < 1e-12
    assert abs(a - oracle.duplex_tm(o, b, dict(P0, saltcorr=5, Na_mM=50.0, Mg_mM=1.0, dNTPs_mM=2.0))) < 1e-12
    c = oracle.duplex_tm(o, b, dict(P0, saltcorr=5, Na_mM=50.0 - 120.0, Mg_mM=1.5, dNTPs_mM=0.5))
    assert abs(a - c) < 1e-9


def _read_published():
    rows = []
    for line in open(os.path.join(GOLDEN, "tm_biopython.txt")):
        line = line.split("#")[0].strip()
        if line:
            rows.append(line.split())
    return rows


def test_tm_published_values_of_the_named_model():
    """Sec. 2.1 names Biopython's NN model; its documentation prints Tm_NN of one
    28-mer under the defaults (dnac1 = dnac2 = 25 nM, 50 mM Na+, entropy salt
    term) and with Tris and Mg2+, to two decimals.  These fix the gas constant,
    the 273.15 offset, the x = dnac1 - dnac2/2 term, the 0.368 (N-1) ln[Na]
    entropy term and the von Ahsen Tris/2 and 120 sqrt(Mg) terms: a change to
    any of them moves at least one value by more than the printed rounding."""
    rows = [r for r in _read_published() if r[0] == "tm"]
    assert len(rows) == 3
    for r in rows:
        seq = r[1]
        d1, d2, na, k, tris, mg, dntp = (float(x) for x in r[2:9])
        p = dict(dnac1_nM=d1, dnac2_nM=d2, Na_mM=na, K_mM=k, Tris_mM=tris, Mg_mM=mg, dNTPs_mM=dntp,
                 saltcorr=int(r[9]))
        got = oracle.duplex_tm(seq, "".join(COMP[b] for b in seq), p)
        assert abs(got - float(r[10])) <= 0.005 + 1e-9, (r, got)


def test_tm_salt_shift_methods():
    """Method 1 (Schildkraut-Lifson 1965) shifts Tm by the published correction
    (salt_correction(Na=50, method=1) = -21.60); at [Na_eq] = 1 M every salt
    term vanishes (log 1 = 0), so methods 0, 1 and 5 then agree; methods the
    library does not offer give NaN."""
    seq = "CGTTCCAAAGATGTGGGCATGAGCTTAC"
    bot = "".join(COMP[b] for b in seq)
    for r in (r for r in _read_published() if r[0] == "salt"):
        na, k, tris, mg, dntp = (float(x) for x in r[1:6])
        ions = dict(dnac1_nM=25.0, dnac2_nM=25.0, Na_mM=na, K_mM=k, Tris_mM=tris, Mg_mM=mg, dNTPs_mM=dntp)
        shift = oracle.duplex_tm(seq, bot, dict(ions, saltcorr=int(r[6]))) - \
            oracle.duplex_tm(seq, bot, dict(ions, saltcorr=0))
        assert abs(shift - float(r[7])) <= 0.005 + 1e-9, (r, shift)
    one_molar = dict(P0, Na_mM=1000.0)
    t0 = oracle.duplex_tm(seq, bot, dict(one_molar, saltcorr=0))
    for m in (1, 5):
        assert abs(oracle.duplex_tm(seq, bot, dict(one_molar, saltcorr=m)) - t0) < 1e-9
    for m in (2, 3, 4, 6, 7):
        assert math.isnan(oracle.duplex_tm(seq, bot, dict(P0, saltcorr=m)))


def test_degeneracy_of_paper_primers():
    """Sec. 1: the two Titan primers together hold 960 oligonucleotides."""
    f, r = synth.PAPER_PAIRS["Titan"]
    assert oracle.degeneracy(f) + oracle.degeneracy(r) == 960
    w = synth.collection(seed=1, n_genomes=1, len_lo=2e5, len_hi=3e5)
    assert oracle.degeneracy(w.pairs[0]["fwd"]) + oracle.degeneracy(w.pairs[0]["rev"]) == 960
    t = synth.tiny(0)
    assert oracle.degeneracy(t.pairs[0]["fwd"]) + oracle.degeneracy(t.pairs[0]["rev"]) == 48


def test_decoy_reversal_is_per_contig_reversal():
    """The decoy collection reverses each contig (not complemented): twice is the
    identity, each contig equals the original read backwards, and a site of a
    palindromic primer pair on the reversed contig sits at the mirrored position."""
    w = synth.random_small(5, n_bases=3000, n_contigs=4)
    r = oracle.reverse_contigs(w.seq, w.contig_off)
    assert np.array_equal(oracle.reverse_contigs(r, w.contig_off), w.seq)
    for a, b in zip(w.contig_off[:-1], w.contig_off[1:]):
        assert bytes(r[int(a):int(b)]) == bytes(w.seq[int(a):int(b)])[::-1]
    # a pattern equal to its own reverse (ACGGCA reversed is ACGGCA) is found at p and at len - L - p
    pal = "ACGGCA"
    pair = synth.pcr_params(pal, pal, k=0, min_len=10, max_len=100)
    fw = oracle.scan(w.seq, w.contig_off, w.contig_genome, [pair])
    rv = oracle.scan(r, w.contig_off, w.contig_genome, [pair])
    lens = np.diff(w.contig_off.astype(np.int64))
    mir = sorted((int(s["contig"]), int(lens[s["contig"]] - 6 - s["pos"]), int(s["primer"]), int(s["strand"])) for s in fw)
    got = sorted((int(s["contig"]), int(s["pos"]), int(s["primer"]), int(s["strand"])) for s in rv)
    assert mir == got


# ----------------------------------------------------------------------------- amplitypes

def test_amplitypes_of_a_hand_built_collection():
    """Four genomes whose amplicons are cut from known sequences: X (twice in
    genome 0, once as the reverse complement read RF), Y and Z.  Variants are
    numbered by first occurrence (X 0, Y 1, Z 2); genomes 0 and 1 carry the
    same multiset {X: 2, Y: 1} in different orders and share amplitype 0;
    genome 2 carries {X: 1, Y: 1} (another copy number: amplitype 1); genome 3
    carries {Z: 1} (amplitype 2); genome 4 has no amplicon (no row)."""
    X, Y, Z = "ACGTTGCAAGGCTT", "ACGTTGCAAGGCTA", "ACGTNGCAAGGCTT"   # Y, Z differ from X in one letter
    rc = lambda q: "".join({"A": "T", "C": "G", "G": "C", "T": "A", "N": "N"}[c] for c in reversed(q))
    spacer = "GGGGG"
    genomes = [[X, Y, rc(X)], [Y, X, X], [X, Y], [Z], ["CCCC"]]
    orients = [[0, 0, 1], [0, 0, 0], [0, 0], [0], [0]]      # the third amplicon of genome 0 is RF
    seq, off, gen, amps = "", [0], [], []
    for g, parts in enumerate(genomes):
        start = len(seq)
        body = spacer.join(parts) + spacer
        seq += body
        off.append(len(seq))
        gen.append(g)
        if g == 4:
            continue
        pos = 0
        for q, o in zip(parts, orients[g]):
            amps.append((g, g, pos, pos + len(q), o))
            pos += len(q) + len(spacer)
    a = np.zeros(len(amps), dtype=oracle.AMPLICON_DTYPE)
    for i, (g, c, s0, e0, o) in enumerate(amps):
        a[i]["genome"], a[i]["contig"], a[i]["start"], a[i]["end"], a[i]["orient"] = g, c, s0, e0, o
    seq_u8 = np.frombuffer(seq.encode(), dtype=np.uint8).copy()
    vid, rows, nv, nt = oracle.amplitypes(seq_u8, np.array(off, dtype=np.uint64), a)
    assert vid.tolist() == [0, 1, 0, 1, 0, 0, 0, 1, 2]
    assert rows == [(0, 0, 3, 2), (1, 0, 3, 2), (2, 1, 2, 2), (3, 2, 1, 1)]
    assert (nv, nt) == (3, 3)
