"""CPU oracle for the in-silico PCR hot path (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does, and
this package never imports the product library: the two share no code.

The oracle itself is plain C (``oracle.c``), fp64 for the melting
temperature, written straight from the definitions in the paper
(Howard-Stone & Mandoiu, "AmpliconHunter", arXiv 2509.13300, Sec. 2.1).
This module compiles it with gcc on first use and wraps it with ctypes.

Parity is pinned, not assumed: see ``tests/test_oracle_pins.py`` for the
brute-force, symmetry, planted-site, closed-form and hand-computed checks.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "hmm.c")]
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

SITE_DTYPE = np.dtype(
    [("genome", "<u4"), ("contig", "<u4"), ("pos", "<u4"),
     ("primer", "u1"), ("strand", "u1"), ("mm", "u1"), ("pair", "u1")])
AMPLICON_DTYPE = np.dtype(
    [("genome", "<u4"), ("contig", "<u4"), ("start", "<u4"), ("end", "<u4"),
     ("left", "<u4"), ("right", "<u4"), ("orient", "u1"), ("pair", "u1"),
     ("pad0", "u1"), ("pad1", "u1")])
assert SITE_DTYPE.itemsize == 16 and AMPLICON_DTYPE.itemsize == 28


class TmParams(ctypes.Structure):
    _fields_ = [("dnac1_nM", ctypes.c_double), ("dnac2_nM", ctypes.c_double),
                ("Na_mM", ctypes.c_double), ("K_mM", ctypes.c_double),
                ("Tris_mM", ctypes.c_double), ("Mg_mM", ctypes.c_double),
                ("dNTPs_mM", ctypes.c_double), ("tm_min", ctypes.c_double),
                ("saltcorr", ctypes.c_int32), ("pad", ctypes.c_int32)]


class NNTable(ctypes.Structure):
    _fields_ = [("stack_dH", ctypes.c_double * 256), ("stack_dS", ctypes.c_double * 256),
                ("term_dH", ctypes.c_double * 16), ("term_dS", ctypes.c_double * 16)]


def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so (gcc, -O2, OpenMP)."""
    with _lock:
        if not force and os.path.exists(_LIB) and all(os.path.getmtime(_LIB) >= os.path.getmtime(f) for f in _SRCS):
            return _LIB
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC",
                               "-o", tmp] + _SRCS + ["-lm"])
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P, I64, I32, U32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32
        lib.or_scan.restype = I64
        lib.or_scan.argtypes = [P, P, U32, P, P, P, P, P, I32, P, I64, I32]
        lib.or_tm.restype = None
        lib.or_tm.argtypes = [P, P, P, I64, P, P, P, P, P, P, I32]
        lib.or_pair.restype = I64
        lib.or_pair.argtypes = [P, I64, P, P, P, P, P, P, I64]
        lib.or_fetch.restype = I64
        lib.or_fetch.argtypes = [P, P, P, I64, P, I64, P]
        lib.or_window_mismatches.restype = I32
        lib.or_window_mismatches.argtypes = [P, ctypes.c_char_p, I32]
        lib.or_duplex_tm.restype = ctypes.c_double
        lib.or_duplex_tm.argtypes = [ctypes.c_char_p, ctypes.c_char_p, P, P]
        lib.or_default_table.restype = None
        lib.or_default_table.argtypes = [P]
        lib.or_degeneracy.restype = I64
        lib.or_degeneracy.argtypes = [ctypes.c_char_p]
        lib.or_edit_distance.restype = I64
        lib.or_edit_distance.argtypes = [ctypes.c_char_p, I64, ctypes.c_char_p, I64]
        lib.or_hmm_build.restype = I64
        lib.or_hmm_build.argtypes = [P, P, I64, P, P, P]
        lib.or_hmm_viterbi.restype = ctypes.c_double
        lib.or_hmm_viterbi.argtypes = [P, P, I64, ctypes.c_char_p, I64]
        lib.or_hmm_forward.restype = ctypes.c_double
        lib.or_hmm_forward.argtypes = [P, P, I64, ctypes.c_char_p, I64]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _cstr_array(strs):
    arr = (ctypes.c_char_p * max(1, len(strs)))()
    for i, s in enumerate(strs):
        arr[i] = s.encode() if isinstance(s, str) else s
    return arr


def _as_pairs(pairs):
    """pairs: list of dicts with keys fwd, rev, k, clamp, min_len, max_len, tm params."""
    return pairs if isinstance(pairs, (list, tuple)) else [pairs]


def tm_params(p: dict) -> TmParams:
    return TmParams(p.get("dnac1_nM", 25.0), p.get("dnac2_nM", 25.0), p.get("Na_mM", 50.0),
                    p.get("K_mM", 0.0), p.get("Tris_mM", 0.0), p.get("Mg_mM", 0.0),
                    p.get("dNTPs_mM", 0.0), p.get("tm_min", float("-inf")),
                    int(p.get("saltcorr", 5)), 0)


def scan(seq: np.ndarray, contig_off: np.ndarray, contig_genome: np.ndarray, pairs, n_threads: int = 0):
    """Sites of every pair, canonical order (pair, contig, pos, primer, strand)."""
    lib = _load()
    pairs = _as_pairs(pairs)
    seq = np.ascontiguousarray(seq, dtype=np.uint8)
    contig_off = np.ascontiguousarray(contig_off, dtype=np.uint64)
    contig_genome = np.ascontiguousarray(contig_genome, dtype=np.uint32)
    fwd = _cstr_array([p["fwd"] for p in pairs])
    rev = _cstr_array([p["rev"] for p in pairs])
    k = np.array([p["k"] for p in pairs], dtype=np.int32)
    clamp = np.array([p.get("clamp", 0) for p in pairs], dtype=np.int32)
    nc = len(contig_off) - 1
    n = lib.or_scan(_ptr(seq), _ptr(contig_off), nc, _ptr(contig_genome), fwd, rev, _ptr(k), _ptr(clamp),
                    len(pairs), None, 0, n_threads)
    out = np.zeros(n, dtype=SITE_DTYPE)
    if n:
        m = lib.or_scan(_ptr(seq), _ptr(contig_off), nc, _ptr(contig_genome), fwd, rev, _ptr(k), _ptr(clamp),
                        len(pairs), _ptr(out), n, n_threads)
        assert m == n
    return out


def tm(seq, contig_off, sites: np.ndarray, pairs, table: NNTable | None = None, n_threads: int = 0):
    """(max Tm in deg C as float64, pass flag Tm >= tm_min as uint8) per site."""
    lib = _load()
    pairs = _as_pairs(pairs)
    seq = np.ascontiguousarray(seq, dtype=np.uint8)
    contig_off = np.ascontiguousarray(contig_off, dtype=np.uint64)
    sites = np.ascontiguousarray(sites, dtype=SITE_DTYPE)
    fwd = _cstr_array([p["fwd"] for p in pairs])
    rev = _cstr_array([p["rev"] for p in pairs])
    params = (TmParams * len(pairs))(*[tm_params(p) for p in pairs])
    tm_out = np.zeros(len(sites), dtype=np.float64)
    pass_out = np.zeros(len(sites), dtype=np.uint8)
    if len(sites):
        lib.or_tm(_ptr(seq), _ptr(contig_off), _ptr(sites), len(sites), fwd, rev, params,
                  ctypes.byref(table) if table is not None else None, _ptr(tm_out), _ptr(pass_out), n_threads)
    return tm_out, pass_out


def pair(sites: np.ndarray, pairs, passed: np.ndarray | None = None):
    """Amplicons, canonical order (pair, contig, start, end, orient)."""
    lib = _load()
    pairs = _as_pairs(pairs)
    sites = np.ascontiguousarray(sites, dtype=SITE_DTYPE)
    Lf = np.array([len(p["fwd"]) for p in pairs], dtype=np.int32)
    Lr = np.array([len(p["rev"]) for p in pairs], dtype=np.int32)
    mn = np.array([p["min_len"] for p in pairs], dtype=np.int32)
    mx = np.array([p["max_len"] for p in pairs], dtype=np.int32)
    pp = None
    if passed is not None:
        passed = np.ascontiguousarray(passed, dtype=np.uint8)
        pp = _ptr(passed)
    n = lib.or_pair(_ptr(sites), len(sites), pp, _ptr(Lf), _ptr(Lr), _ptr(mn), _ptr(mx), None, 0)
    out = np.zeros(n, dtype=AMPLICON_DTYPE)
    if n:
        m = lib.or_pair(_ptr(sites), len(sites), pp, _ptr(Lf), _ptr(Lr), _ptr(mn), _ptr(mx), _ptr(out), n)
        assert m == n
    return out


def fetch(seq, contig_off, amplicons: np.ndarray):
    """(concatenated sequences as bytes, offsets[n+1])."""
    lib = _load()
    seq = np.ascontiguousarray(seq, dtype=np.uint8)
    contig_off = np.ascontiguousarray(contig_off, dtype=np.uint64)
    amplicons = np.ascontiguousarray(amplicons, dtype=AMPLICON_DTYPE)
    offsets = np.zeros(len(amplicons) + 1, dtype=np.uint64)
    total = lib.or_fetch(_ptr(seq), _ptr(contig_off), _ptr(amplicons), len(amplicons), None, 0, _ptr(offsets))
    out = np.zeros(max(1, total), dtype=np.uint8)
    lib.or_fetch(_ptr(seq), _ptr(contig_off), _ptr(amplicons), len(amplicons), _ptr(out), total, _ptr(offsets))
    return out[:total].tobytes(), offsets


def amplitypes(seq, contig_off, amplicons: np.ndarray):
    """Amplicon sequence variants and amplitypes (Sec. 3.3, Amplicon Pattern
    Visualization): a variant is an exact amplicon sequence as fetch() gives it
    (RF reverse-complemented, non-ACGT as N), numbered 0, 1, ... by first
    occurrence in `amplicons`; a genome's amplitype is its multiset of
    (variant, copy number), numbered by first occurrence over the genomes with
    amplicons in ascending id.  Returns (variant id per amplicon, rows
    (genome, amplitype, amplicons, variants) in ascending genome, number of
    variants, number of amplitypes)."""
    seqs, offs = fetch(seq, contig_off, amplicons)
    var = {}
    vid = [var.setdefault(seqs[int(offs[i]):int(offs[i + 1])], len(var)) for i in range(len(amplicons))]
    per = {}
    for g, v in zip(amplicons["genome"].tolist(), vid):
        per.setdefault(g, {}).setdefault(v, 0)
        per[g][v] += 1
    types = {}
    rows = []
    for g in sorted(per):
        pattern = frozenset(per[g].items())
        rows.append((g, types.setdefault(pattern, len(types)), sum(per[g].values()), len(per[g])))
    return np.array(vid, dtype=np.uint32), rows, len(var), len(types)


def reverse_contigs(seq: np.ndarray, contig_off: np.ndarray) -> np.ndarray:
    """The decoy collection (Sec. 2.1, Amplicon analysis): every contig reversed,
    not complemented, in place of the original; contig offsets unchanged."""
    seq = np.asarray(seq, dtype=np.uint8)
    out = np.empty_like(seq)
    for a, b in zip(contig_off[:-1], contig_off[1:]):
        out[int(a):int(b)] = seq[int(a):int(b)][::-1]
    return out


def window_mismatches(window: bytes, primer: str, strand: int) -> int:
    buf = np.frombuffer(window, dtype=np.uint8).copy()
    return _load().or_window_mismatches(_ptr(buf), primer.encode(), strand)


def duplex_tm(oligo: str, bottom: str, params: dict, table: NNTable | None = None) -> float:
    """Tm of one explicit duplex; bottom[i] is the template base opposite oligo[i]."""
    p = tm_params(params)
    return _load().or_duplex_tm(oligo.encode(), bottom.encode(),
                                ctypes.byref(table) if table is not None else None, ctypes.byref(p))


def default_table() -> NNTable:
    t = NNTable()
    _load().or_default_table(ctypes.byref(t))
    return t


def degeneracy(primer: str) -> int:
    return int(_load().or_degeneracy(primer.encode()))


# ---------------------------------------------------------------- profile HMM (hmm.c)
def edit_distance(s: str, r: str) -> int:
    """Unit-cost global alignment distance (0 only for equal A/C/G/T letters)."""
    return int(_load().or_edit_distance(s.encode(), len(s), r.encode(), len(r)))


def hmm_build(seqs):
    """Profile from training sequences (list of str): (reference index, t, e) with
    t[j, X, Y] the transition scores (X, Y in M, I, D; Y = M is the next move, E
    at j = m) and e[j, x] the match emission scores (j = 1..m), in bits."""
    lib = _load()
    data = "".join(seqs).encode()
    off = np.zeros(len(seqs) + 1, dtype=np.uint64)
    off[1:] = np.cumsum([len(x) for x in seqs])
    buf = np.frombuffer(data, dtype=np.uint8).copy() if data else np.zeros(1, np.uint8)
    m = ctypes.c_int64()
    ref = lib.or_hmm_build(_ptr(buf), _ptr(off), len(seqs), ctypes.byref(m), None, None)
    if ref < 0:
        raise ValueError("no training sequence")
    t = np.zeros((m.value + 1, 3, 3), dtype=np.float64)
    e = np.zeros((m.value + 1, 4), dtype=np.float64)
    lib.or_hmm_build(_ptr(buf), _ptr(off), len(seqs), ctypes.byref(m), _ptr(t), _ptr(e))
    return int(ref), t, e


def hmm_viterbi(t: np.ndarray, e: np.ndarray, seq: str) -> float:
    """Glocal Viterbi log-odds score (bits) of seq against the profile (t, e)."""
    t = np.ascontiguousarray(t, dtype=np.float64)
    e = np.ascontiguousarray(e, dtype=np.float64)
    return float(_load().or_hmm_viterbi(_ptr(t), _ptr(e), t.shape[0] - 1, seq.encode(), len(seq)))


def hmm_forward(t: np.ndarray, e: np.ndarray, seq: str) -> float:
    """Glocal Forward log-odds score (bits) of seq against the profile (t, e):
    log2 of the sum over every state path of 2^(path score)."""
    t = np.ascontiguousarray(t, dtype=np.float64)
    e = np.ascontiguousarray(e, dtype=np.float64)
    return float(_load().or_hmm_forward(_ptr(t), _ptr(e), t.shape[0] - 1, seq.encode(), len(seq)))
