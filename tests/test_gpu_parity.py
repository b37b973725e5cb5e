"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer results -- sites, mismatch counts, amplicons, pass flags, sequences
-- must be identical; the fp32 Tm must be within 0.01 deg C of the oracle's
fp64 value (NaN where the oracle has NaN).  Inputs are seeded synthetic
workloads; nothing here is produced by the CUDA path and then trusted.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2509_13300_gb300 import ah, build, synth

pytestmark = pytest.mark.gpu
TM_TOL = 0.01  # deg C


@pytest.fixture(scope="module")
def ctx():
    build.build()
    c = ah.Context(0)
    yield c
    c.close()


def gpu_run(ctx, w, table=None):
    sid = ctx.load(w.seq, w.contig_off, w.contig_genome)
    try:
        pids = [ctx.ah_set_primers(p["fwd"], p["rev"], p) for p in w.pairs]
        if table is not None:
            for p in pids:
                ctx.ah_set_nn_table(p, table)
        sites = ctx.scan(sid, pids)
        tm, ps = ctx.tm(sid, pids, sites)
        amps = ctx.pair(sid, pids, sites)
        amps_tm = ctx.pair(sid, pids, sites, ps)
        seqs, offs = ctx.fetch(sid, amps)
    finally:
        ctx.ah_unload_genomes(sid)
    return dict(sites=sites, tm=tm, pass_=ps, amps=amps, amps_tm=amps_tm, seqs=seqs, offs=offs)


def oracle_run(w, table=None):
    sites = oracle.scan(w.seq, w.contig_off, w.contig_genome, w.pairs)
    tm, ps = oracle.tm(w.seq, w.contig_off, sites, w.pairs, table)
    amps = oracle.pair(sites, w.pairs)
    amps_tm = oracle.pair(sites, w.pairs, ps)
    seqs, offs = oracle.fetch(w.seq, w.contig_off, amps)
    return dict(sites=sites, tm=tm, pass_=ps, amps=amps, amps_tm=amps_tm, seqs=seqs, offs=offs)


def assert_parity(g, o, min_sites=1):
    assert len(g["sites"]) == len(o["sites"]), (len(g["sites"]), len(o["sites"]))
    assert len(o["sites"]) >= min_sites
    assert g["sites"].tobytes() == o["sites"].tobytes()
    tg, to = g["tm"].astype(np.float64), o["tm"]
    nan_g, nan_o = np.isnan(tg), np.isnan(to)
    assert np.array_equal(nan_g, nan_o)
    if (~nan_o).any():
        err = np.abs(tg[~nan_o] - to[~nan_o]).max()
        assert err <= TM_TOL, err
    assert np.array_equal(g["pass_"], o["pass_"])
    assert g["amps"].tobytes() == o["amps"].tobytes()
    assert g["amps_tm"].tobytes() == o["amps_tm"].tobytes()
    assert np.array_equal(g["offs"], o["offs"])
    assert g["seqs"] == o["seqs"]


def test_tiny_workload(ctx):
    """Plain method, tiny: 200 kbp, 3 contigs, 10 planted amplicons, k = 2."""
    w = synth.tiny(0)
    o = oracle_run(w)
    assert_parity(gpu_run(ctx, w), o, min_sites=10)
    # the same with the paper's default 50 deg C threshold (Sec. 3.2)
    w.pairs = [dict(w.pairs[0], tm_min=50.0)]
    o2 = oracle_run(w)
    assert 0 < o2["pass_"].sum() < len(o2["pass_"]) or len(o2["pass_"]) == 0
    assert_parity(gpu_run(ctx, w), o2)


@pytest.mark.parametrize("seed,k,clamp", [(1, 0, 0), (2, 1, 0), (3, 2, 1), (4, 3, 0), (5, 4, 2), (6, 5, 0),
                                          (7, 7, 0), (8, 9, 3), (9, 10, 0)])
def test_random_small_with_edge_letters(ctx, seed, k, clamp):
    """Short primers so hits are frequent; lower case, IUPAC letters and gaps in
    the genome; several contigs including tiny ones; k from 0 to 10."""
    max_len = 900 if k < 4 else 200 if k < 7 else 80
    w = synth.random_small(seed, n_bases=60_000 // (1 + k // 3) + 777 * seed, n_contigs=7, L_f=7 + k + seed % 3,
                           L_r=6 + k + seed % 2, k=k, codes_f="RNY"[: 1 + seed % 3], codes_r="SBD"[: 1 + seed % 3],
                           lower_frac=0.05, iupac_frac=0.003, min_len=30, max_len=max_len)
    w.pairs = [dict(w.pairs[0], clamp=clamp, tm_min=float(seed * 3))]
    assert_parity(gpu_run(ctx, w), oracle_run(w))


@pytest.mark.parametrize("clamp", [0, 3])
def test_longest_primers_with_planted_sites(ctx, clamp):
    """Primers of the longest supported length (32, the width of a window word)
    and 31, planted on both strands with 0..6 substitutions at k = 4, some
    across contig ends and next to no-base runs: the whole path equals the
    oracle."""
    rng = np.random.default_rng(77 + clamp)
    fwd = synth.random_primer(rng, 32, "RYNSW")
    rev = synth.random_primer(rng, 31, "KMY")
    n = 400_000
    g = synth.random_bases(rng, n, 0.5)
    for s0 in rng.integers(0, n - 100, 60):
        g[s0:s0 + int(rng.integers(1, 40))] = ord("N")
    for j in range(80):
        a = int(rng.integers(0, n - 2600))
        f = synth._draw_oligo(rng, fwd, int(rng.integers(0, 7)))
        r = synth._revcomp(synth._draw_oligo(rng, rev, int(rng.integers(0, 7))))
        gap = int(rng.integers(100, 2400))
        left, right = (f, r) if j % 2 == 0 else (r, f)  # FR and RF
        g[a:a + len(left)] = np.frombuffer(left.encode(), np.uint8)
        g[a + 32 + gap:a + 32 + gap + len(right)] = np.frombuffer(right.encode(), np.uint8)
    cuts = np.sort(rng.choice(np.arange(1, n), 6, replace=False)).astype(np.uint64)
    off = np.concatenate([[0], cuts, [n]]).astype(np.uint64)
    w = synth.Workload("longest", g, off, np.zeros(len(off) - 1, np.uint32),
                       [synth.pcr_params(fwd, rev, k=4, min_len=100, max_len=3000, clamp=clamp)],
                       np.zeros(0, dtype=synth.PLANT_DTYPE))
    o = oracle_run(w)
    assert len(o["sites"]) >= 40 and len(o["amps"]) >= 10
    assert_parity(gpu_run(ctx, w), o)


def test_thread_per_site_tm_at_high_degeneracy(ctx):
    """Primers of 8,192 and 4,096 oligos (six N and an R; six N), enough chance
    sites (above 32,768) for the thread-per-site Tm: every site's maximum over
    all oligos within 0.01 C of the oracle's enumeration of every oligo, the
    pass flags exact at a threshold near the median, and the whole path equal."""
    rng = np.random.default_rng(5)
    fwd, rev = "ANCNGNTNANCR", "CNNGNNTANNGC"
    n = 3_200_000
    g = synth.random_bases(rng, n, 0.5)
    off = np.array([0, 400_000, 1_300_000, 2_500_000, n], np.uint64)
    w = synth.Workload("degenerate", g, off, np.zeros(4, np.uint32),
                       [synth.pcr_params(fwd, rev, k=1, min_len=30, max_len=60, tm_min=31.0)],
                       np.zeros(0, dtype=synth.PLANT_DTYPE))
    o = oracle_run(w)
    assert len(o["sites"]) > 32768 and 0.2 < o["pass_"].mean() < 0.8
    assert_parity(gpu_run(ctx, w), o)


def test_k_at_least_length_reports_every_window(ctx):
    w = synth.random_small(21, n_bases=5000, n_contigs=3, L_f=6, L_r=5, k=6, min_len=5, max_len=40)
    assert_parity(gpu_run(ctx, w), oracle_run(w), min_sites=19000)


def test_several_pairs_in_one_pass(ctx):
    rng = np.random.default_rng(5)
    w = synth.random_small(33, n_bases=120_000, n_contigs=5, L_f=12, L_r=10, k=2, min_len=40, max_len=2000)
    pairs = [w.pairs[0]]
    for j in range(4):
        f = synth.random_primer(rng, 10 + j, "RY")
        r = synth.random_primer(rng, 11 + j, "N")
        pairs.append(synth.pcr_params(f, r, k=j % 4, min_len=20 + j, max_len=1500, tm_min=20.0))
    w.pairs = pairs
    assert_parity(gpu_run(ctx, w), oracle_run(w))


def test_many_sites_take_the_thread_per_site_tm_path(ctx):
    """Over 32,768 sites, so ah_tm runs the one-thread-per-site kernel; its
    maximum is within 0.01 C of the oracle's, and with the threshold put
    exactly on an oracle site value (such sites are deferred to the exact
    decision) every pass flag is still the fp64 one."""
    w = synth.random_small(41, n_bases=300_000, n_contigs=4, L_f=11, L_r=10, k=4, codes_f="RYN", codes_r="SWK",
                           min_len=30, max_len=300)
    o = oracle_run(w)
    assert len(o["sites"]) >= 40_000
    ok = ~np.isnan(o["tm"])
    med = float(np.median(o["tm"][ok]))
    at_site = float(o["tm"][ok][np.argmin(np.abs(o["tm"][ok] - med))])
    for thr in (med + 0.003, at_site):
        w.pairs = [dict(w.pairs[0], tm_min=thr)]
        o = oracle_run(w)
        assert 0 < o["pass_"].sum() < len(o["pass_"])
        assert_parity(gpu_run(ctx, w), o)
    # ah_run, twice: the first run overflows the one-synchronisation sizes and
    # finishes step by step; the second (the last count was large) queues only
    # the scan in ah_run_begin and finishes in ah_run_end
    p = w.pairs[0]
    sid = ctx.load(w.seq, w.contig_off, w.contig_genome)
    try:
        pid = ctx.ah_set_primers(p["fwd"], p["rev"], p)
        runs = [ctx.run(sid, [pid], tm_filter=True) for _ in range(2)]
    finally:
        ctx.ah_unload_genomes(sid)
    o_amps = oracle.pair(o["sites"], w.pairs, o["pass_"])
    o_seqs, o_offs = oracle.fetch(w.seq, w.contig_off, o_amps)
    for r in runs:
        assert r["sites"].tobytes() == o["sites"].tobytes()
        assert np.array_equal(r["pass_"], o["pass_"])
        ok = ~np.isnan(o["tm"])
        assert np.abs(r["tm"][ok].astype(np.float64) - o["tm"][ok]).max() <= TM_TOL
        assert r["amps"].tobytes() == o_amps.tobytes() and r["seqs"] == o_seqs


def test_scan_wait_limit_reports_timeout_and_the_context_stays_usable(ctx):
    """Failure detection without a fault: each warp's first slice waits on a
    barrier that no copy will complete (20 us limit); the scan gives up, waits
    for its warps' real copies still in flight and ah_scan returns
    AH_ERR_TIMEOUT; the next scan on the same context is exact."""
    w = synth.random_small(51, n_bases=3_000_000, n_contigs=3, L_f=16, L_r=15, k=2, min_len=30, max_len=900)
    p = w.pairs[0]
    sid = ctx.load(w.seq, w.contig_off, w.contig_genome)
    try:
        pid = ctx.ah_set_primers(p["fwd"], p["rev"], p)
        ctx.debug_scan_stall(True)
        try:
            with pytest.raises(ah.AHError) as e:
                ctx.scan(sid, [pid])
            assert e.value.status == ah.AH_ERR_TIMEOUT
        finally:
            ctx.debug_scan_stall(False)
        sites = ctx.scan(sid, [pid])
    finally:
        ctx.ah_unload_genomes(sid)
    assert sites.tobytes() == oracle.scan(w.seq, w.contig_off, w.contig_genome, w.pairs).tobytes()


def test_full_collection_workload_against_the_oracle(ctx):
    """The whole 100-genome collection workload (0.41 Gbp, 1,777 contigs, the
    960-oligo pair, k = 3, Tm threshold 50 C) through ah_run, against the oracle
    on every genome: sites, pass flags, Tm-filtered amplicons and sequences."""
    import os
    import bench
    w = bench.workload(1, 100)
    p = w.pairs[0]
    sid = ctx.load(w.seq, w.contig_off, w.contig_genome)
    try:
        pid = ctx.ah_set_primers(p["fwd"], p["rev"], p)
        g = ctx.run(sid, [pid], tm_filter=True)
    finally:
        ctx.ah_unload_genomes(sid)
    cores = os.cpu_count() or 1
    s = oracle.scan(w.seq, w.contig_off, w.contig_genome, w.pairs, n_threads=cores)
    tm, ps = oracle.tm(w.seq, w.contig_off, s, w.pairs, n_threads=cores)
    a = oracle.pair(s, w.pairs, ps)
    q, qo = oracle.fetch(w.seq, w.contig_off, a)
    assert len(s) > 5000 and len(a) > 100
    assert g["sites"].tobytes() == s.tobytes()
    ok = ~np.isnan(tm)
    assert np.array_equal(np.isnan(g["tm"]), ~ok)
    assert np.abs(g["tm"][ok].astype(np.float64) - tm[ok]).max() <= TM_TOL
    assert np.array_equal(g["pass_"], ps)
    assert g["amps"].tobytes() == a.tobytes()
    assert g["seqs"] == q and np.array_equal(g["offs"].astype(np.uint64), qo.astype(np.uint64))


@pytest.mark.parametrize("device_input", [False, True])
def test_2bit_load_gives_the_letters(ctx, device_input):
    """ah_load_genomes_2bit over 70 Mbp (two host staging chunks, a tiny
    contig, a contig ending inside a tile, N runs, IUPAC letters, gaps and
    lower case): fetching every contig whole gives the input upper-cased with
    every non-ACGT letter as N, exactly as the ASCII load does."""
    import torch
    rng = np.random.default_rng(23)
    n = 70_000_003
    seq = np.frombuffer(b"ACGT", np.uint8)[rng.integers(0, 4, n)].copy()
    lower = rng.random(n) < 0.01
    seq[lower] += 32
    for s0 in rng.integers(0, n - 200, 3000):  # runs of other letters
        seq[s0:s0 + int(rng.integers(1, 120))] = np.frombuffer(b"NRY-", np.uint8)[int(rng.integers(0, 4))]
    off = np.array([0, 5, 40_000_000, 40_032_781, 69_999_000, n], dtype=np.uint64)
    gen = np.array([0, 0, 1, 1, 2], dtype=np.uint32)
    codes, gaps = ah.encode_2bit(seq)
    src = torch.from_numpy(codes).cuda() if device_input else codes
    amps = np.zeros(len(off) - 1, dtype=ah.AMPLICON_DTYPE)
    amps["genome"] = gen
    amps["contig"] = np.arange(len(off) - 1)
    amps["end"] = np.diff(off.astype(np.int64))
    up = np.where((seq >= 97) & (seq <= 122), seq - 32, seq).astype(np.uint8)
    want = np.where(np.isin(up, np.frombuffer(b"ACGT", np.uint8)), up, ord("N")).astype(np.uint8).tobytes()
    for load in ("2bit", "ascii"):
        if load == "2bit":
            sid = ctx.ah_load_genomes_2bit(src, n, gaps, off, gen)
        else:
            sid = ctx.load(seq, off, gen)
        try:
            got, offs = ctx.fetch(sid, amps)
        finally:
            ctx.ah_unload_genomes(sid)
        assert got == want, load
        assert np.array_equal(offs.astype(np.int64), off.astype(np.int64))


def test_2bit_load_scan_parity(ctx):
    """The whole path on a set loaded from 2-bit codes equals the oracle on the
    letters (short primers, lower case, IUPAC letters and gaps, tiny contigs)."""
    w = synth.random_small(61, n_bases=90_000, n_contigs=7, L_f=9, L_r=8, k=2, codes_f="RN", codes_r="SB",
                           lower_frac=0.05, iupac_frac=0.01, min_len=30, max_len=600)
    codes, gaps = ah.encode_2bit(w.seq)
    sid = ctx.ah_load_genomes_2bit(codes, len(w.seq), gaps, w.contig_off, w.contig_genome)
    try:
        pids = [ctx.ah_set_primers(p["fwd"], p["rev"], p) for p in w.pairs]
        sites = ctx.scan(sid, pids)
        tm, ps = ctx.tm(sid, pids, sites)
        amps = ctx.pair(sid, pids, sites)
        amps_tm = ctx.pair(sid, pids, sites, ps)
        seqs, offs = ctx.fetch(sid, amps)
    finally:
        ctx.ah_unload_genomes(sid)
    g = dict(sites=sites, tm=tm, pass_=ps, amps=amps, amps_tm=amps_tm, seqs=seqs, offs=offs)
    assert_parity(g, oracle_run(w), min_sites=50)


def test_2bit_loads_in_flight_on_two_streams(ctx):
    """Two 2-bit loads queued back to back on two streams, without waiting
    (the batched form's pattern): each set keeps its own no-base runs, so both
    give their letters."""
    import torch
    rng = np.random.default_rng(31)
    seqs, srcs, gapss, offs = [], [], [], []
    for j, n in enumerate((9_000_017, 7_500_001)):
        seq = np.frombuffer(b"ACGT", np.uint8)[rng.integers(0, 4, n)].copy()
        for s0 in rng.integers(0, n - 200, 4000 + 3000 * j):
            seq[s0:s0 + int(rng.integers(1, 60))] = ord("N")
        codes, gaps = ah.encode_2bit(seq)
        seqs.append(seq)
        srcs.append(torch.from_numpy(codes).cuda())
        gapss.append(gaps)
        offs.append(np.array([0, n // 3, n], dtype=np.uint64))
    torch.cuda.synchronize()
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    sids = [ctx.ah_load_genomes_2bit(srcs[j], len(seqs[j]), gapss[j], offs[j], np.zeros(2, np.uint32), streams[j])
            for j in range(2)]
    try:
        for j in range(2):
            amps = np.zeros(2, dtype=ah.AMPLICON_DTYPE)
            amps["contig"] = [0, 1]
            amps["end"] = np.diff(offs[j].astype(np.int64))
            got, _ = ctx.fetch(sids[j], amps)
            want = np.where(seqs[j] == ord("N"), ord("N"), seqs[j]).astype(np.uint8).tobytes()
            assert got == want, j
    finally:
        for sid in sids:
            ctx.ah_unload_genomes(sid)


def test_host_loads_queued_without_waiting(ctx):
    """AH_LOAD_HOST_ASYNC: host loads (2-bit and ASCII, pinned buffers, several
    sets queued back to back on two streams while a run is pending) return
    before their copies finish; every set still gives its letters, and a run on
    each equals the oracle's."""
    import torch
    rng = np.random.default_rng(47)
    w = synth.random_small(62, n_bases=300_000, n_contigs=5, L_f=9, L_r=8, k=2, codes_f="RN", codes_r="SB",
                           min_len=30, max_len=600)
    p = w.pairs[0]
    pid = ctx.ah_set_primers(p["fwd"], p["rev"], p)
    o = oracle_run(w)
    seqs, srcs = [], []
    for j, n in enumerate((5_000_011, 3_200_003, 4_100_000)):
        seq = np.frombuffer(b"ACGTacgt", np.uint8)[rng.integers(0, 8, n)].copy()
        for s0 in rng.integers(0, n - 200, 2000):
            seq[s0:s0 + int(rng.integers(1, 60))] = ord("N")
        seqs.append(seq)
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    # a run in flight on the small set while the big host loads are queued
    sid0 = ctx.load(w.seq, w.contig_off, w.contig_genome)
    sids, keep = [], []
    try:
        for j, seq in enumerate(seqs):
            off = np.array([0, len(seq) // 2, len(seq)], np.uint64)
            if j % 2 == 0:
                codes, gaps = ah.encode_2bit(seq)
                host = torch.from_numpy(codes).pin_memory()
                sids.append(ctx.ah_load_genomes_2bit(host, len(seq), gaps, off, np.zeros(2, np.uint32),
                                                     streams[j % 2], host_async=True))
            else:
                host = torch.from_numpy(seq).pin_memory()
                sids.append(ctx.ah_load_genomes(host, len(seq), off, np.zeros(2, np.uint32), streams[j % 2],
                                                host_async=True))
            keep.append(host)  # unchanged until the set is ready
        r = ctx.run(sid0, [pid], tm_filter=True)
        assert r["sites"].tobytes() == o["sites"].tobytes() and r["amps"].tobytes() == o["amps_tm"].tobytes()
        for j, seq in enumerate(seqs):
            amps = np.zeros(2, dtype=ah.AMPLICON_DTYPE)
            amps["contig"] = [0, 1]
            amps["end"] = [len(seq) // 2, len(seq) - len(seq) // 2]
            got, _ = ctx.fetch(sids[j], amps)
            up = np.where(seq == ord("N"), ord("N"), seq & 0xDF).astype(np.uint8).tobytes()
            assert got == up, j
    finally:
        for sid in sids:
            ctx.ah_unload_genomes(sid)
        ctx.ah_unload_genomes(sid0)
    with pytest.raises(ah.AHError) as e:
        ctx._check(ctx._lib.ah_load_genomes_2bit_ex(ctx.h, ah._ptr(np.zeros(4, np.uint8)), 16, None, 0,
                                                    ah._ptr(np.array([0, 16], np.uint64)), 1,
                                                    ah._ptr(np.zeros(1, np.uint32)), 1, ah.ctypes.byref(
                                                        ah.ctypes.c_uint32()), None))
    assert e.value.status == ah.AH_ERR_ARG  # the reversed flag has no 2-bit form


def test_2bit_load_rejects_bad_gaps(ctx):
    codes = np.zeros(25, np.uint8)
    off, gen = np.array([0, 100], np.uint64), np.zeros(1, np.uint32)
    for bad in ([[10, 0]], [[10, 5], [12, 3]], [[90, 20]], [[50, 5], [10, 5]]):
        with pytest.raises(ah.AHError) as e:
            ctx.ah_load_genomes_2bit(codes, 100, np.array(bad, np.uint64), off, gen)
        assert e.value.status == ah.AH_ERR_ARG


def test_collection_spanning_many_tiles(ctx):
    """Genome-collection generator at reduced size: ~5 Mbp, 6 genomes, many
    contigs, N runs, planted operons with 0-4 substitutions, the 960-oligo pair."""
    w = synth.collection(seed=1, n_genomes=6, len_lo=4e5, len_hi=1.5e6, max_subs=4)
    o = oracle_run(w)
    assert len(o["amps"]) >= 3
    assert_parity(gpu_run(ctx, w), o)


def test_paper_primer_pairs(ctx):
    """The four benchmark pairs printed in the paper (Sec. 2.3) on one collection."""
    pairs = [synth.pcr_params(f, r, k=2, min_len=100, max_len=3000, tm_min=50.0)
             for f, r in synth.PAPER_PAIRS.values()]
    w = synth.collection(seed=4, n_genomes=3, len_lo=3e5, len_hi=8e5, pairs=pairs, plant_max=4, max_subs=2)
    assert_parity(gpu_run(ctx, w), oracle_run(w))


@pytest.mark.parametrize("salt", [0, 1, 5])
def test_salt_methods_and_ions(ctx, salt):
    w = synth.tiny(0)
    w.pairs = [dict(w.pairs[0], saltcorr=salt, K_mM=10.0, Tris_mM=20.0, Mg_mM=1.5, dNTPs_mM=0.2,
                    dnac1_nM=400.0, dnac2_nM=100.0, tm_min=45.0)]
    assert_parity(gpu_run(ctx, w), oracle_run(w))


@pytest.mark.parametrize("salt", [2, 3, 4, 6, 7, -1])
def test_salt_methods_not_offered_are_rejected(ctx, salt):
    """Only the salt methods the oracle pins to published values (0, 1, 5) are offered."""
    p = dict(synth.tiny(0).pairs[0], saltcorr=salt)
    with pytest.raises(ah.AHError) as e:
        ctx.ah_set_primers(p["fwd"], p["rev"], p)
    assert e.value.status == ah.AH_ERR_ARG


def test_custom_nn_table_with_mismatch_terms(ctx):
    """A table with non-zero mismatch stacks and mismatch-specific terminal
    terms, passed to both sides; includes entries that make some duplex
    entropies positive, which forces the enumeration path on the GPU."""
    rng = np.random.default_rng(12)
    t = oracle.default_table()
    ta = ah.NNTable()
    H = np.array(t.stack_dH)
    S = np.array(t.stack_dS)
    zero = (H == 0)
    H[zero] = np.round(rng.uniform(-3, 4, zero.sum()), 1)
    S[zero] = np.round(rng.uniform(-12, 12, zero.sum()), 1)
    TH = np.round(rng.uniform(-1, 3, 16), 1)
    TS = np.round(rng.uniform(-4, 6, 16), 1)
    for tt in (t, ta):
        tt.stack_dH[:] = list(H)
        tt.stack_dS[:] = list(S)
        tt.term_dH[:] = list(TH)
        tt.term_dS[:] = list(TS)
    w = synth.tiny(0)
    w.pairs = [dict(w.pairs[0], tm_min=30.0)]
    g = gpu_run(ctx, w, table=ta)
    o = oracle_run(w, table=t)
    assert_parity(g, o)


def test_threshold_decisions_at_the_boundary(ctx):
    """tm_min set at (and a hair either side of) oracle Tm values: the pass
    flags must still equal the fp64 decisions."""
    w = synth.tiny(0)
    o = oracle_run(w)
    vals = o["tm"][~np.isnan(o["tm"])]
    assert len(vals) > 3
    for v in (vals[0], vals[len(vals) // 2] + 1e-9, vals[-1] - 1e-9):
        w.pairs = [dict(w.pairs[0], tm_min=float(v))]
        assert_parity(gpu_run(ctx, w), oracle_run(w))


def test_threshold_band_decisions(ctx):
    """tm_min placed inside the 0.01 deg C band around site Tm values, at
    offsets from 1e-12 to 9e-3: the pass flags equal the fp64 decisions (the
    fp64 sign test decides most, exhaustive enumeration the closest), and the
    reported Tm stays within 0.01 of the oracle and on the side of its flag."""
    w = synth.tiny(0)
    o_sites = oracle.scan(w.seq, w.contig_off, w.contig_genome, w.pairs)
    o_tm, _ = oracle.tm(w.seq, w.contig_off, o_sites, w.pairs)
    vals = np.unique(o_tm[~np.isnan(o_tm)])
    vals = vals[np.linspace(0, len(vals) - 1, min(5, len(vals))).astype(int)]
    sid = ctx.load(w.seq, w.contig_off, w.contig_genome)
    try:
        p0 = ctx.ah_set_primers(w.pairs[0]["fwd"], w.pairs[0]["rev"], w.pairs[0])
        sites = ctx.scan(sid, [p0])
        assert sites.tobytes() == o_sites.tobytes()
        for v in vals:
            for d in (0.0, 1e-12, -1e-12, 1e-9, -1e-9, 1e-6, -1e-6, 1e-4, -1e-4, 3e-3, -3e-3, 9e-3, -9e-3):
                p = dict(w.pairs[0], tm_min=float(v) + d)
                pid = ctx.ah_set_primers(p["fwd"], p["rev"], p)
                tm, ps = ctx.tm(sid, [pid], sites)
                e_tm, e_ps = oracle.tm(w.seq, w.contig_off, o_sites, [p])
                assert np.array_equal(ps, e_ps), (v, d)
                ok = ~np.isnan(e_tm)
                assert np.abs(tm[ok].astype(np.float64) - e_tm[ok]).max() <= TM_TOL
                tmin = np.float32(p["tm_min"])
                assert np.all((tm[ok] >= tmin) == (ps[ok] == 1)), (v, d)
    finally:
        ctx.ah_unload_genomes(sid)


def test_device_resident_buffers(ctx):
    """Inputs and outputs in device memory (torch CUDA tensors) give the same
    records as host buffers."""
    import torch
    w = synth.tiny(0)
    o = oracle_run(w)
    seq_d = torch.from_numpy(w.seq).cuda()
    sid = ctx.ah_load_genomes(seq_d, len(w.seq), w.contig_off, w.contig_genome)
    pid = ctx.ah_set_primers(w.pairs[0]["fwd"], w.pairs[0]["rev"], w.pairs[0])
    n = len(o["sites"])
    sites_d = torch.zeros(n * 16, dtype=torch.uint8, device="cuda")
    assert ctx.ah_scan(sid, [pid], sites_d, n) == n
    assert sites_d.cpu().numpy().tobytes() == o["sites"].tobytes()
    tm_d = torch.zeros(n, dtype=torch.float32, device="cuda")
    ps_d = torch.zeros(n, dtype=torch.uint8, device="cuda")
    ctx.ah_tm(sid, [pid], sites_d, n, tm_d, ps_d)
    assert np.nanmax(np.abs(tm_d.cpu().numpy() - o["tm"])) <= TM_TOL
    m = len(o["amps"])
    amps_d = torch.zeros(m * 28, dtype=torch.uint8, device="cuda")
    assert ctx.ah_pair(sid, [pid], sites_d, None, n, amps_d, m) == m
    assert amps_d.cpu().numpy().tobytes() == o["amps"].tobytes()
    total = int(o["offs"][-1])
    seq_out = torch.zeros(total, dtype=torch.uint8, device="cuda")
    offs_d = torch.zeros(m + 1, dtype=torch.int64, device="cuda")
    ctx.ah_fetch(sid, amps_d, m, seq_out, total, offs_d)
    assert seq_out.cpu().numpy().tobytes() == o["seqs"]
    assert np.array_equal(offs_d.cpu().numpy().astype(np.uint64), o["offs"])
    ctx.ah_unload_genomes(sid)


def test_errors_are_reported_not_raised_on_device(ctx):
    w = synth.tiny(0)
    p = dict(w.pairs[0])
    with pytest.raises(ah.AHError) as e:
        ctx.ah_set_primers("ACGX", p["rev"], p)
    assert e.value.status == ah.AH_ERR_PRIMER
    with pytest.raises(ah.AHError) as e:
        ctx.ah_set_primers("ACGT", p["rev"], p)  # shorter than 5
    assert e.value.status == ah.AH_ERR_PRIMER
    with pytest.raises(ah.AHError) as e:
        ctx.ah_set_primers("NNNNNNNNNNNN", p["rev"], p)  # degeneracy 4^12 > 10000
    assert e.value.status == ah.AH_ERR_PRIMER
    with pytest.raises(ah.AHError) as e:
        ctx.ah_set_primers(p["fwd"], p["rev"], dict(p, k=11))
    assert e.value.status == ah.AH_ERR_PRIMER
    with pytest.raises(ah.AHError) as e:
        ctx.ah_set_primers(p["fwd"], p["rev"], dict(p, min_len=10, max_len=5))
    assert e.value.status == ah.AH_ERR_ARG
    sid = ctx.load(w.seq, w.contig_off, w.contig_genome)
    pid = ctx.ah_set_primers(p["fwd"], p["rev"], p)
    with pytest.raises(ah.AHError) as e:  # size query: cap = 0 reports the count with AH_ERR_OVERFLOW
        ctx.ah_scan(sid, [pid], None, 0)
    assert e.value.status == ah.AH_ERR_OVERFLOW
    n = e.value.needed
    assert n > 2
    small = np.zeros(n - 1, dtype=ah.SITE_DTYPE)
    with pytest.raises(ah.AHError) as e:
        ctx.ah_scan(sid, [pid], small, n - 1)
    assert e.value.status == ah.AH_ERR_OVERFLOW and e.value.needed == n
    assert not small.view(np.uint8).any()
    with pytest.raises(ah.AHError) as e:
        ctx.ah_scan(sid + 100, [pid], None, 0)
    assert e.value.status == ah.AH_ERR_ARG
    # a site record outside its contig is rejected before any kernel uses it
    bad = np.zeros(1, dtype=ah.SITE_DTYPE)
    bad["contig"] = 2
    bad["pos"] = 10 ** 9
    with pytest.raises(ah.AHError) as e:
        ctx.tm(sid, [pid], bad)
    assert e.value.status == ah.AH_ERR_ARG
    ctx.ah_unload_genomes(sid)
    # the context is still usable afterwards
    assert_parity(gpu_run(ctx, w), oracle_run(w))


def test_memory_budget_is_enforced():
    build.build()
    w = synth.tiny(0)
    with ah.Context(0, mem_budget_bytes=1 << 16) as c:
        with pytest.raises(ah.AHError) as e:
            c.load(w.seq, w.contig_off, w.contig_genome)
        assert e.value.status == ah.AH_ERR_BUDGET
        assert c.device_bytes() < (1 << 16)


def test_empty_and_degenerate_sets(ctx):
    p = synth.tiny(0).pairs[0]
    pid = ctx.ah_set_primers(p["fwd"], p["rev"], p)
    # no bases at all, one empty contig
    sid = ctx.ah_load_genomes(np.zeros(1, np.uint8), 0, np.array([0, 0], np.uint64), np.array([0], np.uint32))
    assert ctx.ah_scan(sid, [pid], None, 0) == 0  # zero sites fit in capacity 0
    ctx.ah_unload_genomes(sid)
    # contigs shorter than the primers, empty contigs in between, all-N contig
    seq = np.frombuffer(b"ACGTACG" + b"N" * 50 + b"ACGT", np.uint8).copy()
    off = np.array([0, 7, 7, 57, 61], np.uint64)
    sid = ctx.ah_load_genomes(seq, len(seq), off, np.array([0, 0, 1, 1], np.uint32))
    assert ctx.ah_scan(sid, [pid], None, 0) == 0
    ctx.ah_unload_genomes(sid)


def test_pack_classifies_every_byte_value(ctx):
    """All 256 byte values, at every offset within a 4-byte word and across
    tile boundaries: exactly A/C/G/T in either case are bases, all else N."""
    rng = np.random.default_rng(3)
    vals = np.tile(np.arange(256, dtype=np.uint8), 600)
    seq = np.concatenate([vals, rng.permutation(vals), np.frombuffer(b"ACGTacgtN" * 5000, np.uint8)])
    off = np.array([0, 70_001, len(seq)], np.uint64)  # a contig boundary inside a word
    sid = ctx.ah_load_genomes(seq, len(seq), off, np.array([0, 1], np.uint32))
    amps = np.zeros(2, dtype=ah.AMPLICON_DTYPE)
    amps["contig"] = [0, 1]
    amps["end"] = [70_001, len(seq) - 70_001]
    got, goff = ctx.fetch(sid, amps)
    want, woff = oracle.fetch(seq, off, amps)
    ctx.ah_unload_genomes(sid)
    assert np.array_equal(goff, woff) and got == want


def test_pack_single_non_bases_in_base_tiles(ctx):
    """Tiles of bases (either case) with single non-base bytes scattered through
    them, at word, row and tile edges: the packer's fast all-bases test must
    send every such column to the exact per-byte test."""
    rng = np.random.default_rng(11)
    n = 7 * 32768 + 1234
    seq = rng.choice(np.frombuffer(b"ACGTacgt", np.uint8), n)
    others = np.array([v for v in range(256) if v not in b"ACGTacgt"], np.uint8)
    edges = [0, 3, 4, 1023, 1024, 31 * 1024, 32767, 32768, 32768 + 31 * 1024 + 1023, 3 * 32768 + 5 * 1024 + 511]
    pos = np.unique(np.concatenate([edges, rng.integers(0, n, 60)]))
    seq[pos] = rng.choice(others, len(pos))
    off = np.array([0, n], np.uint64)
    sid = ctx.ah_load_genomes(seq, n, off, np.array([0], np.uint32))
    amps = np.zeros(1, dtype=ah.AMPLICON_DTYPE)
    amps["end"] = [n]
    got, goff = ctx.fetch(sid, amps)
    want, woff = oracle.fetch(seq, off, amps)
    ctx.ah_unload_genomes(sid)
    assert np.array_equal(goff, woff) and got == want


@pytest.mark.parametrize("tm_filter", [True, False])
def test_run_equals_separate_calls_and_oracle(ctx, tm_filter):
    """ah_run (the fused path) gives the records of ah_scan/ah_tm/ah_pair/ah_fetch
    and of the oracle; too-small outputs are reported, not written."""
    w = synth.collection(seed=2, n_genomes=4, len_lo=3e5, len_hi=9e5)
    w.pairs = [dict(w.pairs[0], tm_min=50.0)]
    o = oracle_run(w)
    sid = ctx.load(w.seq, w.contig_off, w.contig_genome)
    pid = ctx.ah_set_primers(w.pairs[0]["fwd"], w.pairs[0]["rev"], w.pairs[0])
    r = ctx.run(sid, [pid], tm_filter=tm_filter)
    amps = o["amps_tm"] if tm_filter else o["amps"]
    seqs, offs = oracle.fetch(w.seq, w.contig_off, amps)
    assert r["sites"].tobytes() == o["sites"].tobytes()
    assert np.array_equal(r["pass_"], o["pass_"])
    ok = ~np.isnan(o["tm"])
    assert np.array_equal(np.isnan(r["tm"]), ~ok) and np.abs(r["tm"][ok] - o["tm"][ok]).max() <= TM_TOL
    assert r["amps"].tobytes() == amps.tobytes() and len(amps) > 0
    assert r["seqs"] == seqs and np.array_equal(r["offs"], offs)
    # capacity one short on the amplicons: counts reported, sites still written
    n, m = len(r["sites"]), len(r["amps"])
    sites = np.zeros(n, dtype=ah.SITE_DTYPE)
    small = np.zeros(m, dtype=ah.AMPLICON_DTYPE)
    out = ah.RunOut(sites.ctypes.data, n, 0, None, None, small.ctypes.data, m - 1, 0, None, 0, 0, None,
                    1 if tm_filter else 0, 0)
    with pytest.raises(ah.AHError) as e:
        ctx.ah_run(sid, [pid], out)
    assert e.value.status == ah.AH_ERR_OVERFLOW
    assert out.n_sites == n and out.n_amplicons == m and out.n_seq == len(seqs)
    assert sites.tobytes() == o["sites"].tobytes() and not small.view(np.uint8).any()
    ctx.ah_unload_genomes(sid)


def test_many_sites_take_the_device_wide_paths(ctx):
    """More than 16384 sites (device-wide sort instead of the one-block sort)
    and more than 65536 values in the pairing prefix sum (device-wide scan)."""
    w = synth.random_small(41, n_bases=20_000, n_contigs=8, L_f=6, L_r=5, k=6, min_len=12, max_len=12)
    o = oracle_run(w)
    assert len(o["sites"]) > 65536
    assert_parity(gpu_run(ctx, w), o)


def _run_into_device(ctx, sid, pid, caps, tm_filter=True):
    """ah_run into device buffers (torch) with the given capacities (sites,
    amplicons, sequence bytes); returns (status, out struct, host copies)."""
    import torch
    ns, na, nq = caps
    u8 = dict(dtype=torch.uint8, device="cuda")
    b = dict(sites=torch.zeros(max(ns, 1) * 16, **u8), tm=torch.zeros(max(ns, 1), dtype=torch.float32, device="cuda"),
             ps=torch.zeros(max(ns, 1), **u8), amps=torch.zeros(max(na, 1) * 28, **u8),
             seq=torch.zeros(max(nq, 1), **u8), offs=torch.zeros(max(na, 1) + 1, dtype=torch.int64, device="cuda"))
    out = ah.RunOut(b["sites"].data_ptr(), ns, 0, b["tm"].data_ptr(), b["ps"].data_ptr(), b["amps"].data_ptr(), na, 0,
                    b["seq"].data_ptr(), nq, 0, b["offs"].data_ptr(), 1 if tm_filter else 0, 0)
    status = ah.AH_OK
    try:
        ctx.ah_run(sid, [pid], out)
    except ah.AHError as e:
        status = e.status
    torch.cuda.synchronize()
    return status, out, {k: v.cpu().numpy() for k, v in b.items()}


def test_run_into_device_buffers_and_every_fallback(ctx):
    """ah_run with device outputs: generous and exact capacities take the
    one-synchronisation path; a capacity one short on any output is reported
    with the true counts (the step-by-step path), and the next call with room
    is exact again."""
    w = synth.collection(seed=3, n_genomes=3, len_lo=3e5, len_hi=9e5)
    w.pairs = [dict(w.pairs[0], tm_min=50.0)]
    o = oracle_run(w)
    n, m = len(o["sites"]), len(o["amps_tm"])
    seqs, offs = oracle.fetch(w.seq, w.contig_off, o["amps_tm"])
    q = len(seqs)
    assert n > 0 and m > 0
    sid = ctx.load(w.seq, w.contig_off, w.contig_genome)
    pid = ctx.ah_set_primers(w.pairs[0]["fwd"], w.pairs[0]["rev"], w.pairs[0])

    def check_all(b):
        assert b["sites"][:16 * n].tobytes() == o["sites"].tobytes()
        assert np.array_equal(b["ps"][:n], o["pass_"])
        assert b["amps"][:28 * m].tobytes() == o["amps_tm"].tobytes()
        assert b["seq"][:q].tobytes() == seqs
        assert np.array_equal(b["offs"][:m + 1].astype(np.uint64), offs)

    for caps in [(n + 100, m + 100, q + 100), (n, m, q), (20000, 60000, 1 << 22)]:
        st, out, b = _run_into_device(ctx, sid, pid, caps)
        assert st == ah.AH_OK and (out.n_sites, out.n_amplicons, out.n_seq) == (n, m, q)
        check_all(b)
    for short in range(3):
        caps = [n, m, q]
        caps[short] -= 1
        st, out, b = _run_into_device(ctx, sid, pid, tuple(caps))
        assert st == ah.AH_ERR_OVERFLOW and (out.n_sites, out.n_amplicons, out.n_seq) == (n, m, q)
        if short != 0:
            assert b["sites"][:16 * n].tobytes() == o["sites"].tobytes()
    st, out, b = _run_into_device(ctx, sid, pid, (n, m, q))
    assert st == ah.AH_OK
    check_all(b)
    ctx.ah_unload_genomes(sid)


@pytest.mark.parametrize("case", ["sites_above_16384", "amplicons_above_16384", "amplicons_above_65535"])
def test_run_past_the_one_synchronisation_sizes(ctx, case):
    """Counts above what the one-synchronisation launches are sized for
    (sites, amplicons, sequence bytes) finish on the step-by-step path with
    the oracle's records, on the first call and on repeated calls; a small
    workload afterwards is exact again."""
    if case == "sites_above_16384":
        w = synth.random_small(41, n_bases=20_000, n_contigs=8, L_f=6, L_r=5, k=6, min_len=12, max_len=12)
    elif case == "amplicons_above_16384":
        w = synth.random_small(7, n_bases=120_000, n_contigs=1, L_f=5, L_r=5, k=1, codes_f="R", codes_r="Y",
                               min_len=12, max_len=100)
    else:
        w = synth.random_small(9, n_bases=100_000, n_contigs=1, L_f=5, L_r=5, k=1, codes_f="R", codes_r="Y",
                               min_len=10, max_len=250)
    o = oracle_run(w)
    seqs, offs = oracle.fetch(w.seq, w.contig_off, o["amps_tm"])
    sid = ctx.load(w.seq, w.contig_off, w.contig_genome)
    pid = ctx.ah_set_primers(w.pairs[0]["fwd"], w.pairs[0]["rev"], w.pairs[0])
    for _ in range(2):
        r = ctx.run(sid, [pid], tm_filter=True)
        assert r["sites"].tobytes() == o["sites"].tobytes()
        assert np.array_equal(r["pass_"], o["pass_"])
        assert r["amps"].tobytes() == o["amps_tm"].tobytes()
        assert r["seqs"] == seqs and np.array_equal(r["offs"], offs)
    ctx.ah_unload_genomes(sid)
    t = synth.tiny(0)
    ot = oracle_run(t)
    sid = ctx.load(t.seq, t.contig_off, t.contig_genome)
    pid = ctx.ah_set_primers(t.pairs[0]["fwd"], t.pairs[0]["rev"], t.pairs[0])
    r = ctx.run(sid, [pid], tm_filter=False)
    assert r["sites"].tobytes() == ot["sites"].tobytes() and r["amps"].tobytes() == ot["amps"].tobytes()
    ctx.ah_unload_genomes(sid)


@pytest.mark.parametrize("source", ["device", "host"])
def test_run_begin_end_pipeline(ctx, source):
    """ah_run_begin / ah_run_end give ah_run's records; while a run is pending
    other calls are refused; three sets run as a pipeline (the next set packs on
    a second stream after the current scan, or, from host memory, is copied
    and packed while the run computes) each match the oracle."""
    import torch
    ws = [synth.collection(seed=s, n_genomes=2, len_lo=3e5, len_hi=6e5) for s in (4, 5, 6)]
    pair = dict(ws[0].pairs[0], tm_min=50.0)  # one pair for every set (the generator draws one per seed)
    for w in ws:
        w.pairs = [pair]
    p = ws[0].pairs[0]
    pid = ctx.ah_set_primers(p["fwd"], p["rev"], p)
    want = []
    for w in ws:
        o = oracle_run(w)
        seqs, offs = oracle.fetch(w.seq, w.contig_off, o["amps_tm"])
        want.append((o, seqs, offs))
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    scan_done = torch.cuda.Event()
    dev = [torch.from_numpy(w.seq).cuda() for w in ws] if source == "device" else [w.seq for w in ws]
    torch.cuda.synchronize()
    cap = 20000
    u8 = dict(dtype=torch.uint8, device="cuda")
    b = dict(sites=torch.zeros(cap * 16, **u8), tm=torch.zeros(cap, dtype=torch.float32, device="cuda"),
             ps=torch.zeros(cap, **u8), amps=torch.zeros(cap * 28, **u8), seq=torch.zeros(1 << 22, **u8),
             offs=torch.zeros(cap + 1, dtype=torch.int64, device="cuda"))
    out = ah.RunOut(b["sites"].data_ptr(), cap, 0, b["tm"].data_ptr(), b["ps"].data_ptr(), b["amps"].data_ptr(), cap,
                    0, b["seq"].data_ptr(), 1 << 22, 0, b["offs"].data_ptr(), 1, 0)
    prev = ctx.ah_load_genomes(dev[0], len(ws[0].seq), ws[0].contig_off, ws[0].contig_genome, streams[0])
    total_amps = 0
    for i, w in enumerate(ws):
        ctx.ah_run_begin(prev, [pid], out, streams[i % 2], scan_done)
        with pytest.raises(ah.AHError) as e:  # refused while the run is pending
            ctx.ah_scan(prev, [pid], None, 0)
        assert e.value.status == ah.AH_ERR_ARG
        nxt = None
        if i + 1 < len(ws):
            if source == "device":
                streams[(i + 1) % 2].wait_event(scan_done)
            nxt = ctx.ah_load_genomes(dev[i + 1], len(ws[i + 1].seq), ws[i + 1].contig_off,
                                      ws[i + 1].contig_genome, streams[(i + 1) % 2])
        ctx.ah_run_end(out)
        torch.cuda.synchronize()
        o, seqs, offs = want[i]
        n, m, q = out.n_sites, out.n_amplicons, out.n_seq
        assert b["sites"][:16 * n].cpu().numpy().tobytes() == o["sites"].tobytes()
        assert np.array_equal(b["ps"][:n].cpu().numpy(), o["pass_"])
        assert b["amps"][:28 * m].cpu().numpy().tobytes() == o["amps_tm"].tobytes()
        total_amps += m
        assert b["seq"][:q].cpu().numpy().tobytes() == seqs
        assert np.array_equal(b["offs"][:m + 1].cpu().numpy().astype(np.uint64), offs)
        ctx.ah_unload_genomes(prev)
        prev = nxt
    assert total_amps > 0  # the first set carries planted amplicons of this pair
    with pytest.raises(ah.AHError):  # nothing pending
        ctx.ah_run_end(out)


@pytest.mark.parametrize("on_device", [False, True])
def test_decoy_sets_on_reversed_contigs(ctx, on_device):
    """A reversed (decoy) load gives, through every call and ah_run, the oracle's
    records on the contig-wise reversed collection; the off-target rate is the
    ratio of decoy to real amplicons."""
    import torch
    w = synth.collection(seed=2, n_genomes=4, len_lo=3e5, len_hi=9e5)
    w.pairs = [dict(w.pairs[0], tm_min=40.0)]
    rev = oracle.reverse_contigs(w.seq, w.contig_off)
    wr = synth.Workload(**{**w.__dict__, "seq": rev})
    o = oracle_run(wr)
    seq_in = torch.from_numpy(w.seq).cuda() if on_device else w.seq
    sid = ctx.ah_load_genomes(seq_in, len(w.seq), w.contig_off, w.contig_genome, reversed=True)
    try:
        pid = ctx.ah_set_primers(w.pairs[0]["fwd"], w.pairs[0]["rev"], w.pairs[0])
        sites = ctx.scan(sid, [pid])
        assert sites.tobytes() == o["sites"].tobytes() and len(sites) > 0
        tm, ps = ctx.tm(sid, [pid], sites)
        assert np.array_equal(ps, o["pass_"])
        ok = ~np.isnan(o["tm"])
        assert np.abs(tm[ok] - o["tm"][ok]).max() <= TM_TOL
        amps = ctx.pair(sid, [pid], sites)
        assert amps.tobytes() == o["amps"].tobytes()
        seqs, offs = ctx.fetch(sid, amps)
        assert seqs == o["seqs"] and np.array_equal(offs, o["offs"])
        r = ctx.run(sid, [pid], tm_filter=True)
        assert r["amps"].tobytes() == o["amps_tm"].tobytes()
    finally:
        ctx.ah_unload_genomes(sid)
    real = oracle.pair(oracle.scan(w.seq, w.contig_off, w.contig_genome, w.pairs), w.pairs)
    assert len(real) > 0
    rate = len(o["amps"]) / len(real)  # the off-target estimate this load supports
    assert 0.0 <= rate


def test_tm_threshold_sweep(ctx):
    """ah_tm_sweep: per threshold, the amplicons whose two sites pass, those that
    are FF/RR, and the genomes amplified, equal to the oracle's fp64 decisions --
    on a grid and at thresholds placed on (and within 1e-7 of) site Tm values."""
    w = synth.collection(seed=2, n_genomes=6, len_lo=3e5, len_hi=9e5)
    pair = w.pairs[0]
    sites = oracle.scan(w.seq, w.contig_off, w.contig_genome, [pair])
    amps = oracle.pair(sites, [pair])
    tm64, _ = oracle.tm(w.seq, w.contig_off, sites, [pair])
    fin = np.unique(tm64[~np.isnan(tm64)])
    picks = fin[np.linspace(0, len(fin) - 1, 6).astype(int)]
    thr = list(np.arange(20.0, 72.0, 2.0)) + [float(v) for v in picks]
    thr += [float(picks[2]) + 1e-7, float(picks[3]) - 1e-7, float(picks[4]) + 1e-12]
    assert len(thr) <= 64
    want = []
    for T in thr:
        ok = tm64 >= T  # NaN compares false: fails every threshold
        live = ok[amps["left"]] & ok[amps["right"]]
        want.append((int(live.sum()), int((live & (amps["orient"] >= 2)).sum()),
                     len(set(amps["genome"][live].tolist()))))
    sid = ctx.load(w.seq, w.contig_off, w.contig_genome)
    try:
        pid = ctx.ah_set_primers(pair["fwd"], pair["rev"], pair)
        g_sites = ctx.scan(sid, [pid])
        assert g_sites.tobytes() == sites.tobytes()
        g_amps = ctx.pair(sid, [pid], g_sites)
        assert g_amps.tobytes() == amps.tobytes() and len(amps) > 0
        rows, n_genomes = ctx.ah_tm_sweep(sid, [pid], g_sites, g_amps, thr)
    finally:
        ctx.ah_unload_genomes(sid)
    assert n_genomes == len(set(w.contig_genome.tolist()))
    got = [tuple(int(x) for x in r) for r in rows]
    assert got == want
    assert want[0][0] > want[-10][0]  # the counts do move with the threshold


@pytest.mark.parametrize("case", ["collection", "repeats"])
def test_amplicon_variants_and_amplitypes(ctx, case):
    """ah_amplitypes: variant ids and per-genome amplitypes equal the plain
    definition on the fetched sequences (exact sequence identity)."""
    if case == "collection":
        w = synth.collection(seed=8, n_genomes=12, len_lo=2e5, len_hi=6e5)
    else:  # short primers on repeated genomes: many equal sequences and shared patterns
        base = synth.random_small(3, n_bases=30_000, n_contigs=2, L_f=6, L_r=6, k=1, min_len=20, max_len=300)
        reps = 5
        seq = np.concatenate([base.seq] * reps)
        n0 = len(base.seq)
        off = np.concatenate([base.contig_off[:-1] + r * n0 for r in range(reps)] + [[reps * n0]]).astype(np.uint64)
        gen = np.repeat(np.arange(reps, dtype=np.uint32), len(base.contig_off) - 1)
        seq[n0 + 100:n0 + 110] = ord("N")  # genome 1 differs a little
        w = synth.Workload(**{**base.__dict__, "seq": seq, "contig_off": off, "contig_genome": gen})
    pair = w.pairs[0]
    sites = oracle.scan(w.seq, w.contig_off, w.contig_genome, [pair])
    amps = oracle.pair(sites, [pair])
    assert len(amps) > 3
    want_v, want_rows, want_nv, want_nt = oracle.amplitypes(w.seq, w.contig_off, amps)
    sid = ctx.load(w.seq, w.contig_off, w.contig_genome)
    try:
        variant, rows, nv, nt = ctx.amplitypes(sid, amps)
    finally:
        ctx.ah_unload_genomes(sid)
    assert np.array_equal(variant, want_v)
    assert [tuple(int(x) for x in r) for r in rows] == want_rows
    assert (nv, nt) == (want_nv, want_nt)
    if case == "repeats":
        assert nt < len(want_rows)  # some genomes share an amplitype


def test_device_generator_matches_cpu_twin(ctx):
    """ah_generate_bases writes, on the device, the same bytes as the CPU twin,
    for the whole collection and for ranges at other offsets."""
    import torch
    from paper_2509_13300_gb300 import countergen
    c = countergen.collection(seed=7, n_genomes=6, len_lo=2e5, len_hi=8e5)
    want = c.bases()
    out = torch.zeros(c.n_bases, dtype=torch.uint8, device="cuda")
    ctx.generate_bases(c, 0, c.n_bases, out)
    assert out.cpu().numpy().tobytes() == want.tobytes()
    for a, n in ((4, 1), (8, 4099), (40000, 123457), (c.n_bases - 1001 - (c.n_bases - 1001) % 4, 1001)):
        part = torch.zeros(n, dtype=torch.uint8, device="cuda")
        ctx.generate_bases(c, a, n, part)
        assert part.cpu().numpy().tobytes() == want[a:a + n].tobytes()
    with pytest.raises(ah.AHError):  # base0 not a multiple of 4
        ctx.generate_bases(c, 3, 10, out)
    # the same from the collection's tables on the device (stream-ordered calls)
    tables = ctx.device_tables(c)
    out.zero_()
    ctx.generate_bases(c, 0, c.n_bases, out, tables=tables)
    torch.cuda.synchronize()
    assert out.cpu().numpy().tobytes() == want.tobytes()
    for a, n in ((8, 4099), (40000, 123457)):
        part = torch.zeros(n, dtype=torch.uint8, device="cuda")
        ctx.generate_bases(c, a, n, part, tables=tables)
        torch.cuda.synchronize()
        assert part.cpu().numpy().tobytes() == want[a:a + n].tobytes()


def test_large_workload_shape_on_device_generated_genomes(ctx):
    """The large workload's shape (counter-generated genomes, k = 4, window
    100-3000, pairs of 960, 64 and 256 oligos scanned in one pass) on a small
    seed-7 collection generated on the device: sites, Tm and amplicons equal the
    oracle's on the CPU twin's bytes."""
    import torch
    from paper_2509_13300_gb300 import countergen
    rng = np.random.default_rng(7)
    p960 = synth.pcr_params("AGRRTTYGATYHTDGYTYAG", "YCNTTCCYTYDYRGTACT", k=4, min_len=100, max_len=3000,
                            tm_min=45.0)
    # oligo totals as the sum of the two primers' degeneracies: 32 + 32 and 128 + 128
    p64 = synth.pcr_params(synth.random_primer(rng, 19, "RYSWK"), synth.random_primer(rng, 21, "WKMRY"), k=4,
                           min_len=100, max_len=3000, tm_min=45.0)
    p256 = synth.pcr_params(synth.random_primer(rng, 22, "RYSWKMR"), synth.random_primer(rng, 24, "KMRYSWK"), k=4,
                            min_len=100, max_len=3000, tm_min=45.0)
    pairs = [p960, p64, p256]
    c = countergen.collection(seed=7, n_genomes=8, len_lo=2e5, len_hi=1e6, pairs=pairs)
    w = c.workload()
    o_sites = oracle.scan(w.seq, w.contig_off, w.contig_genome, pairs)
    o_tm, o_ps = oracle.tm(w.seq, w.contig_off, o_sites, pairs)
    o_amps = oracle.pair(o_sites, pairs, o_ps)
    assert len(o_amps) > 0
    dev = torch.zeros(c.n_bases, dtype=torch.uint8, device="cuda")
    ctx.generate_bases(c, 0, c.n_bases, dev)
    sid = ctx.ah_load_genomes(dev, c.n_bases, c.contig_off, c.contig_genome)
    try:
        pids = [ctx.ah_set_primers(p["fwd"], p["rev"], p) for p in pairs]
        r = ctx.run(sid, pids, tm_filter=True)
    finally:
        ctx.ah_unload_genomes(sid)
    assert r["sites"].tobytes() == o_sites.tobytes()
    assert np.array_equal(r["pass_"], o_ps)
    ok = ~np.isnan(o_tm)
    assert np.abs(r["tm"][ok] - o_tm[ok]).max() <= TM_TOL
    assert r["amps"].tobytes() == o_amps.tobytes()


def _served_oracle(w, pair, genomes, k, tm_filter):
    """A request's result by the plain definition: the pair scanned at the
    request's k over the pool, sites of the named genomes kept, Tm and
    amplicon calling on those sites alone."""
    p = dict(pair, k=k)
    sites = oracle.scan(w.seq, w.contig_off, w.contig_genome, [p])
    sites = sites[np.isin(sites["genome"], np.asarray(genomes, dtype=np.uint32))]
    passed = None
    if tm_filter and len(sites):
        _, passed = oracle.tm(w.seq, w.contig_off, sites, [p])
    amps = oracle.pair(sites, [p], passed)
    seqs, offs = oracle.fetch(w.seq, w.contig_off, amps)
    return sites, amps, seqs, offs


def test_served_requests_alone_and_in_the_mix(ctx):
    """ah_serve_*: every request's result is the same whether it runs alone
    (one request per batch), in large mixed batches, or in batches cut short
    by the memory budget, and equals the plain definition on the pool."""
    pairs = [synth.pcr_params(*synth.PAPER_PAIRS["Titan"], k=3, min_len=100, max_len=3000, tm_min=45.0),
             synth.pcr_params(*synth.PAPER_PAIRS["V3V4"], k=2, min_len=100, max_len=3000, tm_min=50.0)]
    w = synth.collection(seed=12, n_genomes=10, len_lo=1.5e5, len_hi=5e5, pairs=pairs, max_subs=3)
    n_g = int(w.contig_genome.max()) + 1
    rng = np.random.default_rng(5)
    reqs = []
    for i in range(24):
        g = rng.choice(n_g, size=int(rng.integers(1, n_g + 1)), replace=False)
        reqs.append((g.astype(np.uint32), int(rng.integers(len(pairs))), int(rng.integers(0, 4)),
                     bool(rng.integers(2))))
    reqs.append((np.zeros(0, np.uint32), 0, 2, True))                      # no genomes
    reqs.append((np.array([n_g + 5, 1, 1], np.uint32), 1, 1, False))       # unknown id and a duplicate
    sid = ctx.load(w.seq, w.contig_off, w.contig_genome)
    pids = [ctx.ah_set_primers(p["fwd"], p["rev"], p) for p in pairs]
    try:
        def serve(max_batch, mem_budget, one_at_a_time):
            out = []
            with ah.Server(ctx, sid, mem_budget=mem_budget, max_batch=max_batch) as srv:
                if one_at_a_time:
                    for g, j, k, f in reqs:
                        out.append(srv.wait(srv.submit(g, pids[j], k, f)))
                else:
                    tickets = [srv.submit(g, pids[j], k, f) for g, j, k, f in reqs]
                    out = [srv.wait(t) for t in tickets]
            return out

        alone = serve(1, 1 << 30, True)
        mixed = serve(64, 1 << 30, False)
        budget = serve(64, 200_000, False)
        # the context is usable again after the servers stopped
        assert len(ctx.scan(sid, [pids[0]])) > 0
    finally:
        ctx.ah_unload_genomes(sid)
    assert max(x[4]["batch_size"] for x in mixed) > 8
    assert max(x[4]["batch_size"] for x in budget) < max(x[4]["batch_size"] for x in mixed)
    assert all(x[4]["batch_size"] == 1 for x in alone)
    total_amps = 0
    for n, ((g, j, k, f), a, m, b) in enumerate(zip(reqs, alone, mixed, budget)):
        for x in (m, b):
            assert x[0].tobytes() == a[0].tobytes(), n
            assert x[1].tobytes() == a[1].tobytes(), n
            assert x[2] == a[2] and np.array_equal(x[3], a[3]), n
        info = a[4]
        assert info["status"] == 0 and info["submit_ms"] <= info["start_ms"] <= info["done_ms"]
        want_s, want_a, want_q, want_o = _served_oracle(w, pairs[j], [x for x in g if x < n_g], k, f)
        assert a[0].tobytes() == want_s.tobytes(), n
        assert a[1].tobytes() == want_a.tobytes(), n
        assert a[2] == want_q and np.array_equal(a[3], want_o), n
        total_amps += len(want_a)
    assert total_amps > 10


def test_profile_hmm_build_and_scores(ctx):
    """ah_hmm_build / ah_hmm_score / ah_hmm_forward: the profile trained on the
    exact-match amplicons of an operon family (training set taken end to end: a
    k = 0 run and its fetched sequences) equals the oracle's (fp32 of its fp64
    scores), and the fp32 Viterbi and Forward scores of every k = 2 amplicon and
    of random regions are within the fp32 accumulation bound of the oracle's
    fp64 scores."""
    import torch
    w = synth.operon_family(seed=21, n_genomes=16)
    p = w.pairs[0]
    p0 = dict(p, k=0)
    s0 = oracle.scan(w.seq, w.contig_off, w.contig_genome, [p0])
    a0 = oracle.pair(s0, [p0])
    q0, o0 = oracle.fetch(w.seq, w.contig_off, a0)
    train = [q0[int(o0[i]):int(o0[i + 1])].decode() for i in range(len(a0))]
    assert len(train) >= 8
    ref, T, E = oracle.hmm_build(train)
    s2 = oracle.scan(w.seq, w.contig_off, w.contig_genome, [p])
    a2 = oracle.pair(s2, [p])
    rng = np.random.default_rng(3)  # unrelated regions in either orientation
    extra = np.zeros(40, dtype=oracle.AMPLICON_DTYPE)
    lens = np.diff(w.contig_off.astype(np.int64))
    for r in extra:
        c = int(rng.integers(len(lens)))
        L = int(rng.integers(200, 900))
        s = int(rng.integers(0, lens[c] - L))
        r["genome"], r["contig"], r["start"], r["end"], r["orient"] = w.contig_genome[c], c, s, s + L, rng.integers(2)
    amps = np.concatenate([a2, extra])
    q2, o2 = oracle.fetch(w.seq, w.contig_off, amps)
    seqs = [q2[int(o2[i]):int(o2[i + 1])].decode() for i in range(len(amps))]
    want = np.array([oracle.hmm_viterbi(T, E, x) for x in seqs])
    sid = ctx.load(w.seq, w.contig_off, w.contig_genome)
    try:
        pid0 = ctx.ah_set_primers(p0["fwd"], p0["rev"], p0)
        r0 = ctx.run(sid, [pid0], tm_filter=False)
        gtrain = [r0["seqs"][int(r0["offs"][i]):int(r0["offs"][i + 1])].decode() for i in range(len(r0["amps"]))]
        assert gtrain == train
        hid = ctx.hmm_build(gtrain)
        m, gref, gt, ge = ctx.hmm_tables(hid)
        assert (m, gref) == (T.shape[0] - 1, ref)
        assert np.array_equal(np.isinf(gt), np.isinf(T))
        fin = ~np.isinf(T)
        assert np.abs(gt[fin] - T[fin]).max() <= 1e-5
        assert np.abs(ge - E).max() <= 1e-5
        got = ctx.hmm_score(sid, hid, amps)
        got_f = ctx.hmm_forward(sid, hid, amps)
        # device records and scores give the same
        dev_amps = torch.from_numpy(amps.view(np.uint8).copy()).cuda()
        dev_out = torch.zeros(len(amps), dtype=torch.float32, device="cuda")
        ctx.hmm_score(sid, hid, dev_amps, n=len(amps), out=dev_out)
        assert np.array_equal(dev_out.cpu().numpy(), got)
        with pytest.raises(ah.AHError):
            ctx.hmm_score(sid, hid + 99, amps)
        bad = amps[:1].copy()
        bad["end"] = lens[bad["contig"][0]] + 5
        with pytest.raises(ah.AHError):
            ctx.hmm_score(sid, hid, bad)
        ctx.hmm_free(hid)
    finally:
        ctx.ah_unload_genomes(sid)
    # fp32 accumulation along one path of N = n + m moves: the rounding of each
    # addition is at most 2^-24 of the partial sum, and N roundings of either
    # sign add up like a random walk (sqrt(N)); a partial sum is at most the
    # final score plus the remaining terms, about N times the mean table entry.
    # Ten standard deviations of that walk (observed errors are ~1/30 of it).
    pmean = float(np.concatenate([np.abs(T[fin]), np.abs(E[1:]).ravel()]).mean())
    N = np.array([len(x) for x in seqs]) + m
    tol = 10.0 * np.sqrt(N) * 2.0 ** -24 * (np.abs(want) + N * pmean) + 1e-4
    err = np.abs(got.astype(np.float64) - want)
    assert (err <= tol).all(), (err.max(), tol.min())
    assert want[:len(a2)].min() > want[len(a2):].max()  # family members above unrelated regions
    # Forward: the same walk, plus per log-sum step an absolute error of a few
    # 2^-23 from log2(1 + 2^d) (exp2f / log2f within 2 ulp)
    want_f = np.array([oracle.hmm_forward(T, E, x) for x in seqs])
    tol_f = 10.0 * np.sqrt(N) * (2.0 ** -24 * (np.abs(want_f) + N * pmean) + 4 * 2.0 ** -23) + 1e-4
    err_f = np.abs(got_f.astype(np.float64) - want_f)
    assert (err_f <= tol_f).all(), (err_f.max(), tol_f.min())
    assert (want_f >= want - 1e-9).all() and (got_f >= got - 1e-3).all()  # the sum is at least the best path


@pytest.mark.parametrize("kernel", ["wave", "rows"])
def test_profile_hmm_kernels_on_profiles_of_several_lengths(ctx, kernel, monkeypatch):
    """Both scoring kernels (the warp wavefront and the block-per-group kernel,
    forced by AH_HMM_KERNEL for both scores) against the oracle's fp64 Viterbi
    and Forward scores, on profiles of m + 1 = 40, 129, 255 and 640 columns
    (the wavefront's stripes hold 128: a lone partial stripe, a last stripe of
    one column, a nearly full one, five full ones) and on amplicons of 0, 1 and
    2 letters up to 1,700."""
    monkeypatch.setenv("AH_HMM_KERNEL", kernel)
    w = synth.operon_family(seed=21, n_genomes=16)
    p = w.pairs[0]
    p0 = dict(p, k=0)
    s0 = oracle.scan(w.seq, w.contig_off, w.contig_genome, [p0])
    a0 = oracle.pair(s0, [p0])
    q0, o0 = oracle.fetch(w.seq, w.contig_off, a0)
    train = [q0[int(o0[i]):int(o0[i + 1])].decode() for i in range(len(a0))]
    assert min(len(x) for x in train) >= 254
    s2 = oracle.scan(w.seq, w.contig_off, w.contig_genome, [p])
    amps = oracle.pair(s2, [p])[:24]
    rng = np.random.default_rng(8)
    lens = np.diff(w.contig_off.astype(np.int64))
    extra = np.zeros(24, dtype=oracle.AMPLICON_DTYPE)
    for q, r in enumerate(extra):
        c = int(rng.integers(len(lens)))
        L = [0, 1, 2][q] if q < 3 else int(rng.integers(3, 1700))
        s = int(rng.integers(0, lens[c] - L))
        r["genome"], r["contig"], r["start"], r["end"], r["orient"] = w.contig_genome[c], c, s, s + L, q % 2
    amps = np.concatenate([amps, extra])
    qa, oa = oracle.fetch(w.seq, w.contig_off, amps)
    seqs = [qa[int(oa[i]):int(oa[i + 1])].decode() for i in range(len(amps))]
    sid = ctx.load(w.seq, w.contig_off, w.contig_genome)
    try:
        for cut in (39, 128, 254, None):
            tr = [x[:cut] for x in train] if cut else train
            _, T, E = oracle.hmm_build(tr)
            m = T.shape[0] - 1
            assert m == (cut or m)
            hid = ctx.hmm_build(tr)
            got = ctx.hmm_score(sid, hid, amps).astype(np.float64)
            got_f = ctx.hmm_forward(sid, hid, amps).astype(np.float64)
            ctx.hmm_free(hid)
            want = np.array([oracle.hmm_viterbi(T, E, x) for x in seqs])
            want_f = np.array([oracle.hmm_forward(T, E, x) for x in seqs])
            fin = ~np.isinf(T)
            # the fp32 accumulation bound of the test above (a random walk of
            # roundings along one path of N = n + m moves, ten standard deviations)
            pmean = float(np.concatenate([np.abs(T[fin]), np.abs(E[1:]).ravel()]).mean())
            N = np.array([len(x) for x in seqs]) + m
            tol = 10.0 * np.sqrt(N) * 2.0 ** -24 * (np.abs(want) + N * pmean) + 1e-4
            tol_f = 10.0 * np.sqrt(N) * (2.0 ** -24 * (np.abs(want_f) + N * pmean) + 4 * 2.0 ** -23) + 1e-4
            assert np.isfinite(got).all() and np.isfinite(got_f).all(), (cut, kernel)
            err, err_f = np.abs(got - want), np.abs(got_f - want_f)
            assert (err <= tol).all(), (cut, kernel, err.max(), int(err.argmax()))
            assert (err_f <= tol_f).all(), (cut, kernel, err_f.max(), int(err_f.argmax()))
    finally:
        ctx.ah_unload_genomes(sid)
