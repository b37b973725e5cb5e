"""Host logic of bench.py's forms (CPU): chunking a collection into whole
genomes, the rebased contig tables of a genome range, and the form workloads'
primer pairs (oligo totals 16 / 64 / 256 / 960 and the paper's four)."""
import numpy as np

import bench
import oracle
from paper_2509_13300_gb300 import countergen


def test_genome_chunks_cover_the_collection_with_whole_genomes():
    c = countergen.collection(seed=3, n_genomes=40, len_lo=1e5, len_hi=9e5)
    for cap in (1, 250_000, 2_000_000, 10**12):
        ch = bench.genome_chunks(c, cap)
        assert ch[0][0] == 0 and ch[-1][1] == 40
        assert all(a < b for a, b in ch) and all(ch[i][1] == ch[i + 1][0] for i in range(len(ch) - 1))
        goff = c.genome_off.astype(np.int64)
        for a, b in ch:  # at most cap bases, unless a single genome is longer
            assert goff[b] - goff[a] <= cap or b == a + 1


def test_sub_tables_rebase_contigs_of_a_genome_range():
    c = countergen.collection(seed=4, n_genomes=12, len_lo=1e5, len_hi=5e5)
    b0, b1, off, gen = bench.sub_tables(c, 3, 7)
    assert b0 == int(c.genome_off[3]) and b1 == int(c.genome_off[7])
    assert off[0] == 0 and int(off[-1]) == b1 - b0 and len(off) == len(gen) + 1
    assert set(gen.tolist()) == {3, 4, 5, 6}
    # the same contigs as the full table, shifted
    sel = (c.contig_genome >= 3) & (c.contig_genome < 7)
    assert np.array_equal(np.diff(off.astype(np.int64)), np.diff(c.contig_off.astype(np.int64))[sel])


def test_form_pairs():
    syn = bench.synthetic_pairs(2, (2, 3, 4, 2))
    assert [oracle.degeneracy(p["fwd"]) + oracle.degeneracy(p["rev"]) for p in syn] == [16, 64, 256, 960]
    assert [p["k"] for p in syn] == [2, 3, 4, 2]
    assert all(17 <= len(p["fwd"]) <= 25 and 17 <= len(p["rev"]) <= 25 for p in syn)
    paper = bench.paper_pairs(4)
    assert len(paper) == 4 and all(p["k"] == 4 for p in paper)
    large = bench.large_pairs()
    assert [oracle.degeneracy(p["fwd"]) + oracle.degeneracy(p["rev"]) for p in large] == [960, 64, 256]


def _small_large_like():
    """A few short genomes with the large workload's three pairs (CPU-sized)."""
    return countergen.collection(seed=5, n_genomes=3, len_lo=6e4, len_hi=1.2e5, pairs=bench.large_pairs())


def test_oracle_sample_is_seeded_whole_genomes_and_bounded():
    c = countergen.collection(seed=7, n_genomes=300, len_lo=1e5, len_hi=8e5)
    a = bench.oracle_sample(c, 1.0, 4)
    assert np.array_equal(a, bench.oracle_sample(c, 1.0, 4))       # seeded
    assert np.all(np.diff(a) > 0) and a[0] >= 0 and a[-1] < 300     # sorted genome ids
    gl = np.diff(c.genome_off.astype(np.int64))
    want = max(1.0e6, 0.12e6 * 4 * 1.0)
    assert gl[a].sum() >= want and gl[a].sum() - gl[a].max() < want  # just enough bases
    assert len(bench.oracle_sample(c, 4.0, 4)) > len(a)


def test_genome_records_of_a_chunk_equal_each_genome_alone():
    """Slicing one run over several genomes into per-genome records (contigs
    rebased, amplicon ends re-indexed, sequences cut out) gives exactly the
    oracle's records of each genome run alone."""
    c = _small_large_like()
    pairs = bench.large_pairs()
    b0, b1, off, gen = bench.sub_tables(c, 0, 3)
    seq = c.bases(b0, b1)
    s = oracle.scan(seq, off, gen, pairs)
    tm, ps = oracle.tm(seq, off, s, pairs)
    am = oracle.pair(s, pairs, ps)
    qs, qo = oracle.fetch(seq, off, am)
    res = (s, tm.astype(np.float32), ps, am, qs, qo)
    want, _ = bench.oracle_on_genomes(c, pairs, np.arange(3), 1)
    got = {g: bench.genome_records(c, (b0, b1, off, gen), res, g) for g in range(3)}
    summ = bench.parity_summary(c, got, want)
    assert summ["all_equal"] and summ["genomes"] == 3 and summ["sites"] == len(s)


def test_parity_summary_flags_each_kind_of_difference():
    c = _small_large_like()
    pairs = bench.large_pairs()
    want, _ = bench.oracle_on_genomes(c, pairs, np.array([1]), 1)
    s_, tm, ps, am, qs, qo = want[1]
    assert len(s_) > 0

    def got(**kw):
        d = dict(s=s_.copy(), tm=tm.astype(np.float32), ps=ps.copy(), am=am.copy(), qs=qs, qo=qo.copy())
        d.update(kw)
        return {1: (d["s"], d["tm"], d["ps"], d["am"], d["qs"], d["qo"])}

    assert bench.parity_summary(c, got(), want)["all_equal"]
    s2 = s_.copy()
    s2["mm"][0] ^= 1
    assert not bench.parity_summary(c, got(s=s2), want)["sites_equal"]
    p2 = ps.copy()
    p2[0] ^= 1
    assert not bench.parity_summary(c, got(ps=p2), want)["pass_equal"]
    t2 = tm.astype(np.float32)
    i = int(np.nonzero(~np.isnan(t2))[0][0])
    t2[i] += 0.02
    r = bench.parity_summary(c, got(tm=t2), want)
    assert not r["all_equal"] and 0.015 < r["max_dtm_C"] < 0.025
    if len(am):
        a2 = am.copy()
        a2["end"][0] += 1
        assert not bench.parity_summary(c, got(am=a2), want)["amplicons_equal"]
        q2 = bytes([qs[0] ^ 1]) + qs[1:]
        assert not bench.parity_summary(c, got(qs=q2), want)["sequences_equal"]


def test_device_encode_2bit_equals_the_host_encoder():
    """The bench's torch encoder (run here on CPU tensors) gives the codes and
    runs of ah.encode_2bit, also across its internal steps and at the end."""
    import torch
    from paper_2509_13300_gb300 import ah
    rng = np.random.default_rng(8)
    letters = np.frombuffer(b"ACGTacgtNNNNRY-", dtype=np.uint8)
    for n, step in ((1, 4), (37, 8), (1001, 16), (5000, 1 << 28)):
        seq = letters[rng.integers(0, len(letters), n)]
        seq[-1] = ord("N")  # a run reaching the end
        codes, gaps = bench.device_encode_2bit(torch, torch.from_numpy(seq.copy()), step=step)
        c2, g2 = ah.encode_2bit(seq)
        assert codes.numpy().tobytes() == c2.tobytes() and np.array_equal(gaps, g2), (n, step)


def test_form_keys_summarise_each_form_and_report_a_failing_one(monkeypatch):
    """The default line's `forms` key: each form runs on its own workload with the
    overrides of the key (two batched passes after three, the served requests of
    --forms-requests), a summary of its line is kept, and a form that raises is
    reported by its error without stopping the others."""
    import argparse
    seen = {}

    def batched(args, emit=True):
        seen["batched"] = (args.steps, args.warmup, args.n_genomes, emit)
        return {"config": {"workload": "batched-w", "input": "2-bit"}, "value": 2000.0, "unit": "Gbp/s",
                "s_per_pass": 0.05, "steps": args.steps,
                "plain": {"value": 14.0, "form": "one genome per load", "genomes": 400},
                "plain_all_pairs": {"value": 27.0, "form": "one run of all pairs"},
                "batched_over_plain": 2000.0 / 14.0, "batched_over_plain_all_pairs": 2000.0 / 27.0,
                "h2d_gbs": 170.0, "results_per_pass": {"sites": 1}, "clocks": {"sm_mhz": 2070.0}}

    def served(args, emit=True):
        seen["served"] = (args.requests, args.n_genomes, emit)
        raise RuntimeError("no device")

    monkeypatch.setattr(bench, "bench_batched", batched)
    monkeypatch.setattr(bench, "bench_served", served)
    args = argparse.Namespace(steps=20, warmup=5, n_genomes=123, forms_requests=77, requests=2000)
    out = bench.form_keys(args)
    assert seen == {"batched": (2, 3, None, False), "served": (77, None, False)}
    assert out["batched"]["workload"] == "batched-w" and out["batched"]["batched_over_plain"] == 2000.0 / 14.0
    assert out["batched"]["plain"]["genomes"] == 400 and out["batched"]["wall_s"] >= 0.0
    assert out["served"] == {"error": "RuntimeError: no device"}
    assert args.steps == 20 and args.n_genomes == 123  # the caller's arguments are left alone
