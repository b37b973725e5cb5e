"""ah_pair_noalloc: amplicon calling that allocates no memory.

Callers that cannot allocate during a call (an application whose allocator
owns all of device memory, or a latency-bound loop that must stay off the
driver's allocator) use this variant of ah_pair; its scratch is a fixed
device array inside the library.  These tests call it through the C ABI
twice in a row and check each result against the ordinary ah_pair on the
same sites and against the oracle's pairing (integer outputs: exact), also
near the per-call site limit, and check that the device's free memory does
not move across calls.  They live in a file of their own that pytest
collects last, and pass alone in a fresh process as well as after the other
tests.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2509_13300_gb300 import ah, build, synth

pytestmark = pytest.mark.gpu


def _call(lib, windows, n_pairs, sites_d, pass_d, n, out_d, cap):
    n_out = ctypes.c_uint64()
    st = lib.ah_pair_noalloc(windows.ctypes.data_as(ctypes.c_void_p), n_pairs, ctypes.c_void_p(sites_d.data_ptr()),
                             ctypes.c_void_p(pass_d.data_ptr()) if pass_d is not None else None, n,
                             ctypes.c_void_p(out_d.data_ptr()) if out_d is not None else None, cap,
                             ctypes.byref(n_out), None)
    return st, n_out.value


def test_pair_noalloc_matches_pair_on_two_calls():
    import torch
    build.build()
    lib = ah.lib()
    w = synth.random_small(7, n_bases=80_000, n_contigs=5, L_f=9, L_r=8, k=2, min_len=30, max_len=700)
    w.pairs = [dict(w.pairs[0], tm_min=-20.0)]  # short primers: splits the sites ~1:4
    p = w.pairs[0]
    with ah.Context(0) as ctx:
        sid = ctx.load(w.seq, w.contig_off, w.contig_genome)
        pid = ctx.ah_set_primers(p["fwd"], p["rev"], p)
        sites = ctx.scan(sid, [pid])
        _, passed = ctx.tm(sid, [pid], sites)
        want_tm = ctx.pair(sid, [pid], sites, passed)  # the existing entry point
        want_all = ctx.pair(sid, [pid], sites)
        ctx.ah_unload_genomes(sid)
    n = len(sites)
    assert n > 100 and len(want_all) > len(want_tm) > 0
    windows = np.array([[len(p["fwd"]), len(p["rev"]), p["min_len"], p["max_len"]]], dtype=np.int32)
    torch.cuda.set_device(0)
    sites_d = torch.from_numpy(sites.view(np.uint8).copy()).cuda()
    pass_d = torch.from_numpy(passed.copy()).cuda()
    assert want_tm.tobytes() == oracle.pair(sites, w.pairs, passed).tobytes()  # the reference pairing
    assert want_all.tobytes() == oracle.pair(sites, w.pairs).tobytes()
    for call in range(2):
        for pass_arg, want in ((pass_d, want_tm), (None, want_all)):
            st, need = _call(lib, windows, 1, sites_d, pass_arg, n, None, 0)  # size query
            assert st == ah.AH_ERR_OVERFLOW and need == len(want), (call, st, need)
            out_d = torch.full((len(want) * 28,), 0xAB, dtype=torch.uint8, device="cuda")
            st, got = _call(lib, windows, 1, sites_d, pass_arg, n, out_d, len(want))
            assert st == ah.AH_OK and got == len(want), (call, st, got)
            assert out_d.cpu().numpy().tobytes() == want.tobytes(), call


def test_pair_noalloc_rejects_oversize_and_host_buffers():
    import torch
    build.build()
    lib = ah.lib()
    windows = np.array([[20, 22, 100, 2500]], dtype=np.int32)
    sites_d = torch.zeros(16, dtype=torch.uint8, device="cuda")
    st, _ = _call(lib, windows, 1, sites_d, None, (1 << 18) + 1, None, 0)
    assert st == ah.AH_ERR_ARG
    host = torch.zeros(16, dtype=torch.uint8)
    st, _ = _call(lib, windows, 1, host, None, 1, None, 0)
    assert st == ah.AH_ERR_ARG
    bad = np.zeros(1, dtype=ah.SITE_DTYPE)
    bad["pair"] = 3  # only one pair window given
    st, _ = _call(lib, windows, 1, torch.from_numpy(bad.view(np.uint8).copy()).cuda(), None, 1, None, 0)
    assert st == ah.AH_ERR_ARG


def _synthetic_sites(rng, n, n_contigs, contig_len, L_f, L_r):
    """n distinct sites of one pair in canonical order (contig, pos, primer, strand)."""
    keys = set()
    while len(keys) < n:
        c = rng.integers(0, n_contigs, n)
        p = rng.integers(0, contig_len - max(L_f, L_r), n)
        ps = rng.integers(0, 4, n)
        keys.update(zip(c.tolist(), p.tolist(), ps.tolist()))
    keys = sorted(keys)[:n]
    s = np.zeros(n, dtype=ah.SITE_DTYPE)
    s["contig"] = [k[0] for k in keys]
    s["pos"] = [k[1] for k in keys]
    s["primer"] = [k[2] >> 1 for k in keys]
    s["strand"] = [k[2] & 1 for k in keys]
    return s


def test_pair_noalloc_near_the_site_limit_matches_the_oracle_and_allocates_nothing():
    """200,000 sites (the prefix sum takes the library's device-wide scan
    inside the fixed array): equal to the oracle's all-pairs amplicon calling,
    with and without pass flags, on two calls; after the first call the
    device's free memory and torch's allocator stay where they were."""
    import torch
    build.build()
    lib = ah.lib()
    torch.cuda.set_device(0)
    rng = np.random.default_rng(17)
    L_f, L_r = 18, 20
    sites = _synthetic_sites(rng, 200_000, 200, 1_000_000, L_f, L_r)
    passed = (rng.random(len(sites)) < 0.7).astype(np.uint8)
    pair = dict(fwd="A" * L_f, rev="C" * L_r, min_len=100, max_len=2500)
    want_all = oracle.pair(sites, [pair])
    want_tm = oracle.pair(sites, [pair], passed)
    assert len(want_all) > len(want_tm) > 10_000
    windows = np.array([[L_f, L_r, pair["min_len"], pair["max_len"]]], dtype=np.int32)
    sites_d = torch.from_numpy(sites.view(np.uint8).copy()).cuda()
    pass_d = torch.from_numpy(passed).cuda()
    outs = {id(want_all): torch.empty(len(want_all) * 28, dtype=torch.uint8, device="cuda"),
            id(want_tm): torch.empty(len(want_tm) * 28, dtype=torch.uint8, device="cuda")}
    torch.cuda.synchronize()
    for call in range(3):
        if call == 1:
            free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
        for pass_arg, want in ((pass_d, want_tm), (None, want_all)):
            out_d = outs[id(want)]
            st, got = _call(lib, windows, 1, sites_d, pass_arg, len(sites), out_d, len(want))
            assert st == ah.AH_OK and got == len(want), (call, st, got)
            assert out_d.cpu().numpy().tobytes() == want.tobytes(), call
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0 and torch.cuda.memory_allocated() == alloc0


def test_pair_noalloc_rejects_bad_windows_without_sites_and_unsorted_lists():
    import torch
    build.build()
    lib = ah.lib()
    sites_d = torch.zeros(16, dtype=torch.uint8, device="cuda")
    bad_window = np.array([[20, 22, 300, 100]], dtype=np.int32)  # min_len > max_len
    st, _ = _call(lib, bad_window, 1, sites_d, None, 0, None, 0)
    assert st == ah.AH_ERR_ARG
    s = np.zeros(2, dtype=ah.SITE_DTYPE)
    s["contig"] = [0, 0]
    s["pos"] = [500, 100]  # out of canonical order
    windows = np.array([[20, 22, 100, 2500]], dtype=np.int32)
    st, _ = _call(lib, windows, 1, torch.from_numpy(s.view(np.uint8).copy()).cuda(), None, 2, None, 0)
    assert st == ah.AH_ERR_ARG
