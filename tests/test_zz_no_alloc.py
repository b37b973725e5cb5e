"""ah_pair_noalloc: amplicon calling that allocates no memory.

Callers that cannot allocate during a call (for instance while a stream is
being captured into a CUDA graph, or under an allocator that owns all of
device memory) use this variant of ah_pair; its scratch is a fixed device
array inside the library.  This test calls it through the C ABI twice in a
row and checks each result against the ordinary ah_pair on the same sites
(both are integer outputs, so the comparison is exact).  It lives in a file
of its own that pytest collects last, and passes alone in a fresh process as
well as after the other tests.
"""
import ctypes

import numpy as np
import pytest

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
