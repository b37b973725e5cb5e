#!/usr/bin/env python3
"""Benchmark of the in-silico PCR hot path on one GB300 (or N, one process per GPU).

Default workload (N = 1): the large collection -- 50,000 synthetic genomes of
1-8 Mbp (169 Gbp, counter-based generator, seed 7), 1-200 contigs each, GC
U(0.3, 0.7), 0.1% N runs, planted operon-like regions; three degenerate pairs
of 960, 64 and 256 oligos at k = 4; window 100-3000 bp; Tm threshold 50 C.

One step = the whole hot path over the collection through the C ABI, in
chunks of whole genomes: load/pack the resident ASCII bases, scan both
strands for the three pairs, Tm of every site, pair, fetch the amplicon
sequences.  `value` is bases x pairs scanned per second with the inputs
already in HBM; `e2e` is the same with host (pinned) input and output
buffers on the first chunk(s), the copies inside the timed region; the
`collection` key is the 100-genome (0.4 Gbp, one pair, k = 3) workload.
Under torchrun every rank scans its own seeded collection (weak scaling, no
data-path collective); value = all ranks' bases x pairs / max rank time.

--impl reference times the CPU oracle on a bounded sample of the same
workload (the reference arm of this benchmark).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gbp/s scanned per primer pair (both strands, k mm)"
WORKLOAD = "collection-100genomes-0.4Gbp-pair960-k3"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
# logic-pipe issue roof of a GB300: 152 SMs x LOP3 lane-ops/clk x clock; the lane rate
# is measured at the start of every run (ah_debug_pipe_rates: 61 measured on GB300,
# half of the 128-lane integer-add rate); this value is only the fallback
SMS, LOP_LANES_PER_CLK = 152, 61.0


def logic_lanes(ah):
    """(LOP3 lanes/clk/SM, its source): measured on this GPU, else the fallback."""
    try:
        lop, iadd = ah.debug_pipe_rates()
        return lop, f"measured on this GPU (ah_debug_pipe_rates: LOP3 {lop:.1f}, IADD {iadd:.1f} lanes/clk/SM)"
    except Exception as e:  # noqa: BLE001 -- the probe is an aid; the roofline still gets a denominator
        return LOP_LANES_PER_CLK, f"fallback {LOP_LANES_PER_CLK} (probe failed: {e})"


def workload(seed: int, n_genomes: int = 100):
    from paper_2509_13300_gb300 import synth
    w = synth.collection(seed=seed, n_genomes=n_genomes, len_lo=2e6, len_hi=7e6, k=3, min_len=100, max_len=2500)
    w.pairs = [dict(w.pairs[0], tm_min=50.0, dnac1_nM=250.0, Na_mM=50.0)]
    return w


class ClockSampler:
    """nvidia-smi samples (every 50 ms), kept only when taken inside the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def wait_first(self, timeout: float = 10.0):
        """Block until nvidia-smi has printed its first sample (it starts slowly)."""
        t0 = time.perf_counter()
        while self.proc and not self.lines and time.perf_counter() - t0 < timeout:
            time.sleep(0.01)

    def mark(self, start: bool):
        if start:
            self.t_start = time.perf_counter()
        else:
            self.t_end = time.perf_counter()

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        t0, t1 = getattr(self, "t_start", float("-inf")), getattr(self, "t_end", float("inf"))
        inside = [ln for t, ln in self.lines if t0 <= t <= t1 + 0.06]
        for ln in inside:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx = max(mx, float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def cpu_baseline(w, target_s: float = 15.0):
    """The oracle as it stands, on a bounded sample (leading genomes) of the
    workload, on all host cores: scan + Tm + pair + fetch."""
    import oracle
    cores = os.cpu_count() or 1
    goff = w.genome_off
    # ~1.5 Mbp/s per 8 Neoverse/Xeon cores measured for the oracle scan; size the sample for ~target_s
    want = max(2e6, 0.2e6 * cores * target_s)
    g = 1
    while g < len(goff) - 1 and goff[g] < want:
        g += 1
    nb = int(goff[g])
    nc = int(np.searchsorted(w.contig_off, nb))
    seq = w.seq[:nb]
    off = w.contig_off[:nc + 1]
    cg = w.contig_genome[:nc]
    t0 = time.perf_counter()
    s = oracle.scan(seq, off, cg, w.pairs, n_threads=cores)
    tm, ps = oracle.tm(seq, off, s, w.pairs, n_threads=cores)
    a = oracle.pair(s, w.pairs, ps)
    oracle.fetch(seq, off, a)
    dt = time.perf_counter() - t0
    return {"value": nb / dt / 1e9, "unit": "Gbp/s", "cores": cores, "kind": "oracle",
            "sample": f"first {g} of {len(goff) - 1} genomes ({nb / 1e6:.1f} Mbp, {nc} contigs), scan+Tm+pair+fetch, "
                      f"{dt:.1f} s"}


def run_reference(args):
    """The reference arm: the oracle as it stands, on the host cores, on a
    bounded sample of the large workload (genomes drawn with seed 7), for the
    same metric and unit as the default line."""
    rank, world, _ = dist_info()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        if rank != 0:
            dist.barrier()
            return
    pairs = large_pairs()
    coll = large_collection(7, args.n_genomes)
    cores = os.cpu_count() or 1
    sample = oracle_sample(coll, args.ref_seconds, cores)
    nb = int(sum(coll.genome_off[g + 1] - coll.genome_off[g] for g in sample.tolist()))
    vals, secs = [], []
    for i in range(args.warmup + args.steps):
        _, t = oracle_on_genomes(coll, pairs, sample, cores)
        if i >= args.warmup:
            vals.append(nb * len(pairs) / t / 1e9)
            secs.append(t)
    v = float(np.mean(vals))
    desc = (f"{len(sample)} of {len(coll.genome_off) - 1} genomes drawn with seed 7 ({nb / 1e6:.1f} Mbp), "
            f"3 pairs, scan+Tm+pair+fetch per step")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Gbp/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.mean(secs)) * 1e3 if secs else None,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8+f64", "data": "synthetic",
            "config": {"workload": LARGE_WORKLOAD, "sample": desc},
            "cpu_baseline": {"value": v, "unit": "Gbp/s", "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": v, "unit": "Gbp/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def load_peaks():
    try:
        p = json.load(open(PEAKS_FILE))
        return float(p["hbm_gbs"]), "measured", p
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback", {}


def traffic_record(kernel: str):
    """DRAM bytes per unit (base or site) of a kernel from a committed ncu
    capture, if it still matches this build (a launch's traffic grows with the
    bases it packs or scans: the bench scales it to the launches it times)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        rec = json.load(open(path)).get(kernel)
    except (OSError, ValueError):
        return None
    if not rec:
        return None
    from paper_2509_13300_gb300 import build
    if rec.get("kernel_digest") != build.kernel_digest(kernel):  # the kernel changed since the capture
        return None
    return rec


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 1000 plain, 2 batched passes, 10 HMM passes)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--ref-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="keep the default (or AH_SCAN_TUNING) scan variant")
    ap.add_argument("--n-genomes", type=int, default=None, help="smaller collections for profiling runs")
    ap.add_argument("--no-pipeline", action="store_true",
                    help="one set at a time (default: the next set packs on a second stream after the current scan)")
    ap.add_argument("--form", default="large", choices=["large", "collection", "plain", "batched", "served", "hmm"],
                    help="large: the 50,000-genome line (default); collection (alias plain): the 100-genome "
                         "line; batched / served / hmm: those forms' lines")
    ap.add_argument("--e2e-chunks", type=int, default=4,
                    help="large: chunks timed end to end from host input (0: none; 11 or more: every chunk)")
    ap.add_argument("--no-collection", action="store_true", help="large: skip the collection workload's key")
    ap.add_argument("--no-forms", action="store_true", help="large: skip the batched and served forms' keys")
    ap.add_argument("--forms-requests", type=int, default=400, help="large: requests of the served form's key")
    ap.add_argument("--chunk-bases", type=int, default=2_000_000_000, help="batched: bases per set (whole genomes)")
    ap.add_argument("--plain-genomes", type=int, default=400, help="batched: genomes timed in the plain form")
    ap.add_argument("--batched-input", default="2bit", choices=["2bit", "ascii"], help="batched: host input format")
    ap.add_argument("--requests", type=int, default=2000, help="served: requests")
    ap.add_argument("--rate", type=float, default=20.0, help="served: Poisson arrivals per second")
    ap.add_argument("--max-batch", type=int, default=64, help="served: requests per batch")
    ap.add_argument("--mem-budget", type=int, default=4 << 30, help="served: bytes one batch may plan for")
    ap.add_argument("--large-chunk", type=int, default=16_000_000_000, help="large: bases per chunk (whole genomes)")
    ap.add_argument("--check-genomes", type=int, default=6, help="large: sampled genomes checked by the oracle here")
    ap.add_argument("--dump-genomes", type=int, default=0,
                    help="large: GPU results of this many seeded genomes saved for --check-dump")
    ap.add_argument("--dump-path", default="large_sample.npz")
    ap.add_argument("--check-dump", default=None, help="oracle check of a large-form dump (CPU only)")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = 2 if args.impl == "reference" else {"batched": 2, "hmm": 10, "large": 10}.get(args.form, 1000)
    if args.check_dump:
        sys.exit(check_large_dump(args.check_dump))
    if args.impl == "reference":
        return run_reference(args)
    if args.form == "batched":
        return bench_batched(args)
    if args.form == "served":
        return bench_served(args)
    if args.form == "hmm":
        return bench_hmm(args)
    if args.form in ("collection", "plain"):
        return bench_collection(args)
    return bench_large_main(args)


def bench_collection(args, emit: bool = True):
    """The genome-collection workload (100 genomes, 0.4 Gbp, one 960-oligo pair,
    k = 3): one step = load/pack + run of the whole collection."""
    rank, world, local = dist_info()
    import torch
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    from paper_2509_13300_gb300 import ah, build
    build.build()

    w = workload(1 + rank, args.n_genomes or 100)
    p = w.pairs[0]
    n_bases = w.n_bases
    # one stream carries the library's work and the timing events
    stream = torch.cuda.Stream()
    seq_d = torch.from_numpy(w.seq).to("cuda")
    torch.cuda.synchronize()
    ctx = ah.Context(local)
    pid = ctx.ah_set_primers(p["fwd"], p["rev"], p)

    # capacities from one warm-up pass (also compiles and tunes the generated scan kernel)
    sid = ctx.ah_load_genomes(seq_d, n_bases, w.contig_off, w.contig_genome, stream)
    tune = None if args.no_tune else ctx.ah_tune_scan(sid, [pid], 0, stream)
    r = ctx.run(sid, [pid], tm_filter=True)
    ctx.ah_unload_genomes(sid)
    cap_s, cap_a, cap_q = len(r["sites"]) + 1, len(r["amps"]) + 1, len(r["seqs"]) + 1

    def run_out(dev: str, pinned: bool):
        def buf(n, dt):
            t = torch.empty(n, dtype=dt, device=dev)
            return t.pin_memory() if pinned else t
        b = dict(sites=buf(cap_s * 16, torch.uint8), tm=buf(cap_s, torch.float32), ps=buf(cap_s, torch.uint8),
                 amps=buf(cap_a * 28, torch.uint8), seq=buf(cap_q, torch.uint8), offs=buf(cap_a + 1, torch.int64))
        o = ah.RunOut(b["sites"].data_ptr(), cap_s, 0, b["tm"].data_ptr(), b["ps"].data_ptr(), b["amps"].data_ptr(),
                      cap_a, 0, b["seq"].data_ptr(), cap_q, 0, b["offs"].data_ptr(), 1, 0)
        return o, b

    out_d, bufs_d = run_out("cuda", False)
    streams = [stream, torch.cuda.Stream()]
    scan_done = torch.cuda.Event()

    def steps_device(K, ev=None):
        """K steps of load + run + unload.  Pipelined (default): two sets in flight --
        set i+1 is packed on the other stream once set i's scan has finished, so the
        packing overlaps the rest of run i (ah_run_begin / ah_run_end)."""
        if args.no_pipeline:
            for i in range(K):
                sid = ctx.ah_load_genomes(seq_d, n_bases, w.contig_off, w.contig_genome, stream)
                ctx.ah_run(sid, [pid], out_d, stream)
                ctx.ah_unload_genomes(sid)
                if ev is not None:
                    ev[i + 1].record(stream)
            return
        prev = ctx.ah_load_genomes(seq_d, n_bases, w.contig_off, w.contig_genome, streams[0])
        for i in range(K):
            ctx.ah_run_begin(prev, [pid], out_d, streams[i % 2], scan_done)
            nxt = None
            if i + 1 < K:
                streams[(i + 1) % 2].wait_event(scan_done)
                nxt = ctx.ah_load_genomes(seq_d, n_bases, w.contig_off, w.contig_genome, streams[(i + 1) % 2])
            ctx.ah_run_end(out_d)
            if ev is not None:
                ev[i + 1].record(streams[i % 2])
            ctx.ah_unload_genomes(prev)
            prev = nxt

    steps_device(args.warmup)
    n, m = out_d.n_sites, out_d.n_amplicons
    # timed region: CUDA events bracket the two streaming kernels (pack, scan) only
    ctx.ah_set_profiling(3)
    barrier(world)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    with ClockSampler(local) as clk:
        clk.wait_first()
        clk.mark(True)
        ev[0].record(stream)
        steps_device(args.steps, ev)
        torch.cuda.synchronize()
        clk.mark(False)
    n, m = out_d.n_sites, out_d.n_amplicons
    barrier(world)
    per_step = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
    t_ms = ev[0].elapsed_time(ev[-1])
    t_max = max_over_ranks(t_ms, world)
    bases_all = sum_over_ranks(float(n_bases), world)
    value = bases_all * args.steps / (t_max / 1e3) / 1e9  # Gbp/s, one pair

    live = {}
    for st in ("pack", "scan"):
        ms, launches, calls = ctx.ah_get_profile(st)
        live[st] = {"ms_per_step": ms / args.steps, "avg_launch_us": (ms / calls * 1e3) if calls else None}
    _, total_launches, _ = ctx.ah_get_profile(None)
    # stage breakdown: a separate, untimed pass with events around every stage
    prof_steps = min(args.steps, 50)
    ctx.ah_set_profiling(1)
    steps_device(prof_steps)
    stages = {"note": f"untimed pass of {prof_steps} steps, CUDA events around every stage"}
    for st in ("pack", "scan", "sort", "decode", "validate", "tm", "pair", "fetch"):
        ms, launches, calls = ctx.ah_get_profile(st)
        stages[st] = {"ms_per_step": ms / prof_steps, "launches_per_step": launches / prof_steps,
                      "avg_launch_us": (ms / calls * 1e3) if calls else None}
    ctx.ah_set_profiling(0)
    # the packing alone: loads with nothing else on the GPU (events of the "pack" stage)
    ctx.ah_set_profiling(3)
    n_alone = 20
    for _ in range(n_alone):
        sid = ctx.ah_load_genomes(seq_d, n_bases, w.contig_off, w.contig_genome, stream)
        torch.cuda.synchronize()
        ctx.ah_unload_genomes(sid)
    pack_alone_ms, _, _ = ctx.ah_get_profile("pack")
    ctx.ah_set_profiling(0)
    pack_alone_us = pack_alone_ms / n_alone * 1e3

    # ---- roofline of the dominant kernel (live CUDA-event durations) ----
    hbm_peak, peak_kind, peaks = load_peaks()
    clocks = clk.summary()
    scan_us = live["scan"]["avg_launch_us"]  # measured inside the timed region
    pack_us = live["pack"]["avg_launch_us"]
    dominant = "scan" if live["scan"]["ms_per_step"] >= live["pack"]["ms_per_step"] else "pack"
    scan_hbm = 0.5 * n_bases / (scan_us * 1e-6) / 1e9  # 4 planes x 1 bit per base
    pack_hbm = 1.5 * n_bases / (pack_us * 1e-6) / 1e9  # 1 B/base read + 0.5 B/base written
    # logic-pipe ops of the generated scan kernel per launch (static count of its LOP3s per word)
    lop_per_word = ctx_scan_lop_count(p, tune or {"R": 4, "arith_pct": 0})
    words = n_bases / 32.0
    scan_tops = lop_per_word * words / (scan_us * 1e-6) / 1e12
    clk_mhz = clocks["sm_mhz"] or 2070.0
    lanes, lanes_src = logic_lanes(ah)
    alu_peak = SMS * lanes * clk_mhz * 1e6 / 1e12
    if dominant == "scan":
        tr = traffic_record("ah_scan_kernel")
        roof = {"bound": "alu", "achieved": scan_tops, "peak": alu_peak, "unit": "Tops/s",
                "frac": scan_tops / alu_peak, "traffic": tr["dram_bytes_per_base"] * n_bases if tr else None,
                "kernel": "ah_scan_kernel",
                "peak_note": f"logic pipe: {SMS} SMs x {lanes:.1f} LOP3 lanes/clk x {clk_mhz:.0f} MHz "
                             f"(median SM clock under load); lanes {lanes_src}",
                "algorithmic": f"{lop_per_word} LOP3 per 32 starts per pass over the planes",
                "hbm_achieved_gbs": scan_hbm, "hbm_peak_gbs": hbm_peak,
                "hbm_frac": scan_hbm / hbm_peak, "hbm_peak_kind": peak_kind,
                "hbm_algorithmic": "0.5 B/base (4 one-hot planes x 1 bit)"}
    else:
        tr = traffic_record("pack_kernel")
        roof = {"bound": "hbm", "achieved": pack_hbm, "peak": hbm_peak, "unit": "GB/s",
                "frac": pack_hbm / hbm_peak, "traffic": tr["dram_bytes_per_base"] * n_bases if tr else None,
                "kernel": "pack_kernel", "peak_kind": peak_kind,
                "algorithmic": "1.5 B/base (1 B ASCII read + 0.5 B planes written)",
                "note": "live duration: the packing runs beside the previous set's sort/Tm/pair/fetch"}
    pack_alone = 1.5 * n_bases / (pack_alone_us * 1e-6) / 1e9
    pack_alone_rec = {"achieved": pack_alone, "frac": pack_alone / hbm_peak, "us_per_launch": pack_alone_us,
                      "note": "the packing with nothing else on the GPU, outside the timed region"}
    if dominant == "pack":
        roof["alone"] = pack_alone_rec

    # ---- end to end through the public API with host (pinned) buffers ----
    # the input as 2-bit codes and no-base runs (ah_load_genomes_2bit), and as ASCII
    seq_h = torch.from_numpy(w.seq).pin_memory()
    codes, gaps = ah.encode_2bit(w.seq)
    codes_h = torch.from_numpy(codes).pin_memory()
    out_h, bufs_h = run_out("cpu", True)
    inputs = {"2bit": (lambda st_: ctx.ah_load_genomes_2bit(codes_h, n_bases, gaps, w.contig_off, w.contig_genome,
                                                            st_, host_async=True), codes.nbytes + gaps.nbytes),
              "ascii": (lambda st_: ctx.ah_load_genomes(seq_h, n_bases, w.contig_off, w.contig_genome, st_,
                                                        host_async=True), n_bases)}

    def counts_host(kind):
        n, m, q = out_h.n_sites, out_h.n_amplicons, out_h.n_seq
        h2d = inputs[kind][1] + w.contig_off.nbytes + w.contig_genome.nbytes
        d2h = 16 * n + 4 * n + n + 28 * m + q + 8 * (m + 1)
        return h2d, d2h

    def steps_host(K, kind):
        """K steps through the C ABI with host (pinned) input and outputs.  Pipelined
        (default): the next set's host load -- its copies and packing -- is issued
        right after this run is queued, so the host link stays busy while the run
        computes; the loads are queued without waiting for their copies
        (AH_LOAD_HOST_ASYNC: the pinned inputs stay unchanged)."""
        load = inputs[kind][0]
        if args.no_pipeline:
            for _ in range(K):
                sid = load(stream)
                ctx.ah_run(sid, [pid], out_h, stream)
                ctx.ah_unload_genomes(sid)
            return counts_host(kind)
        prev = load(streams[0])
        for i in range(K):
            ctx.ah_run_begin(prev, [pid], out_h, streams[i % 2], None)
            nxt = None
            if i + 1 < K:
                nxt = load(streams[(i + 1) % 2])
            ctx.ah_run_end(out_h)
            ctx.ah_unload_genomes(prev)
            prev = nxt
        return counts_host(kind)

    e2e = None
    if args.e2e_steps > 0:
        res = {}
        for kind in ("2bit", "ascii"):
            steps_host(2, kind)
            barrier(world)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(streams[0])
            h2d, d2h = steps_host(args.e2e_steps, kind)
            for s_ in streams:
                streams[0].wait_stream(s_)
            e1.record(streams[0])
            torch.cuda.synchronize()
            e2e_ms = max_over_ranks(e0.elapsed_time(e1), world)
            res[kind] = {"value": bases_all * args.e2e_steps / (e2e_ms / 1e3) / 1e9, "unit": "Gbp/s",
                         "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "steps": args.e2e_steps,
                         "pipeline": not args.no_pipeline, "host_loads": "queued without waiting (AH_LOAD_HOST_ASYNC)"}
        e2e = dict(res["2bit"], input="2-bit base codes + no-base runs (ah_load_genomes_2bit) from pinned host memory",
                   ascii_input=res["ascii"])

    if rank != 0:
        ctx.close()
        return None
    cpu = None if args.no_cpu_baseline or world > 1 else cpu_baseline(w)
    line = {
        "metric": METRIC, "value": value, "unit": "Gbp/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_bases_per_gpu": n_bases, "n_contigs": w.n_contigs, "pairs": 1,
                   "oligos": 960, "k": 3, "window": [100, 2500], "tm_min_C": 50.0, "tm_dtype": "f32",
                   "sites": int(n), "amplicons": int(m), "parallelism": f"replicas x{world}",
                   "scan_tuning": tune,
                   "pipeline": ("one set at a time" if args.no_pipeline else
                                "2 sets in flight: set i+1 packs on a second stream after set i's scan"),
                   "l2": "inputs larger than L2 (0.4 GB ASCII + 0.2 GB planes per step)"},
        "latency_ms": {"p50": float(np.percentile(per_step, 50)), "p99": float(np.percentile(per_step, 99))},
        "stages": stages, "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": int(total_launches), "clocks": clocks,
        "timed_region_kernel_us": {st: live[st]["avg_launch_us"] for st in live},
    }
    if emit:
        print(json.dumps(line), flush=True)
    ctx.close()
    return line


def ctx_scan_lop_count(pair: dict, tune: dict) -> int:
    """LOP3 instructions the generated scan kernel (the tuned variant) issues
    per word of 32 starts for this pair: counted in its generated source."""
    from paper_2509_13300_gb300 import ah
    return ah.scan_lop3_per_word(pair["fwd"], pair["rev"], int(pair["k"]), tune["R"], tune["arith_pct"])



# ---------------------------------------------------------------------------
# Batched and served forms (bench.py --form batched | served): one JSON line
# each, beside the plain form's.  Genomes come from the counter-based
# generator, made on the device (ah_generate_bases).
# ---------------------------------------------------------------------------
def synthetic_pairs(seed: int, ks):
    """Four degenerate pairs of 17-25 nt whose oligo totals (sum of the two
    primers' degeneracies) are 16, 64, 256 and 960; k cycles over ks."""
    from paper_2509_13300_gb300 import synth
    rng = np.random.default_rng(seed)
    two = lambda n: "".join(rng.choice(list(synth.TWO_WAY), n))
    three = lambda n: "".join(rng.choice(list(synth.THREE_WAY), n))
    fr = [(synth.random_primer(rng, 17, two(3)), synth.random_primer(rng, 18, two(3))),      # 8 + 8
          (synth.random_primer(rng, 19, two(5)), synth.random_primer(rng, 21, two(5))),      # 32 + 32
          (synth.random_primer(rng, 22, two(7)), synth.random_primer(rng, 24, two(7))),      # 128 + 128
          (synth.random_primer(rng, 20, two(6) + three(2)),                                  # 576
           synth.random_primer(rng, 22, "N" + two(5) + three(1)))]                          # + 384
    return [synth.pcr_params(f, r, k=int(ks[i % len(ks)]), min_len=100, max_len=3000, tm_min=45.0)
            for i, (f, r) in enumerate(fr)]


def paper_pairs(k: int):
    """The four pairs printed in the paper (Sec. 2.3)."""
    from paper_2509_13300_gb300 import synth
    return [synth.pcr_params(f, r, k=k, min_len=100, max_len=3000, tm_min=45.0) for f, r in synth.PAPER_PAIRS.values()]


def device_collection(ctx, coll, torch, chunk: int = 1 << 31):
    """The collection's ASCII bases in device memory, generated on the device."""
    dev = torch.empty(coll.n_bases, dtype=torch.uint8, device="cuda")
    for b0 in range(0, coll.n_bases, chunk):
        ctx.generate_bases(coll, b0, min(chunk, coll.n_bases - b0), dev[b0:])
    torch.cuda.synchronize()
    return dev


def aligned_chunks(ctx, coll, tabs, torch):
    """The collection's ASCII bases in device memory, generated on the device,
    laid out so that every chunk's first base sits at a 16-byte aligned address
    (device input at such an address is staged by bulk copies).  Returns the
    buffer and each chunk's offset in it."""
    starts, pos = [], 16
    for b0, b1, _, _ in tabs:
        starts.append(pos)
        pos = (pos + (b1 - b0) + 16 + 15) // 16 * 16
    dev = torch.empty(pos, dtype=torch.uint8, device="cuda")
    step = 1 << 31
    for (b0, b1, _, _), a in zip(tabs, starts):
        for c0 in range(b0, b1, step):  # generated ranges start on a multiple of 4
            g0 = c0 - c0 % 4
            n = min(step, b1 - c0) + (c0 - g0)
            ctx.generate_bases(coll, g0, n, dev[a + (c0 - b0) - (c0 - g0):])
    torch.cuda.synchronize()
    return dev, starts


def device_encode_2bit(torch, ascii_d, step: int = 1 << 28):
    """The 2-bit codes and no-base runs of ah_load_genomes_2bit for ASCII bases in
    device memory (torch ops, before any timed region): codes on the device,
    runs as an (n, 2) uint64 numpy array."""
    n = ascii_d.numel()
    lut = torch.full((256,), 255, dtype=torch.uint8, device=ascii_d.device)
    for i, ch in enumerate(b"ACGT"):
        lut[ch] = i
        lut[ch + 32] = i
    codes = torch.empty((n + 3) // 4, dtype=torch.uint8, device=ascii_d.device)
    starts, ends = [], []
    prev = torch.zeros(1, dtype=torch.int8, device=ascii_d.device)
    for a in range(0, n, step):  # step is a multiple of 4
        b = min(n, a + step)
        c = lut.index_select(0, ascii_d[a:b].int())
        bad = c == 255
        c = torch.where(bad, torch.zeros_like(c), c)
        if (b - a) % 4:
            c = torch.cat([c, torch.zeros(4 - (b - a) % 4, dtype=torch.uint8, device=c.device)])
        q = c.view(-1, 4)
        codes[a // 4:a // 4 + q.shape[0]] = q[:, 0] | (q[:, 1] << 2) | (q[:, 2] << 4) | (q[:, 3] << 6)
        bi = bad.to(torch.int8)
        d = torch.diff(bi, prepend=prev)
        starts.append(torch.nonzero(d == 1).flatten() + a)
        ends.append(torch.nonzero(d == -1).flatten() + a)
        prev = bi[-1:]
    st_ = torch.cat(starts).cpu().numpy().astype(np.uint64)
    en = torch.cat(ends).cpu().numpy().astype(np.uint64)
    if len(en) < len(st_):  # a run reaching the end
        en = np.append(en, np.uint64(n))
    return codes, np.stack([st_, en - st_], axis=1) if len(st_) else np.zeros((0, 2), np.uint64)


def genome_chunks(coll, max_bases: int):
    """Consecutive genome ranges [g0, g1) of at most max_bases bases (one genome at least)."""
    goff = coll.genome_off
    out, g0 = [], 0
    G = len(goff) - 1
    while g0 < G:
        g1 = int(np.searchsorted(goff, goff[g0] + max_bases, side="right")) - 1
        g1 = min(G, max(g1, g0 + 1))
        out.append((g0, g1))
        g0 = g1
    return out


def sub_tables(coll, g0: int, g1: int):
    """Base range and rebased contig tables of genomes [g0, g1)."""
    b0, b1 = int(coll.genome_off[g0]), int(coll.genome_off[g1])
    c0 = int(np.searchsorted(coll.contig_off, b0, side="left"))
    c1 = int(np.searchsorted(coll.contig_off, b1, side="left"))
    off = np.ascontiguousarray(coll.contig_off[c0:c1 + 1] - np.uint64(b0))
    gen = np.ascontiguousarray(coll.contig_genome[c0:c1])
    return b0, b1, off, gen


class HostOut:
    """Pinned host output buffers of one ah_run (grown on overflow)."""

    def __init__(self, torch, ah, caps=(1 << 16, 1 << 14, 1 << 24)):
        self.torch, self.ah = torch, ah
        self.alloc(caps)

    def alloc(self, caps):
        t = self.torch
        s, a, q = (max(int(x), 1) for x in caps)
        self.caps = (s, a, q)
        self.b = [t.empty(n, dtype=t.uint8).pin_memory() for n in (16 * s, 4 * s, s, 28 * a, q, 8 * (a + 1))]
        self.o = self.ah.RunOut(self.b[0].data_ptr(), s, 0, self.b[1].data_ptr(), self.b[2].data_ptr(),
                                self.b[3].data_ptr(), a, 0, self.b[4].data_ptr(), q, 0, self.b[5].data_ptr(), 1, 0)

    def run(self, ctx, sid, pids, stream):
        for _ in range(3):
            try:
                return ctx.ah_run(sid, pids, self.o, stream)
            except self.ah.AHError as e:
                if e.status != self.ah.AH_ERR_OVERFLOW:
                    raise
                o = self.o
                self.alloc((o.n_sites * 5 // 4 + 1, o.n_amplicons * 5 // 4 + 1, o.n_seq * 5 // 4 + 1))
        raise RuntimeError("ah_run kept overflowing")

    def d2h_bytes(self):
        o = self.o
        return 21 * o.n_sites + 28 * o.n_amplicons + o.n_seq + 8 * (o.n_amplicons + 1)


def bench_batched(args, emit: bool = True):
    """Batched form: thousands of genomes of uneven length per set, streamed
    from pinned host memory in double-buffered chunks, several pairs in one
    scan launch; against the plain form (one genome per load and run)."""
    import torch
    from paper_2509_13300_gb300 import ah, build, countergen
    build.build()
    torch.cuda.set_device(0)
    n_g = args.n_genomes or 10_000
    pairs = synthetic_pairs(2, (2, 3, 4, 2))
    t0 = time.perf_counter()
    coll = countergen.collection(seed=2, n_genomes=n_g, len_lo=0.5e6, len_hi=8e6, pairs=pairs)
    t_layout = time.perf_counter() - t0
    ctx = ah.Context(0)
    pids = [ctx.ah_set_primers(p["fwd"], p["rev"], p) for p in pairs]
    N = coll.n_bases
    # the collection in pinned host memory (generated on the device, copied down once)
    host = torch.empty(N, dtype=torch.uint8, pin_memory=True)
    gen = torch.empty(min(N, 1 << 31), dtype=torch.uint8, device="cuda")
    for b0 in range(0, N, len(gen)):
        n = min(len(gen), N - b0)
        ctx.generate_bases(coll, b0, n, gen)
        host[b0:b0 + n].copy_(gen[:n])
    del gen
    chunks = genome_chunks(coll, args.chunk_bases)
    tabs = [sub_tables(coll, g0, g1) for g0, g1 in chunks]
    cmax = max(b1 - b0 for b0, b1, _, _ in tabs)
    two = args.batched_input == "2bit"
    codes_h, gaps_h = [], []
    if two:  # every chunk as 2-bit codes and no-base runs in pinned host memory (encoded once)
        for b0, b1, _, _ in tabs:
            cd, gp = device_encode_2bit(torch, host[b0:b1].cuda())
            ch = torch.empty(cd.numel(), dtype=torch.uint8, pin_memory=True)
            ch.copy_(cd)
            codes_h.append(ch)
            gaps_h.append(gp)
        del cd
        torch.cuda.empty_cache()
    dbuf = [torch.empty((cmax + 3) // 4 + 16 if two else cmax, dtype=torch.uint8, device="cuda") for _ in range(2)]
    cs = torch.cuda.Stream()                              # host-to-device copies
    st = [torch.cuda.Stream(), torch.cuda.Stream()]       # two sets in flight
    copied = [torch.cuda.Event() for _ in range(2)]
    packed = [torch.cuda.Event() for _ in range(2)]
    scan_done = torch.cuda.Event()
    outs = HostOut(torch, ah)
    totals = {}

    def copy(i):
        b0, b1, _, _ = tabs[i]
        with torch.cuda.stream(cs):
            if i >= 2:
                cs.wait_event(packed[i % 2])            # buffer free once chunk i-2 is packed
            if two:
                dbuf[i % 2][:codes_h[i].numel()].copy_(codes_h[i], non_blocking=True)
            else:
                dbuf[i % 2][:b1 - b0].copy_(host[b0:b1], non_blocking=True)
            copied[i % 2].record(cs)

    def load(i):
        b0, b1, off, gen_ = tabs[i]
        s = st[i % 2]
        s.wait_event(copied[i % 2])
        if two:
            sid = ctx.ah_load_genomes_2bit(dbuf[i % 2], b1 - b0, gaps_h[i], off, gen_, s)
        else:
            sid = ctx.ah_load_genomes(dbuf[i % 2], b1 - b0, off, gen_, s)
        packed[i % 2].record(s)
        return sid

    def one_pass():
        """Every chunk once: set i+1 packs on the other stream while set i runs,
        and chunk i+2 crosses the link meanwhile."""
        n_s = n_a = n_q = d2h = 0
        for i in range(min(2, len(tabs))):
            copy(i)
        sid = load(0)
        for i in range(len(tabs)):
            nxt = load(i + 1) if i + 1 < len(tabs) else None
            if i + 2 < len(tabs):
                copy(i + 2)
            outs.run(ctx, sid, pids, st[i % 2])
            n_s, n_a, n_q = n_s + outs.o.n_sites, n_a + outs.o.n_amplicons, n_q + outs.o.n_seq
            d2h += outs.d2h_bytes()
            ctx.ah_unload_genomes(sid)
            sid = nxt
        totals.update(sites=n_s, amplicons=n_a, seq=n_q, d2h_bytes=d2h)

    # the host link alone: every chunk's pinned host -> device copy, back to back
    h2d_chunk, link_bytes = [], 0
    for i, (b0, b1, _, _) in enumerate(tabs):
        nb = codes_h[i].numel() if two else b1 - b0
        link_bytes += nb
        h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        h0.record(cs)
        with torch.cuda.stream(cs):
            dbuf[i % 2][:nb].copy_(codes_h[i] if two else host[b0:b1], non_blocking=True)
        h1.record(cs)
        torch.cuda.synchronize()
        h2d_chunk.append(nb / (h0.elapsed_time(h1) / 1e3) / 1e9)
    h2d_s = sum((codes_h[i].numel() if two else b1 - b0) / (g * 1e9)
                for i, ((b0, b1, _, _), g) in enumerate(zip(tabs, h2d_chunk)))
    h2d_gbs = link_bytes / h2d_s / 1e9
    copy(0)
    sid0 = load(0)
    tune = None if args.no_tune else ctx.ah_tune_scan(sid0, pids, 0, st[0])
    ctx.ah_unload_genomes(sid0)
    torch.cuda.synchronize()
    for _ in range(max(1, args.warmup)):
        one_pass()
    torch.cuda.synchronize()
    ctx.ah_set_profiling(0)
    ctx.ah_get_profile(None)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        clk.wait_first()
        clk.mark(True)
        e0.record(st[0])
        for _ in range(args.steps):
            one_pass()
        st[0].wait_stream(st[1])
        st[0].wait_stream(cs)
        e1.record(st[0])
        torch.cuda.synchronize()
        clk.mark(False)
    _, launches, _ = ctx.ah_get_profile(None)
    t_batched = e0.elapsed_time(e1) / 1e3
    # stage split: one more pass with events around every stage (untimed)
    ctx.ah_set_profiling(1)
    one_pass()
    stages = {}
    for name in ("pack", "scan", "sort", "decode", "tm", "pair", "fetch", "host.run", "host.run.wait", "host.load"):
        ms, l, calls = ctx.ah_get_profile(name)
        stages[name] = {"ms": ms, "launches": l}
    ctx.ah_set_profiling(0)
    gbps = N * len(pairs) * args.steps / t_batched / 1e9
    # plain forms on a sample of genomes (host input, host outputs): one genome per
    # load, then one run per pair (one launch per genome per pair), and one run
    # with every pair
    rng = np.random.default_rng(0)
    sample = np.sort(rng.choice(n_g, size=min(n_g, args.plain_genomes), replace=False))
    plain_out = HostOut(torch, ah)
    hs = torch.cuda.current_stream()

    plain_codes = {}
    if two:  # each sampled genome alone as 2-bit codes in pinned host memory
        for g in np.sort(np.random.default_rng(0).choice(n_g, size=min(n_g, args.plain_genomes), replace=False)):
            b0, b1, _, _ = sub_tables(coll, int(g), int(g) + 1)
            cd, gp = ah.encode_2bit(host[b0:b1].numpy())
            plain_codes[int(g)] = (torch.from_numpy(cd).pin_memory(), gp)

    def plain(g, per_pair):
        b0, b1, off, gen_ = sub_tables(coll, int(g), int(g) + 1)
        if two:
            cd, gp = plain_codes[int(g)]
            sid = ctx.ah_load_genomes_2bit(cd, b1 - b0, gp, off, gen_, hs)
        else:
            sid = ctx.ah_load_genomes(host[b0:b1], b1 - b0, off, gen_, hs)
        for ids in ([[p] for p in pids] if per_pair else [pids]):
            plain_out.run(ctx, sid, ids, hs)
        ctx.ah_unload_genomes(sid)
        return b1 - b0

    plain_res = {}
    for per_pair in (True, False):
        for g in sample[:5]:
            plain(g, per_pair)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        nb = sum(plain(g, per_pair) for g in sample)
        torch.cuda.synchronize()
        t_plain = time.perf_counter() - t0
        plain_res[per_pair] = (nb * len(pairs) / t_plain / 1e9, t_plain, nb)
    gbps_plain, t_plain, nb = plain_res[True]
    line = {
        "form": "batched", "metric": "Gbp/s scanned per primer pair (both strands, k mm)", "value": gbps,
        "unit": "Gbp/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "s_per_pass": t_batched / args.steps, "higher_is_better": True, "data": "synthetic (counter-based, seed 2)",
        "config": {"workload": f"batched-{n_g}genomes-{N / 1e9:.1f}Gbp-{len(pairs)}pairs",
                   "n_genomes": n_g, "n_bases": N, "n_contigs": len(coll.contig_genome),
                   "pairs": [(p["fwd"], p["rev"], p["k"]) for p in pairs], "chunks": len(tabs),
                   "chunk_bases_max": cmax,
                   "input": ("2-bit codes and no-base runs (ah_load_genomes_2bit)" if two else "ASCII") +
                            " in pinned host memory, H2D copy of chunk i+2 overlapping set i's run and set i+1's "
                            "packing; the plain forms load the same format", "outputs": "pinned host (sites, Tm, pass, amplicons, "
                   "sequences)", "scan_tuning": tune, "layout_s": t_layout},
        "results_per_pass": totals, "gpu_launches_per_pass": launches / max(1, args.steps),
        "h2d_gbs": h2d_gbs, "h2d_gbs_per_chunk": [round(g, 1) for g in h2d_chunk],
        "h2d_bound_s_per_pass": h2d_s, "h2d_bytes_per_pass": link_bytes,
        "plain": {"value": gbps_plain, "unit": "Gbp/s", "genomes": len(sample), "bases": int(nb),
                  "form": "one genome per ah_load_genomes (host input), one ah_run per pair (host outputs)",
                  "s": t_plain},
        "plain_all_pairs": {"value": plain_res[False][0], "unit": "Gbp/s", "s": plain_res[False][1],
                            "form": "one genome per ah_load_genomes, one ah_run with the 4 pairs"},
        "batched_over_plain": gbps / gbps_plain, "batched_over_plain_all_pairs": gbps / plain_res[False][0], "clocks": clk.summary(), "stages_ms_one_pass": stages,
    }
    if emit:
        print(json.dumps(line), flush=True)
    ctx.close()
    return line


def bench_served(args, emit: bool = True):
    """Served form: a request loop over a resident pool; Poisson arrivals, then
    a saturated burst, against sequential plain solves of the same requests."""
    import torch
    from paper_2509_13300_gb300 import ah, build, countergen
    build.build()
    torch.cuda.set_device(0)
    n_g = args.n_genomes or 5_000
    pairs = paper_pairs(4) + synthetic_pairs(3, (4,))
    t0 = time.perf_counter()
    coll = countergen.collection(seed=3, n_genomes=n_g, len_lo=2e6, len_hi=7e6, pairs=pairs)
    t_layout = time.perf_counter() - t0
    ctx = ah.Context(0)
    pid = [ctx.ah_set_primers(p["fwd"], p["rev"], p) for p in pairs]
    dev = device_collection(ctx, coll, torch)
    N = coll.n_bases
    sid = ctx.ah_load_genomes(dev, N, coll.contig_off, coll.contig_genome)
    # requests: subset size Zipf over 1..n_g (P(s) ~ 1/s), members uniform without replacement
    rng = np.random.default_rng(3)
    R = args.requests
    w = 1.0 / np.arange(1, n_g + 1)
    sizes = rng.choice(np.arange(1, n_g + 1), size=R, p=w / w.sum())
    req = [(np.sort(rng.choice(n_g, size=int(z), replace=False)).astype(np.uint32), int(rng.integers(len(pairs))),
            int(rng.integers(0, 5))) for z in sizes]
    gbases = np.diff(coll.genome_off.astype(np.int64))
    req_bases = [int(gbases[g].sum()) for g, _, _ in req]
    def serve(arrivals, max_batch, budget, n=None):
        """Serve the first n requests at the given arrival times; returns per request
        (n_sites, n_amplicons, digest of sites, amplicons and sequences) and the stats."""
        import hashlib
        import threading as th
        n = R if n is None else n
        res = [None] * n
        with ah.Server(ctx, sid, mem_budget=budget, max_batch=max_batch) as srv:
            tickets = [None] * n
            ready = [th.Event() for _ in range(n)]

            def submitter():
                t_start = time.perf_counter()
                for i, (g, j, k) in enumerate(req[:n]):
                    dt = arrivals[i] - (time.perf_counter() - t_start)
                    if dt > 0:
                        time.sleep(dt)
                    tickets[i] = srv.submit(g, pid[j], k, True)
                    ready[i].set()

            thr = th.Thread(target=submitter)
            thr.start()
            for i in range(n):
                ready[i].wait()
                sites, amps, seq, offs, info = srv.wait(tickets[i])
                h = hashlib.sha1(sites.tobytes())
                h.update(amps.tobytes())
                h.update(seq)
                res[i] = (len(sites), len(amps), h.hexdigest(), info)
            thr.join()
        info = [r[3] for r in res]
        lat = np.array([x["done_ms"] - x["submit_ms"] for x in info])
        span = (max(x["done_ms"] for x in info) - min(x["submit_ms"] for x in info)) / 1e3
        return res, {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                     "mean_ms": float(lat.mean()), "makespan_s": span,
                     "gbps": sum(req_bases[:n]) / span / 1e9,
                     "batches": len({x["batch"] for x in info}),
                     "mean_batch": float(np.mean([x["batch_size"] for x in info])),
                     "max_batch": int(max(x["batch_size"] for x in info))}

    # warm-up: the scan variant of every (pair, k) compiles on first use
    with ah.Server(ctx, sid, mem_budget=args.mem_budget, max_batch=1) as srv:
        for j in range(len(pairs)):
            for k in range(5):
                srv.wait(srv.submit(np.arange(0, 2, dtype=np.uint32), pid[j], k, True))
    serve(np.zeros(R), args.max_batch, args.mem_budget, n=min(R, 100))
    arr = np.cumsum(rng.exponential(1.0 / args.rate, size=R))
    res_p, poisson = serve(arr, args.max_batch, args.mem_budget)
    res_s, saturated = serve(np.zeros(R), args.max_batch, args.mem_budget)
    for x, y in zip(res_p, res_s):   # the same results whatever they were batched with
        assert x[:3] == y[:3]
    # stage split of a saturated pass (untimed, events around every stage)
    ctx.ah_set_profiling(1)
    _, prof_run = serve(np.zeros(R), args.max_batch, args.mem_budget, n=min(R, 400))
    stages = {"requests": min(R, 400), "makespan_s": prof_run["makespan_s"]}
    for name in ("scan", "sort", "decode", "tm", "pair", "fetch", "host.serve.tiles", "host.serve.device",
                 "host.serve.filter_wait", "host.serve.fetch", "host.serve.batch"):
        ms, l, calls = ctx.ah_get_profile(name)
        stages[name] = {"ms": ms, "launches": l, "calls": calls}
    ctx.ah_set_profiling(0)
    # sequential plain solves: each request's genomes gathered into one buffer
    # (untimed), packed as their own set, one ah_run
    ctx_pids = {}
    out = HostOut(torch, ah)
    hs = torch.cuda.current_stream()
    goff = coll.genome_off.astype(np.int64)
    coff = coll.contig_off.astype(np.int64)
    cfirst = np.searchsorted(coff, goff[:-1], side="left")
    clast = np.searchsorted(coff, goff[1:], side="left")
    gbuf = torch.empty(max(req_bases), dtype=torch.uint8, device="cuda")
    t_seq = 0.0
    lat = []
    for (g, j, k), rr in zip(req, res_s):
        if (j, k) not in ctx_pids:
            p = dict(pairs[j], k=k)
            ctx_pids[(j, k)] = ctx.ah_set_primers(p["fwd"], p["rev"], p)
        parts, offs, gens, o = [], [0], [], 0
        for x in g.tolist():
            parts.append(dev[int(goff[x]):int(goff[x + 1])])
            c = coff[cfirst[x]:clast[x] + 1] - goff[x] + o
            offs.extend(c[1:].tolist())
            gens.extend([x] * (clast[x] - cfirst[x]))
            o += int(gbases[x])
        torch.cat(parts, out=gbuf[:o])
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        s2 = ctx.ah_load_genomes(gbuf, o, np.array(offs, np.uint64), np.array(gens, np.uint32), hs)
        out.run(ctx, s2, [ctx_pids[(j, k)]], hs)
        ctx.ah_unload_genomes(s2)
        dt = time.perf_counter() - t1
        t_seq += dt
        lat.append(dt * 1e3)
        assert out.o.n_sites == rr[0] and out.o.n_amplicons == rr[1]
    seq_plain = {"gbps": sum(req_bases) / t_seq / 1e9, "s": t_seq, "p50_ms": float(np.percentile(lat, 50)),
                 "p99_ms": float(np.percentile(lat, 99)),
                 "form": "each request alone: its genomes (gathered in device memory, untimed) packed as "
                         "their own set, one ah_run"}
    ctx.ah_unload_genomes(sid)
    line = {
        "form": "served", "metric": "p50/p99 request latency; aggregate Gbp/s scanned per primer pair",
        "value": saturated["gbps"], "unit": "Gbp/s", "n_gpus": 1, "higher_is_better": True,
        "data": "synthetic (counter-based, seed 3)",
        "config": {"workload": f"served-pool{n_g}genomes-{N / 1e9:.1f}Gbp-8pairs", "n_genomes": n_g, "n_bases": N,
                   "requests": R, "rate_per_s": args.rate,
                   "subset": "Zipf size over 1..n (P ~ 1/s), members uniform without replacement",
                   "k": "uniform 0..4", "pairs": [(p["fwd"], p["rev"]) for p in pairs], "tm_filter": True,
                   "max_batch": args.max_batch, "mem_budget": args.mem_budget, "layout_s": t_layout,
                   "request_gbp_total": sum(req_bases) / 1e9},
        "poisson": poisson, "saturated": saturated, "sequential_plain": seq_plain, "stages_ms_saturated": stages,
        "saturated_over_sequential": saturated["gbps"] / seq_plain["gbps"],
        "same_results_poisson_and_saturated": True,   # per-request digests compared above
    }
    if emit:
        print(json.dumps(line), flush=True)
    ctx.close()
    return line


def large_pairs():
    """The 960-oligo pair and two further pairs of 64 and 256 oligos (sum of the
    two primers' degeneracies), k = 4, window 100-3000 bp, Tm threshold 50 C."""
    from paper_2509_13300_gb300 import synth
    rng = np.random.default_rng(7)
    mk = lambda f, r: synth.pcr_params(f, r, k=4, min_len=100, max_len=3000, tm_min=50.0)
    p960 = mk("AGRRTTYGATYHTDGYTYAG", "YCNTTCCYTYDYRGTACT")
    p64 = mk(synth.random_primer(rng, 19, "RYSWK"), synth.random_primer(rng, 21, "WKMRY"))
    p256 = mk(synth.random_primer(rng, 22, "RYSWKMR"), synth.random_primer(rng, 24, "KMRYSWK"))
    return [p960, p64, p256]


class DevOut:
    """Device output buffers of one ah_run (grown on overflow)."""

    def __init__(self, torch, ah, caps):
        self.torch, self.ah = torch, ah
        self.alloc(caps)

    def alloc(self, caps):
        t = self.torch
        s, a, q = (max(int(x), 1) for x in caps)
        self.b = None
        t.cuda.empty_cache()
        self.b = [t.empty(n, dtype=t.uint8, device="cuda") for n in (16 * s, 4 * s, s, 28 * a, q, 8 * (a + 1))]
        self.o = self.ah.RunOut(self.b[0].data_ptr(), s, 0, self.b[1].data_ptr(), self.b[2].data_ptr(),
                                self.b[3].data_ptr(), a, 0, self.b[4].data_ptr(), q, 0, self.b[5].data_ptr(), 1, 0)

    def run(self, ctx, sid, pids, stream):
        for _ in range(3):
            try:
                return ctx.ah_run(sid, pids, self.o, stream)
            except self.ah.AHError as e:
                if e.status != self.ah.AH_ERR_OVERFLOW:
                    raise
                o = self.o
                self.alloc((o.n_sites * 5 // 4 + 1, o.n_amplicons * 5 // 4 + 1, o.n_seq * 5 // 4 + 1))
        raise RuntimeError("ah_run kept overflowing")

    def host_seq(self, m, q):
        """Sequence bytes and offsets of the last run's m amplicons."""
        return (self.b[4][:q].cpu().numpy().tobytes(), self.b[5][:8 * (m + 1)].cpu().numpy().view(np.uint64))

    def host(self, n, m):
        """Sites, Tm, pass and amplicons of the last run, as numpy arrays."""
        from paper_2509_13300_gb300 import ah
        b = [x.cpu().numpy() for x in self.b[:4]]
        return (b[0][:16 * n].view(ah.SITE_DTYPE), b[1][:4 * n].view(np.float32), b[2][:n],
                b[3][:28 * m].view(ah.AMPLICON_DTYPE))


def genome_slice(coll, chunk_tab, res, g):
    """Results of genome g out of its chunk's run, re-indexed as the genome alone:
    contigs from 0, amplicon ends indexing the genome's own site list."""
    from paper_2509_13300_gb300 import ah
    b0, b1, off, gen_ = chunk_tab
    sites, tm, ps, amps = res
    sel = np.nonzero(sites["genome"] == g)[0]
    c0 = int(np.nonzero(gen_ == g)[0][0])
    sg = sites[sel].copy()
    sg["contig"] -= c0
    remap = np.full(len(sites), -1, np.int64)
    remap[sel] = np.arange(len(sel))
    am = amps[amps["genome"] == g].copy()
    am["contig"] -= c0
    am["left"] = remap[am["left"]]
    am["right"] = remap[am["right"]]
    return sg, tm[sel].copy(), ps[sel].copy(), am


def check_genome_against_oracle(coll, pairs, g, got, cores):
    """The oracle on genome g alone (bases from the CPU twin); exact sites,
    pass flags and amplicons, Tm within 0.01 C."""
    import oracle
    a, b = int(coll.genome_off[g]), int(coll.genome_off[g + 1])
    seq = coll.bases(a, b)
    c0 = int(np.searchsorted(coll.contig_off, a, side="left"))
    c1 = int(np.searchsorted(coll.contig_off, b, side="left"))
    off = (coll.contig_off[c0:c1 + 1] - np.uint64(a)).astype(np.uint64)
    gen_ = np.full(c1 - c0, g, dtype=np.uint32)
    s = oracle.scan(seq, off, gen_, pairs, n_threads=cores)
    tm, ps = oracle.tm(seq, off, s, pairs, n_threads=cores)
    am = oracle.pair(s, pairs, ps)
    sg, tg, pg, ag = got
    ok = ~np.isnan(tm)
    return {"genome": int(g), "bases": b - a, "sites": len(s), "amplicons": len(am),
            "sites_equal": sg.tobytes() == s.tobytes(), "pass_equal": bool(np.array_equal(pg, ps)),
            "tm_nan_equal": bool(np.array_equal(np.isnan(tg), ~ok)),
            "tm_max_err": float(np.abs(tg[ok].astype(np.float64) - tm[ok]).max()) if ok.any() else 0.0,
            "amplicons_equal": ag.tobytes() == am.tobytes()}


LARGE_WORKLOAD = "large-50000genomes-169Gbp-3pairs-k4"


def large_collection(seed: int = 7, n_genomes: int | None = None):
    """The large workload's layout: 50,000 counter-generated genomes of 1-8 Mbp
    (seed 7), the three pairs of large_pairs()."""
    from paper_2509_13300_gb300 import countergen
    return countergen.collection(seed=seed, n_genomes=n_genomes or 50_000, len_lo=1e6, len_hi=8e6,
                                 pairs=large_pairs())


def oracle_sample(coll, target_s: float, cores: int, seed: int = 7):
    """Genomes drawn in a seeded random order until about target_s of oracle
    work (the oracle scans ~0.12 Mbp/s per core with these three pairs at k = 4)."""
    order = np.random.default_rng(seed).permutation(len(coll.genome_off) - 1)
    gl = np.diff(coll.genome_off.astype(np.int64))
    want = max(1.0e6, 0.12e6 * cores * target_s)
    n = int(np.searchsorted(np.cumsum(gl[order]), want)) + 1
    return np.sort(order[:max(1, min(n, len(order)))])


def oracle_on_genomes(coll, pairs, genomes, cores):
    """The oracle (scan, Tm, pair, fetch) on each genome alone; bases from the
    CPU twin of the counter-based generator.  Returns per genome (sites, Tm,
    pass, amplicons, sequences, sequence offsets) and the oracle's seconds."""
    import oracle
    out, t = {}, 0.0
    for g in genomes.tolist():
        a, b = int(coll.genome_off[g]), int(coll.genome_off[g + 1])
        seq = coll.bases(a, b)
        c0 = int(np.searchsorted(coll.contig_off, a, side="left"))
        c1 = int(np.searchsorted(coll.contig_off, b, side="left"))
        off = (coll.contig_off[c0:c1 + 1] - np.uint64(a)).astype(np.uint64)
        gen_ = np.full(c1 - c0, g, dtype=np.uint32)
        t0 = time.perf_counter()
        s_ = oracle.scan(seq, off, gen_, pairs, n_threads=cores)
        tm, ps = oracle.tm(seq, off, s_, pairs, n_threads=cores)
        am = oracle.pair(s_, pairs, ps)
        qs, qo = oracle.fetch(seq, off, am)
        t += time.perf_counter() - t0
        out[g] = (s_, tm, ps, am, qs, qo)
    return out, t


def parity_summary(coll, got, want):
    """Compare the GPU's records of each sampled genome with the oracle's:
    bit-exact sites, pass flags, amplicons and sequences; Tm within 0.01 C."""
    res = {"genomes": 0, "bases": 0, "sites": 0, "amplicons": 0, "sites_equal": True, "pass_equal": True,
           "tm_nan_equal": True, "amplicons_equal": True, "sequences_equal": True, "max_dtm_C": 0.0}
    for g, (s_, tm, ps, am, qs, qo) in want.items():
        sg, tg, pg, ag, gq, go = got[g]
        ok = ~np.isnan(tm)
        res["genomes"] += 1
        res["bases"] += int(coll.genome_off[g + 1] - coll.genome_off[g])
        res["sites"] += len(s_)
        res["amplicons"] += len(am)
        res["sites_equal"] &= sg.tobytes() == s_.tobytes()
        res["pass_equal"] &= bool(np.array_equal(pg, ps))
        res["tm_nan_equal"] &= bool(np.array_equal(np.isnan(tg), ~ok))
        if ok.any() and len(tg) == len(tm):
            res["max_dtm_C"] = max(res["max_dtm_C"], float(np.abs(tg[ok].astype(np.float64) - tm[ok]).max()))
        res["amplicons_equal"] &= ag.tobytes() == am.tobytes()
        res["sequences_equal"] &= gq == qs and np.array_equal(go.astype(np.uint64), qo.astype(np.uint64))
    res["all_equal"] = bool(res["sites_equal"] and res["pass_equal"] and res["tm_nan_equal"] and
                            res["amplicons_equal"] and res["sequences_equal"] and res["max_dtm_C"] <= 0.01)
    return res


def genome_records(coll, chunk_tab, res, g):
    """Records of genome g out of its chunk's run outputs, re-indexed as the
    genome alone (contigs from 0, amplicon ends into the genome's own sites),
    with its amplicons' sequences and offsets."""
    sites, tm, ps, amps, seq, offs = res
    sg, tg, pg, am = genome_slice(coll, chunk_tab, (sites, tm, ps, amps), g)
    sel = np.nonzero(amps["genome"] == g)[0]
    parts = [seq[int(offs[i]):int(offs[i + 1])] for i in sel]
    q = b"".join(parts)
    qo = np.concatenate([[0], np.cumsum([len(x) for x in parts])]).astype(np.uint64)
    return sg, tg, pg, am, q, qo


def bench_large_main(args):
    """Default line: the large workload (50,000 genomes, 169 Gbp, three pairs of
    960, 64 and 256 oligos at k = 4, window 100-3000 bp, Tm threshold 50 C).

    The ASCII bases are generated on the device once, before the timed region
    (counter-based Philox4x32-10, seed 7 + rank), and stay resident in HBM.
    One step = one pass over the collection in chunks of whole genomes
    (<= 16 Gbp): pack (ah_load_genomes from the resident bases), scan of the
    three pairs, canonical sort, Tm, Tm-filtered pairing and fetch
    (ah_run_begin / ah_run_end) into device buffers; chunk i+1 packs on a
    second stream once chunk i's scan is done.  value = bases x pairs x steps /
    time.  Under torchrun every rank runs its own collection (weak scaling)."""
    rank, world, local = dist_info()
    import torch
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    from paper_2509_13300_gb300 import ah, build
    build.build()
    pairs = large_pairs()
    t0 = time.perf_counter()
    coll = large_collection(7 + rank, args.n_genomes)
    t_layout = time.perf_counter() - t0
    n_g = len(coll.genome_off) - 1
    N, npair = coll.n_bases, len(pairs)
    ctx = ah.Context(local)
    pids = [ctx.ah_set_primers(p["fwd"], p["rev"], p) for p in pairs]
    tabs = [sub_tables(coll, g0, g1) for g0, g1 in genome_chunks(coll, args.large_chunk)]
    cmax = max(b1 - b0 for b0, b1, _, _ in tabs)
    t0 = time.perf_counter()
    # resident ASCII, generated outside the timed region; every chunk 16-byte aligned
    seq_d, at = aligned_chunks(ctx, coll, tabs, torch)
    t_gen = time.perf_counter() - t0
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    scan_done = torch.cuda.Event()

    def load(i, s):
        b0, b1, off, gen_ = tabs[i]
        return ctx.ah_load_genomes(seq_d[at[i]:at[i] + b1 - b0], b1 - b0, off, gen_, s)

    # tuning on the first chunk; output capacities from one pass of ah_run
    sid = load(0, streams[0])
    tune = None if args.no_tune else ctx.ah_tune_scan(sid, pids, 0, streams[0])
    ctx.ah_unload_genomes(sid)
    out = DevOut(torch, ah, (cmax * 1.2e-3 * npair / 3, 1 << 16, 1 << 26))
    caps = [0, 0, 0]
    for i in range(len(tabs)):
        sid = load(i, streams[0])
        out.run(ctx, sid, pids, streams[0])
        o = out.o
        caps = [max(caps[0], o.n_sites), max(caps[1], o.n_amplicons), max(caps[2], o.n_seq)]
        ctx.ah_unload_genomes(sid)
    out.alloc((caps[0] * 9 // 8 + 1024, caps[1] * 9 // 8 + 64, caps[2] * 9 // 8 + 4096))
    totals = {}

    def one_pass(keep=None):
        """Every chunk once, two sets in flight: chunk i+1 is packed on the other
        stream once chunk i's scan has finished (ah_run_begin records scan_done)."""
        n_s = n_a = n_q = 0
        kept = {}
        prev = load(0, streams[0])
        for i in range(len(tabs)):
            ctx.ah_run_begin(prev, pids, out.o, streams[i % 2], scan_done)
            nxt = None
            if i + 1 < len(tabs):
                streams[(i + 1) % 2].wait_event(scan_done)
                nxt = load(i + 1, streams[(i + 1) % 2])
            ctx.ah_run_end(out.o)
            o = out.o
            n_s, n_a, n_q = n_s + o.n_sites, n_a + o.n_amplicons, n_q + o.n_seq
            if keep is not None and keep.get(i):
                torch.cuda.synchronize()
                res = out.host(o.n_sites, o.n_amplicons) + out.host_seq(o.n_amplicons, o.n_seq)
                for g in keep[i]:
                    kept[g] = genome_records(coll, tabs[i], res, g)
            ctx.ah_unload_genomes(prev)
            prev = nxt
        totals.update(sites=n_s, amplicons=n_a, seq_bytes=n_q)
        return kept

    for _ in range(max(3, args.warmup)):
        one_pass()
    torch.cuda.synchronize()
    # timed region: CUDA events on the launching streams; pack and scan stages timed live
    ctx.ah_set_profiling(3)
    barrier(world)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    with ClockSampler(local) as clk:
        clk.wait_first()
        clk.mark(True)
        ev[0].record(streams[0])
        for _ in range(args.steps):
            one_pass()
        streams[0].wait_stream(streams[1])
        ev[1].record(streams[0])
        torch.cuda.synchronize()
        clk.mark(False)
    barrier(world)
    t_ms = ev[0].elapsed_time(ev[1])
    t_max = max_over_ranks(t_ms, world)
    bases_all = sum_over_ranks(float(N), world)
    value = bases_all * npair * args.steps / (t_max / 1e3) / 1e9
    live = {}
    for st in ("pack", "scan"):
        ms, launches, calls = ctx.ah_get_profile(st)
        live[st] = {"ms_per_step": ms / args.steps, "launches_per_step": launches / args.steps}
    _, total_launches, _ = ctx.ah_get_profile(None)
    # stage breakdown: one more pass with events around every stage (untimed)
    ctx.ah_set_profiling(1)
    one_pass()
    stages = {"note": "untimed pass, CUDA events around every stage; chunk i+1's packing overlaps chunk i's run"}
    for st in ("pack", "tables", "scan", "sort", "decode", "tm", "pair", "fetch"):
        ms, launches, calls = ctx.ah_get_profile(st)
        stages[st] = {"ms_per_step": ms, "launches_per_step": launches}
    ctx.ah_set_profiling(0)
    # the packing alone: every chunk loaded with nothing else queued (events of the "pack" stage)
    ctx.ah_set_profiling(3)
    for i in range(len(tabs)):
        sid = load(i, streams[0])
        torch.cuda.synchronize()
        ctx.ah_unload_genomes(sid)
    pack_alone_ms, _, _ = ctx.ah_get_profile("pack")
    ctx.ah_set_profiling(0)

    # ---- roofline of the dominant kernel (live CUDA-event durations of the timed region) ----
    hbm_peak, peak_kind, _ = load_peaks()
    clocks = clk.summary()
    clk_mhz = clocks["sm_mhz"] or 2070.0
    scan_s = live["scan"]["ms_per_step"] / 1e3
    pack_s = live["pack"]["ms_per_step"] / 1e3
    words = N / 32.0
    lop = sum(ah.scan_lop3_per_word(p["fwd"], p["rev"], int(p["k"]), (tune or {}).get("R", 4), 0) for p in pairs)
    lanes, lanes_src = logic_lanes(ah)
    alu_peak = SMS * lanes * clk_mhz * 1e6 / 1e12
    scan_tops = lop * words / scan_s / 1e12
    # each launch group reads its chunk's planes once
    scan_hbm = 0.5 * N * (live["scan"]["launches_per_step"] / len(tabs)) / scan_s / 1e9
    pack_hbm = 1.5 * N / pack_s / 1e9
    # the scan dominates the serialised launch list; the packing's live time is
    # stretched by the run it overlaps, so it is reported beside (pack_roofline)
    tr_pack = traffic_record("pack_kernel")
    per_launch = N / len(tabs)  # bases per chunk: one packing and one launch per launch group
    pack_roof = {"bound": "hbm", "achieved": pack_hbm, "peak": hbm_peak, "unit": "GB/s", "frac": pack_hbm / hbm_peak,
                 "traffic": tr_pack["dram_bytes_per_base"] * per_launch if tr_pack else None, "kernel": "pack_kernel",
                 "peak_kind": peak_kind, "algorithmic": "1.5 B/base (1 B ASCII read + 0.5 B planes written)",
                 "note": "live duration includes the sort/Tm/pair/fetch kernels of the previous chunk it runs beside"}
    pack_alone = 1.5 * N / (pack_alone_ms / 1e3) / 1e9
    pack_roof["alone"] = {"achieved": pack_alone, "frac": pack_alone / hbm_peak, "ms_per_pass": pack_alone_ms,
                          "note": "every chunk packed with nothing else on the GPU, outside the timed region"}
    tr = traffic_record("ah_scan_kernel")
    roof = {"bound": "alu", "achieved": scan_tops, "peak": alu_peak, "unit": "Tops/s",
            "frac": scan_tops / alu_peak, "traffic": tr["dram_bytes_per_base"] * per_launch if tr else None,
            "kernel": "ah_scan_kernel",
            "peak_note": f"logic pipe: {SMS} SMs x {lanes:.1f} LOP3 lanes/clk x {clk_mhz:.0f} MHz (median SM clock "
                         f"under load); lanes {lanes_src}",
            "algorithmic": f"{lop} LOP3 per 32 starts for the three pairs ({len(tabs)} chunks x "
                           f"{live['scan']['launches_per_step'] / len(tabs):.0f} launches per chunk)",
            "hbm_achieved_gbs": scan_hbm, "hbm_peak_gbs": hbm_peak, "hbm_frac": scan_hbm / hbm_peak,
            "hbm_peak_kind": peak_kind, "hbm_algorithmic": "0.5 B/base of planes per launch"}
    roof["scope"] = ("achieved: all launches of the kernel in one step; traffic: DRAM bytes of one launch (one launch "
                     "group over an average chunk), scaled by bases from an ncu capture of a 0.31 Gbp launch")

    # ---- end to end through the C ABI: host (pinned) input and outputs, the first chunks ----
    e2e = None
    ne = min(max(0, args.e2e_chunks), len(tabs))
    if ne > 0:
        torch.cuda.empty_cache()
        hout = HostOut(torch, ah, (caps[0] * 9 // 8 + 1024, caps[1] * 9 // 8 + 64, caps[2] * 9 // 8 + 4096))
        reps = max(2, args.e2e_steps // 2)

        def measure(n_chunks, load, in_bytes):
            """reps steps over the first n_chunks chunks from host input; the next
            chunk's host load (copies + packing) is issued while the current run computes."""
            def host_pass():
                h2d = d2h = 0
                prev = load(0, streams[0])
                h2d += in_bytes[0]
                for i in range(n_chunks):
                    ctx.ah_run_begin(prev, pids, hout.o, streams[i % 2], None)
                    nxt = None
                    if i + 1 < n_chunks:
                        nxt = load(i + 1, streams[(i + 1) % 2])
                        h2d += in_bytes[i + 1]
                    ctx.ah_run_end(hout.o)
                    d2h += hout.d2h_bytes()
                    ctx.ah_unload_genomes(prev)
                    prev = nxt
                return h2d, d2h

            host_pass()
            barrier(world)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(streams[0])
            for _ in range(reps):
                h2d, d2h = host_pass()
            streams[0].wait_stream(streams[1])
            e1.record(streams[0])
            torch.cuda.synchronize()
            e_ms = max_over_ranks(e0.elapsed_time(e1), world)
            sub = sum_over_ranks(float(sum(tabs[i][1] - tabs[i][0] for i in range(n_chunks))), world)
            return sub * npair * reps / (e_ms / 1e3) / 1e9, int(h2d), int(d2h)

        # 2-bit codes and no-base runs in pinned host memory (encoded before the timed region)
        codes_h, gaps_h = [], []
        for i in range(ne):
            b0, b1 = tabs[i][0], tabs[i][1]
            cd, gp = device_encode_2bit(torch, seq_d[at[i]:at[i] + b1 - b0])
            ch = torch.empty(cd.numel(), dtype=torch.uint8, pin_memory=True)
            ch.copy_(cd)
            del cd
            codes_h.append(ch)
            gaps_h.append(gp)

        # the host link alone on this machine: one pinned host -> device copy of the first chunk's codes
        link_gbs = None
        if codes_h:
            dtmp = torch.empty(codes_h[0].numel(), dtype=torch.uint8, device="cuda")
            l0, l1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            for _ in range(2):
                l0.record(streams[0])
                with torch.cuda.stream(streams[0]):
                    dtmp.copy_(codes_h[0], non_blocking=True)
                l1.record(streams[0])
                torch.cuda.synchronize()
            link_gbs = codes_h[0].numel() / (l0.elapsed_time(l1) / 1e3) / 1e9
            del dtmp
            torch.cuda.empty_cache()

        def load2(i, st_):
            b0, b1, off, gen_ = tabs[i]
            return ctx.ah_load_genomes_2bit(codes_h[i], b1 - b0, gaps_h[i], off, gen_, st_, host_async=True)

        in2 = [codes_h[i].numel() + gaps_h[i].nbytes + tabs[i][2].nbytes + tabs[i][3].nbytes for i in range(ne)]
        v2, h2d2, d2h2 = measure(ne, load2, in2)
        del codes_h
        # the same from ASCII host input, first chunk (the link carries 4x the bytes)
        b0, b1, off0, gen0 = tabs[0]
        host = torch.empty(b1 - b0, dtype=torch.uint8, pin_memory=True)
        host.copy_(seq_d[at[0]:at[0] + b1 - b0])
        va, h2da, d2ha = measure(1, lambda i, st_: ctx.ah_load_genomes(host, b1 - b0, off0, gen0, st_, host_async=True),
                                 [b1 - b0 + off0.nbytes + gen0.nbytes])
        del host
        sub_gbp = sum(tabs[i][1] - tabs[i][0] for i in range(ne)) / 1e9
        e2e = {"value": v2, "unit": "Gbp/s", "h2d_bytes_per_step": h2d2, "d2h_bytes_per_step": d2h2, "steps": reps,
               "input": "2-bit base codes + no-base runs from pinned host memory (ah_load_genomes_2bit); outputs "
                        "(sites, Tm, pass flags, amplicons, sequences) to pinned host memory",
               "subset": f"first {ne} of {len(tabs)} chunks ({sub_gbp:.1f} Gbp of {N / 1e9:.1f}) per step",
               "pipeline": "the next chunk's host load (copy + packing) is issued while the current run computes; "
                           "host loads are queued without waiting for their copies (AH_LOAD_HOST_ASYNC: the pinned "
                           "inputs stay unchanged until the sets are ready)",
               "link_h2d_gbs": link_gbs,
               "ascii_input": {"value": va, "unit": "Gbp/s", "h2d_bytes_per_step": h2da, "d2h_bytes_per_step": d2ha,
                               "subset": f"first chunk ({(b1 - b0) / 1e9:.1f} Gbp) from ASCII (ah_load_genomes)"}}

    # ---- oracle sample: the CPU baseline and parity with the GPU's records of the same genomes ----
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        sample = oracle_sample(coll, 15.0, cores)
        chunk_of = np.searchsorted(np.array([b1 for _, b1, _, _ in tabs]), coll.genome_off[sample], side="right")
        keep = {}
        for g, ci in zip(sample.tolist(), chunk_of.tolist()):
            keep.setdefault(ci, []).append(g)
        got = one_pass(keep)
        want, t_cpu = oracle_on_genomes(coll, pairs, sample, cores)
        nb = int(sum(coll.genome_off[g + 1] - coll.genome_off[g] for g in sample.tolist()))
        cpu = {"value": nb * npair / t_cpu / 1e9, "unit": "Gbp/s", "cores": cores, "kind": "oracle",
               "sample": f"{len(sample)} of {n_g} genomes drawn with seed 7 ({nb / 1e6:.1f} Mbp), 3 pairs, "
                         f"scan+Tm+pair+fetch, {t_cpu:.1f} s",
               "parity": parity_summary(coll, got, want)}
    if rank == 0 and world == 1 and args.dump_genomes:
        # GPU records of a seeded sample of genomes from one pass of the timed configuration,
        # for the oracle to check on another machine (--check-dump regenerates the genomes)
        dump = np.sort(np.random.default_rng(7).choice(n_g, size=min(args.dump_genomes, n_g), replace=False))
        chunk_of = np.searchsorted(np.array([b1 for _, b1, _, _ in tabs]), coll.genome_off[dump], side="right")
        keep = {}
        for g, ci in zip(dump.tolist(), chunk_of.tolist()):
            keep.setdefault(ci, []).append(g)
        got = one_pass(keep)
        arrs = {}
        for g in dump.tolist():
            sg, tg, pg, ag, _, _ = got[g]
            arrs.update({f"s{g}": sg, f"t{g}": tg, f"p{g}": pg, f"a{g}": ag})
        np.savez_compressed(args.dump_path, sample=dump, n_genomes=n_g, **arrs)
    del seq_d
    ctx.close()
    torch.cuda.empty_cache()

    # ---- the collection workload's key (100 genomes, 0.4 Gbp, one pair, k = 3) ----
    coll_key = None
    if not args.no_collection and world == 1:
        sub = argparse.Namespace(**vars(args))
        sub.steps, sub.warmup, sub.e2e_steps, sub.no_cpu_baseline, sub.n_genomes = 400, 5, 20, True, None
        c = bench_collection(sub, emit=False)
        if c:
            coll_key = {"workload": c["config"]["workload"], "value": c["value"], "unit": c["unit"],
                        "ms_per_step": c["ms_per_step"], "steps": sub.steps,
                        "timed_region_kernel_us": c["timed_region_kernel_us"], "roofline": c["roofline"],
                        "e2e": c["e2e"]}
    forms = None
    if not args.no_forms and world == 1:
        forms = form_keys(args)
    if rank != 0:
        return None
    line = {
        "metric": METRIC, "value": value, "unit": "Gbp/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32+f32",
        "data": "synthetic (counter-based Philox4x32-10 bases, seed 7 + rank, generated on the device)",
        "config": {"workload": LARGE_WORKLOAD if n_g == 50_000 else f"large-{n_g}genomes-{N / 1e9:.1f}Gbp-3pairs-k4",
                   "n_genomes": n_g, "n_bases_per_gpu": N,
                   "n_contigs": len(coll.contig_genome), "pairs": npair, "oligos": [960, 64, 256], "k": 4,
                   "window": [100, 3000], "tm_min_C": 50.0, "tm_dtype": "f32", "chunks": len(tabs),
                   "chunk_bases_max": cmax, "parallelism": f"replicas x{world}", "scan_tuning": tune,
                   "value_counts": "bases x primer pairs per second (each base once per pair scanned)",
                   "input": "ASCII bases resident in HBM (generated before the timed region), each chunk "
                            "at a 16-byte aligned address",
                   "l2": "inputs larger than L2 (169 GB resident ASCII; up to 8 GB of planes per chunk)",
                   "layout_s": t_layout, "generation_s": t_gen},
        "results_per_pass": dict(totals), "amplicons_per_s": totals["amplicons"] * args.steps / (t_max / 1e3),
        "stages": stages, "roofline": roof, "pack_roofline": pack_roof, "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": int(total_launches), "clocks": clocks,
        "timed_region_ms_per_step": {st: live[st]["ms_per_step"] for st in live},
        "collection": coll_key, "forms": forms,
    }
    print(json.dumps(line), flush=True)
    return line


def form_keys(args):
    """The batched and served forms on their own workloads (10,000 genomes
    streamed from pinned host memory against one load and run per genome; a
    resident 5,000-genome pool serving Poisson-arriving requests, then the
    same requests all at once, against sequential plain solves), run after the
    large workload's memory is released.  A form that fails is reported by its
    error and does not stop the line."""
    import torch
    out = {}
    for name, fn, over in (("batched", bench_batched, {"steps": 2, "warmup": 3}),
                           ("served", bench_served, {"requests": args.forms_requests})):
        sub = argparse.Namespace(**vars(args))
        sub.n_genomes = None
        for k, v in over.items():
            setattr(sub, k, v)
        t0 = time.perf_counter()
        r = None
        try:
            r = fn(sub, emit=False)
        except Exception as e:  # noqa: BLE001 - reported in the line
            out[name] = {"error": f"{type(e).__name__}: {e}"[:300]}
        try:  # the form's memory back before the next one (a failed form may leave the device unusable)
            torch.cuda.synchronize()
            torch.cuda.empty_cache()
        except Exception:  # noqa: BLE001
            pass
        if r is None:
            continue
        if name == "batched":
            out[name] = {"workload": r["config"]["workload"], "value": r["value"], "unit": r["unit"],
                         "s_per_pass": r["s_per_pass"], "steps": r["steps"],
                         "plain": {"value": r["plain"]["value"], "form": r["plain"]["form"],
                                   "genomes": r["plain"]["genomes"]},
                         "plain_all_pairs": {"value": r["plain_all_pairs"]["value"],
                                             "form": r["plain_all_pairs"]["form"]},
                         "batched_over_plain": r["batched_over_plain"],
                         "batched_over_plain_all_pairs": r["batched_over_plain_all_pairs"],
                         "input": r["config"]["input"], "h2d_gbs": r["h2d_gbs"],
                         "results_per_pass": r["results_per_pass"], "clocks": r["clocks"]}
        else:
            out[name] = {"workload": r["config"]["workload"], "requests": r["config"]["requests"],
                         "rate_per_s": r["config"]["rate_per_s"], "k": r["config"]["k"],
                         "max_batch": r["config"]["max_batch"], "mem_budget": r["config"]["mem_budget"],
                         "poisson": r["poisson"], "saturated": r["saturated"],
                         "sequential_plain": r["sequential_plain"],
                         "saturated_over_sequential": r["saturated_over_sequential"],
                         "same_results_poisson_and_saturated": r["same_results_poisson_and_saturated"]}
        out[name]["wall_s"] = time.perf_counter() - t0
    return out


def bench_hmm(args):
    """Profile-HMM form: a profile trained on the exact-match amplicons of an
    operon family scores every k = 2 amplicon of the collection (glocal Viterbi,
    fp32, and the Forward score beside it); throughput in cell updates per
    second, a sample checked by the oracle."""
    import torch
    from paper_2509_13300_gb300 import ah, build, synth
    build.build()
    torch.cuda.set_device(0)
    n_g = args.n_genomes or 2000
    t0 = time.perf_counter()
    w = synth.operon_family(seed=21, n_genomes=n_g)
    t_gen = time.perf_counter() - t0
    p = w.pairs[0]
    p0 = dict(p, k=0)
    ctx = ah.Context(0)
    sid = ctx.load(w.seq, w.contig_off, w.contig_genome)
    pid0 = ctx.ah_set_primers(p0["fwd"], p0["rev"], p0)
    pid2 = ctx.ah_set_primers(p["fwd"], p["rev"], p)
    r0 = ctx.run(sid, [pid0], tm_filter=False)
    train = [r0["seqs"][int(r0["offs"][i]):int(r0["offs"][i + 1])] for i in range(len(r0["amps"]))]
    t0 = time.perf_counter()
    hid = ctx.hmm_build(train)
    t_build = time.perf_counter() - t0
    m, ref, T, E = ctx.hmm_tables(hid)
    r2 = ctx.run(sid, [pid2], tm_filter=False)
    amps = r2["amps"]
    lens = (amps["end"] - amps["start"]).astype(np.int64)
    cells = float(lens.sum()) * m
    dev_amps = torch.from_numpy(amps.view(np.uint8).copy()).cuda()
    out = torch.zeros(len(amps), dtype=torch.float32, device="cuda")
    stream = torch.cuda.Stream()
    for _ in range(max(1, args.warmup)):
        ctx.hmm_score(sid, hid, dev_amps, n=len(amps), out=out, stream=stream)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    torch.cuda.synchronize()
    with ClockSampler(0) as clk:
        clk.wait_first()
        clk.mark(True)
        ev[0].record(stream)
        for _ in range(args.steps):
            ctx.hmm_score(sid, hid, dev_amps, n=len(amps), out=out, stream=stream)
        ev[1].record(stream)
        torch.cuda.synchronize()
        clk.mark(False)
    dt = ev[0].elapsed_time(ev[1]) / 1e3 / args.steps
    got = out.cpu().numpy()
    # the Forward score (log-sum over state paths) of the same amplicons, timed the same way
    out_f = torch.zeros(len(amps), dtype=torch.float32, device="cuda")
    for _ in range(max(1, args.warmup)):
        ctx.hmm_forward(sid, hid, dev_amps, n=len(amps), out=out_f, stream=stream)
    torch.cuda.synchronize()
    ev[0].record(stream)
    for _ in range(args.steps):
        ctx.hmm_forward(sid, hid, dev_amps, n=len(amps), out=out_f, stream=stream)
    ev[1].record(stream)
    torch.cuda.synchronize()
    dt_f = ev[0].elapsed_time(ev[1]) / 1e3 / args.steps
    got_f = out_f.cpu().numpy()
    # the other kernel of each score on the same amplicons (AH_HMM_KERNEL), for comparison
    other = {}
    try:
        for name, kern, fn, o in (("viterbi", "wave", ctx.hmm_score, out), ("forward", "rows", ctx.hmm_forward, out_f)):
            os.environ["AH_HMM_KERNEL"] = kern
            fn(sid, hid, dev_amps, n=len(amps), out=o, stream=stream)
            torch.cuda.synchronize()
            ev[0].record(stream)
            for _ in range(args.steps):
                fn(sid, hid, dev_amps, n=len(amps), out=o, stream=stream)
            ev[1].record(stream)
            torch.cuda.synchronize()
            d = ev[0].elapsed_time(ev[1]) / 1e3 / args.steps
            other[name] = {"kernel": kern, "value": cells / d / 1e9, "unit": "GCUPS", "ms_per_step": d * 1e3}
        other["viterbi"]["max_abs_diff_bits"] = float(np.abs(out.cpu().numpy() - got).max())
        other["forward"]["max_abs_diff_bits"] = float(np.abs(out_f.cpu().numpy() - got_f).max())
    finally:
        os.environ.pop("AH_HMM_KERNEL", None)
    # the oracle on a sample: its own profile from the same training sequences
    import oracle
    rng = np.random.default_rng(0)
    sample = np.sort(rng.choice(len(amps), size=min(len(amps), args.check_genomes * 4), replace=False))
    oref, oT, oE = oracle.hmm_build([x.decode() for x in train])
    qs, qo = oracle.fetch(w.seq, w.contig_off, amps[sample])
    t0 = time.perf_counter()
    want = np.array([oracle.hmm_viterbi(oT, oE, qs[int(qo[i]):int(qo[i + 1])].decode()) for i in range(len(sample))])
    t_cpu = time.perf_counter() - t0
    want_f = np.array([oracle.hmm_forward(oT, oE, qs[int(qo[i]):int(qo[i + 1])].decode())
                       for i in range(len(sample))])
    cpu_cells = float(lens[sample].sum()) * m
    # fp32 accumulation along a path of N = n + m moves, ten standard deviations of
    # a random walk of roundings (the bound of the parity tests)
    pmean = float(np.concatenate([np.abs(oT[~np.isinf(oT)]), np.abs(oE[1:]).ravel()]).mean())
    N = lens[sample] + m
    tol = 10.0 * np.sqrt(N) * 2.0 ** -24 * (np.abs(want) + N * pmean) + 1e-4
    tol_f = 10.0 * np.sqrt(N) * (2.0 ** -24 * (np.abs(want_f) + N * pmean) + 4 * 2.0 ** -23) + 1e-4
    err = np.abs(got[sample].astype(np.float64) - want)
    err_f = np.abs(got_f[sample].astype(np.float64) - want_f)
    clocks = clk.summary()
    # FADD + FMNMX per cell of the recurrence (M 6, I 5, D 5); the block-per-group kernel
    # that scores Viterbi executes 19 (its delete-chain scan evaluates D's terms twice)
    fp_ops_per_cell = 16
    fp32_peak = 152 * 128 * (clocks["sm_mhz"] or 2070.0) * 1e6
    achieved = cells / dt * fp_ops_per_cell
    line = {
        "form": "hmm", "metric": "cell updates per second (glocal Viterbi, profile x amplicon)",
        "value": cells / dt / 1e9, "unit": "GCUPS", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt * 1e3, "higher_is_better": True, "data": "synthetic (operon family, seed 21)",
        "config": {"workload": f"hmm-operonfamily-{n_g}genomes", "n_bases": w.n_bases, "profile_columns": m,
                   "training_amplicons": len(train), "reference_index": ref, "scored_amplicons": len(amps),
                   "letters_scored": int(lens.sum()), "generation_s": t_gen, "profile_build_s": t_build},
        "amplicons_per_s": len(amps) / dt,
        "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": fp32_peak / 1e12, "unit": "TFLOP/s (fp32 add/max)",
                     "frac": achieved / fp32_peak, "ops_per_cell": fp_ops_per_cell,
                     "peak_note": "152 SMs x 128 fp32 lanes x median SM clock"},
        "oracle_check": {"amplicons": len(sample), "max_abs_err_bits": float(err.max()) if len(err) else 0.0,
                         "within_fp32_bound": bool((err <= tol).all()), "min_bound_bits": float(tol.min()) if len(tol) else 0.0},
        "forward": {"value": cells / dt_f / 1e9, "unit": "GCUPS", "ms_per_step": dt_f * 1e3,
                    "score": "glocal Forward (log-sum over state paths), fp32",
                    "oracle_check": {"amplicons": len(sample),
                                     "max_abs_err_bits": float(err_f.max()) if len(err_f) else 0.0,
                                     "within_fp32_bound": bool((err_f <= tol_f).all())}},
        "kernels": {"viterbi": "hmm_score_kernel (a block per group of amplicons, rows in lockstep)",
                    "forward": "hmm_wave_kernel (one warp per amplicon, anti-diagonal steps)"},
        "other_kernel": other,
        "cpu_baseline": {"value": cpu_cells / t_cpu / 1e9, "unit": "GCUPS", "cores": 1, "kind": "oracle",
                         "sample": f"{len(sample)} amplicons, fp64 Viterbi, {t_cpu:.1f} s"},
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    ctx.hmm_free(hid)
    ctx.ah_unload_genomes(sid)
    ctx.close()

def check_large_dump(path: str):
    """The oracle, on this machine, against the GPU results a large-form run
    dumped for its sampled genomes (the genomes are regenerated by the CPU twin)."""
    from paper_2509_13300_gb300 import countergen
    d = np.load(path)
    n_g = int(d["n_genomes"])
    pairs = large_pairs()
    coll = countergen.collection(seed=7, n_genomes=n_g, len_lo=1e6, len_hi=8e6, pairs=pairs)
    cores = os.cpu_count() or 1
    res = []
    t0 = time.perf_counter()
    for g in d["sample"].tolist():
        got = (d[f"s{g}"], d[f"t{g}"], d[f"p{g}"], d[f"a{g}"])
        r = check_genome_against_oracle(coll, pairs, g, got, cores)
        res.append(r)
        print(json.dumps(r), flush=True)
    ok = all(r["sites_equal"] and r["pass_equal"] and r["tm_nan_equal"] and r["amplicons_equal"]
             and r["tm_max_err"] <= 0.01 for r in res)
    print(json.dumps({"genomes": len(res), "all_equal": ok, "bases": sum(r["bases"] for r in res),
                      "sites": sum(r["sites"] for r in res), "amplicons": sum(r["amplicons"] for r in res),
                      "tm_max_err": max(r["tm_max_err"] for r in res), "cores": cores,
                      "seconds": time.perf_counter() - t0}), flush=True)
    return 0 if ok else 1

if __name__ == "__main__":
    main()
