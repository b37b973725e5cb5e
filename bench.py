#!/usr/bin/env python3
"""Benchmark of the in-silico PCR hot path on one GB300 (or N, one process per GPU).

Workload (N = 1): the genome-collection configuration -- 100 synthetic
genomes, lengths log-uniform in 2-7 Mbp (~0.4 Gbp), 1-200 contigs each, GC
U(0.3, 0.7), 0.1% N runs, planted operon-like regions; one degenerate pair of
20 and 22 nt with 960 oligos in total; k = 3; window 100-2500 bp; Tm with
50 mM Na+, 0.25 uM primer, threshold 50 C.

One step = the whole hot path on that batch through the C ABI: load/pack the
resident ASCII genomes, scan both strands, Tm of every site, pair, fetch the
amplicon sequences.  `value` is Gbp scanned per primer pair per second with
the inputs already in HBM; `e2e` is the same with host (pinned) input and
output buffers, the copies inside the timed region.  Under torchrun every
rank scans its own seeded collection (weak scaling, no data-path collective);
value = all ranks' bases / max rank time.

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
# logic-pipe issue roof of a GB300: 152 SMs x 64 lane-ops/clk (LOP3 is half rate) x clock
SMS, LOP_LANES_PER_CLK = 152, 64


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
            "sample": f"first {g} of 100 genomes ({nb / 1e6:.1f} Mbp, {nc} contigs), scan+Tm+pair+fetch, "
                      f"{dt:.1f} s"}


def run_reference(args):
    rank, world, _ = dist_info()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        if rank != 0:
            dist.barrier()
            return
    w = workload(1)
    steps = []
    for i in range(args.warmup + args.steps):
        r = cpu_baseline(w, target_s=args.ref_seconds)
        if i >= args.warmup:
            steps.append(r)
    v = float(np.mean([r["value"] for r in steps]))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Gbp/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8+f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": steps[0]["sample"]},
            "cpu_baseline": {"value": v, "unit": "Gbp/s", "cores": steps[0]["cores"], "kind": "oracle",
                             "sample": steps[0]["sample"]},
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
    """DRAM bytes per launch from a committed ncu summary, if it still matches this build."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        rec = json.load(open(path)).get(kernel)
    except (OSError, ValueError):
        return None
    if not rec:
        return None
    from paper_2509_13300_gb300 import build
    if rec.get("source_digest") != build.source_digest():
        return None
    return rec


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--ref-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="keep the default (or AH_SCAN_TUNING) scan variant")
    ap.add_argument("--n-genomes", type=int, default=100, help="smaller collections for profiling runs")
    ap.add_argument("--no-pipeline", action="store_true",
                    help="one set at a time (default: the next set packs on a second stream after the current scan)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    rank, world, local = dist_info()
    import torch
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    from paper_2509_13300_gb300 import ah, build
    build.build()

    w = workload(1 + rank, args.n_genomes)
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
    alu_peak = SMS * LOP_LANES_PER_CLK * clk_mhz * 1e6 / 1e12
    if dominant == "scan":
        tr = traffic_record("ah_scan_kernel")
        roof = {"bound": "alu", "achieved": scan_tops, "peak": alu_peak, "unit": "Tops/s",
                "frac": scan_tops / alu_peak, "traffic": tr["dram_bytes_per_launch"] if tr else None,
                "kernel": "ah_scan_kernel",
                "peak_note": f"logic pipe: {SMS} SMs x {LOP_LANES_PER_CLK} LOP3 lanes/clk x {clk_mhz:.0f} MHz "
                             f"(median SM clock under load)",
                "algorithmic": f"{lop_per_word} LOP3 per 32 starts per pass over the planes",
                "hbm_achieved_gbs": scan_hbm, "hbm_peak_gbs": hbm_peak,
                "hbm_frac": scan_hbm / hbm_peak, "hbm_peak_kind": peak_kind,
                "hbm_algorithmic": "0.5 B/base (4 one-hot planes x 1 bit)"}
    else:
        tr = traffic_record("pack_kernel")
        roof = {"bound": "hbm", "achieved": pack_hbm, "peak": hbm_peak, "unit": "GB/s",
                "frac": pack_hbm / hbm_peak, "traffic": tr["dram_bytes_per_launch"] if tr else None,
                "kernel": "pack_kernel", "peak_kind": peak_kind,
                "algorithmic": "1.5 B/base (1 B ASCII read + 0.5 B planes written)"}

    # ---- end to end through the public API with host (pinned) buffers ----
    seq_h = torch.from_numpy(w.seq).pin_memory()
    out_h, bufs_h = run_out("cpu", True)

    def step_host():
        sid = ctx.ah_load_genomes(seq_h, n_bases, w.contig_off, w.contig_genome, stream)
        ctx.ah_run(sid, [pid], out_h, stream)
        ctx.ah_unload_genomes(sid)
        n, m, q = out_h.n_sites, out_h.n_amplicons, out_h.n_seq
        h2d = n_bases + w.contig_off.nbytes + w.contig_genome.nbytes
        d2h = 16 * n + 4 * n + n + 28 * m + q + 8 * (m + 1)
        return h2d, d2h

    e2e = None
    if args.e2e_steps > 0:
        step_host()
        barrier(world)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.e2e_steps):
            h2d, d2h = step_host()
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_ms = max_over_ranks(e0.elapsed_time(e1), world)
        e2e = {"value": bases_all * args.e2e_steps / (e2e_ms / 1e3) / 1e9, "unit": "Gbp/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "steps": args.e2e_steps}

    if rank != 0:
        ctx.close()
        return
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
    print(json.dumps(line), flush=True)
    ctx.close()


def ctx_scan_lop_count(pair: dict, tune: dict) -> int:
    """LOP3 instructions the generated scan kernel (the tuned variant) issues
    per word of 32 starts for this pair: counted in its generated source."""
    from paper_2509_13300_gb300 import ah
    return ah.scan_lop3_per_word(pair["fwd"], pair["rev"], int(pair["k"]), tune["R"], tune["arith_pct"])


if __name__ == "__main__":
    main()
