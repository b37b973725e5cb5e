"""The multi-process path of bench.py on CPU: two gloo ranks under torchrun
(127.0.0.1).  Ranks scan their own seeded collections (weak scaling, no
data-path collective); the only collectives are the barrier and the max / sum
of timings and bases, and the reference arm runs on rank 0 alone."""
import json
import os
import socket
import subprocess
import sys
import textwrap

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _torchrun(args, timeout=240):
    env = dict(os.environ, OMP_NUM_THREADS="1")
    for attempt in range(2):  # a second port if the first was taken between probe and bind
        cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
               "--master-addr=127.0.0.1", f"--master-port={_free_port()}"] + args
        r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=timeout, env=env)
        if r.returncode == 0:
            break
    assert r.returncode == 0, r.stderr[-3000:]
    return [json.loads(l) for l in r.stdout.splitlines() if l.startswith("{")]


def test_timing_reductions_over_two_gloo_ranks(tmp_path):
    script = tmp_path / "ranks.py"
    script.write_text(textwrap.dedent(f"""
        import json, sys
        sys.path.insert(0, {ROOT!r})
        import torch.distributed as dist
        import bench
        dist.init_process_group("gloo")
        rank, world, _ = bench.dist_info()
        mx = bench.max_over_ranks(1.0 + rank, world)
        sm = bench.sum_over_ranks(10.0 * (rank + 1), world)
        bench.barrier(world)
        with open({str(tmp_path)!r} + f"/rank{{rank}}.json", "w") as f:  # one file per rank: no interleaving
            json.dump({{"rank": rank, "world": world, "max": mx, "sum": sm}}, f)
        dist.destroy_process_group()
    """))
    _torchrun([str(script)])
    out = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    assert [d["rank"] for d in out] == [0, 1]
    assert all(d["world"] == 2 and d["max"] == 2.0 and d["sum"] == 30.0 for d in out)


def test_ranks_scan_their_own_collections():
    import bench
    a, b = bench.workload(1, 2), bench.workload(2, 2)  # collection workload: seed 1 + rank
    assert a.n_bases != b.n_bases or not np.array_equal(a.seq[:1000], b.seq[:1000])
    c, d = bench.large_collection(7, 3), bench.large_collection(8, 3)  # large workload: seed 7 + rank
    assert c.n_bases != d.n_bases or not np.array_equal(c.bases(0, 1000), d.bases(0, 1000))


def test_reference_arm_runs_on_rank_zero_alone():
    out = _torchrun(["bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0",
                     "--n-genomes", "2", "--ref-seconds", "0.2"])
    assert len(out) == 1
    line = out[0]
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0
