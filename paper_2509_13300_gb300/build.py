"""Build the native library libampliconhunter.so in-tree (sm_103a only).

    python -m paper_2509_13300_gb300.build

compiles every csrc/*.cu translation unit in parallel with nvcc
(-gencode arch=compute_103a,code=sm_103a) and links them into
paper_2509_13300_gb300/_build/libampliconhunter.so.  The scan kernel itself
is generated and compiled at run time (NVRTC, sm_103a) for each primer set.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libampliconhunter.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA_HOME, "bin", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CFLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
                 "-I" + INCLUDE, "-I" + CSRC]


def _headers_mtime() -> float:
    hs = glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(INCLUDE, "*.h"))
    return max(os.path.getmtime(h) for h in hs)


def _compile(src: str, obj: str, extra: list[str]) -> str:
    cmd = [NVCC] + CFLAGS + extra + ["-c", src, "-o", obj + ".tmp"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")
    os.replace(obj + ".tmp", obj)
    return r.stderr


def source_digest() -> str:
    """Hash of the library sources (kernels, generator, headers): identifies a build."""
    import hashlib
    h = hashlib.sha256()
    for f in sorted(glob.glob(os.path.join(CSRC, "*")) + glob.glob(os.path.join(INCLUDE, "*.h"))):
        h.update(os.path.basename(f).encode())
        h.update(open(f, "rb").read())
    return h.hexdigest()[:16]


# the source files that define each profiled kernel (with the internal header)
KERNEL_SOURCES = {"ah_scan_kernel": ["scan_jit.cu"], "pack_kernel": ["pack.cu"], "tm_kernel": ["tm.cu"],
                  "tm_fast_kernel": ["tm.cu"],
                  "rank_sort_decode_kernel": ["sites.cu"], "hmm_score_kernel": ["hmm.cu"]}


def kernel_digest(kernel: str) -> str | None:
    """Hash of one kernel's sources: a profile of the kernel stays valid while it matches."""
    import hashlib
    files = KERNEL_SOURCES.get(kernel)
    if not files:
        return None
    h = hashlib.sha256()
    for f in files + ["ah_internal.h"]:
        h.update(f.encode())
        h.update(open(os.path.join(CSRC, f), "rb").read())
    return h.hexdigest()[:16]


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None) -> str:
    """Compile what changed and link the library; returns its path."""
    extra = extra or []
    os.makedirs(OUT, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    hdr = _headers_mtime()
    jobs = []
    objs = []
    for s in srcs:
        o = os.path.join(OUT, os.path.basename(s)[:-3] + ".o")
        objs.append(o)
        if force or not os.path.exists(o) or os.path.getmtime(o) < max(os.path.getmtime(s), hdr):
            jobs.append((s, o))
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            for (s, _), log in zip(jobs, ex.map(lambda j: _compile(j[0], j[1], extra), jobs)):
                if verbose and log.strip():
                    print(f"[{os.path.basename(s)}]\n{log}", file=sys.stderr)
    if jobs or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(o) for o in objs):
        cmd = [NVCC] + ARCH + ["-shared", "-o", LIB + ".tmp"] + objs + [
            "-lnvrtc", "-Xlinker", "-rpath," + os.path.join(CUDA_HOME, "lib64"),
            "-L" + os.path.join(CUDA_HOME, "lib64")]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
