"""Python binding of the C ABI in include/ampliconhunter.h (ctypes).

Argument marshalling only: every step of the hot path runs in the native
library's CUDA kernels.  Arrays may be numpy arrays (host) or torch tensors
(host or CUDA); the library detects device pointers itself.  The library is
loaded on first use; if it has not been built this raises, there is no
fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

AH_OK, AH_ERR_ARG, AH_ERR_PRIMER, AH_ERR_OOM, AH_ERR_BUDGET, AH_ERR_OVERFLOW, AH_ERR_CUDA, AH_ERR_TIMEOUT, \
    AH_ERR_JIT, AH_ERR_DEVICE_CHECK = range(10)
STATUS_NAMES = {0: "AH_OK", 1: "AH_ERR_ARG", 2: "AH_ERR_PRIMER", 3: "AH_ERR_OOM", 4: "AH_ERR_BUDGET",
                5: "AH_ERR_OVERFLOW", 6: "AH_ERR_CUDA", 7: "AH_ERR_TIMEOUT", 8: "AH_ERR_JIT",
                9: "AH_ERR_DEVICE_CHECK"}
AH_LOAD_REVERSED = 1  # ah_load_genomes_ex flag: contigs packed reversed (decoy genomes)
AH_LOAD_HOST_ASYNC = 2  # load flag: host input copies queued, not waited for (keep the input unchanged)

SITE_DTYPE = np.dtype([("genome", "<u4"), ("contig", "<u4"), ("pos", "<u4"), ("primer", "u1"),
                       ("strand", "u1"), ("mm", "u1"), ("pair", "u1")])
AMPLICON_DTYPE = np.dtype([("genome", "<u4"), ("contig", "<u4"), ("start", "<u4"), ("end", "<u4"),
                           ("left", "<u4"), ("right", "<u4"), ("orient", "u1"), ("pair", "u1"),
                           ("pad0", "u1"), ("pad1", "u1")])

# Every symbol include/ampliconhunter.h declares.
EXPORTS = ["ah_create", "ah_destroy", "ah_last_error", "ah_device_bytes", "ah_load_genomes", "ah_unload_genomes",
           "ah_set_primers", "ah_set_nn_table", "ah_scan", "ah_tm", "ah_pair", "ah_fetch", "ah_set_profiling",
           "ah_get_profile", "ah_pair_noalloc", "ah_tune_scan", "ah_run", "ah_run_begin", "ah_run_end",
           "ah_load_genomes_ex", "ah_load_genomes_2bit", "ah_load_genomes_2bit_ex", "ah_tm_sweep", "ah_amplitypes",
           "ah_generate_bases", "ah_serve_start",
           "ah_serve_submit", "ah_serve_wait", "ah_serve_stop", "ah_hmm_build", "ah_hmm_tables", "ah_hmm_score",
           "ah_hmm_forward", "ah_hmm_free"]


class AHError(RuntimeError):
    """A non-zero ah_status.  For AH_ERR_OVERFLOW, `needed` is the count the
    call reported in its n_out argument."""

    def __init__(self, status: int, msg: str, needed: int | None = None):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status
        self.needed = needed


class PcrParams(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("clamp", ctypes.c_int32), ("min_len", ctypes.c_int32),
                ("max_len", ctypes.c_int32), ("tm_min", ctypes.c_double), ("dnac1_nM", ctypes.c_double),
                ("dnac2_nM", ctypes.c_double), ("Na_mM", ctypes.c_double), ("K_mM", ctypes.c_double),
                ("Tris_mM", ctypes.c_double), ("Mg_mM", ctypes.c_double), ("dNTPs_mM", ctypes.c_double),
                ("saltcorr", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class TuneResult(ctypes.Structure):
    _fields_ = [("R", ctypes.c_int32), ("arith_pct", ctypes.c_int32), ("min_blocks", ctypes.c_int32),
                ("order", ctypes.c_int32), ("stages", ctypes.c_int32), ("warps_per_cta", ctypes.c_int32),
                ("regs", ctypes.c_int32), ("reserved", ctypes.c_int32), ("us_per_tile", ctypes.c_double),
                ("tiles", ctypes.c_uint64)]


class RunOut(ctypes.Structure):
    """ah_run_out: caller-set buffers/capacities; the call fills the n_* counts."""
    _fields_ = [("sites", ctypes.c_void_p), ("sites_cap", ctypes.c_uint64), ("n_sites", ctypes.c_uint64),
                ("tm", ctypes.c_void_p), ("pass_", ctypes.c_void_p),
                ("amplicons", ctypes.c_void_p), ("amplicons_cap", ctypes.c_uint64), ("n_amplicons", ctypes.c_uint64),
                ("seq", ctypes.c_void_p), ("seq_cap", ctypes.c_uint64), ("n_seq", ctypes.c_uint64),
                ("seq_offsets", ctypes.c_void_p), ("tm_filter", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class ServeConfig(ctypes.Structure):
    _fields_ = [("mem_budget", ctypes.c_size_t), ("max_batch", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class Request(ctypes.Structure):
    _fields_ = [("genomes", ctypes.c_void_p), ("n_genomes", ctypes.c_uint32), ("pair_id", ctypes.c_uint32),
                ("k", ctypes.c_int32), ("tm_filter", ctypes.c_int32)]


class RequestInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("batch", ctypes.c_uint32), ("batch_size", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32), ("n_sites", ctypes.c_uint64), ("n_amplicons", ctypes.c_uint64),
                ("n_seq", ctypes.c_uint64), ("bases", ctypes.c_uint64), ("submit_ms", ctypes.c_double), ("start_ms", ctypes.c_double),
                ("done_ms", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


class NNTable(ctypes.Structure):
    _fields_ = [("stack_dH", ctypes.c_double * 256), ("stack_dS", ctypes.c_double * 256),
                ("term_dH", ctypes.c_double * 16), ("term_dS", ctypes.c_double * 16)]


_lib = None


def library_path() -> str:
    return _build.LIB


def lib():
    """The loaded native library (raises if it is not built)."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"native library missing: {path}; build it with "
                               "paper_2509_13300_gb300.build.build()")
        L = ctypes.CDLL(path)
        P, U32, U64, I32, S = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32, ctypes.c_size_t
        sig = {
            "ah_create": (I32, [ctypes.c_int, S, ctypes.POINTER(P)]),
            "ah_destroy": (None, [P]),
            "ah_last_error": (ctypes.c_char_p, [P]),
            "ah_device_bytes": (S, [P]),
            "ah_load_genomes": (I32, [P, P, U64, P, U32, P, ctypes.POINTER(U32), P]),
            "ah_load_genomes_ex": (I32, [P, P, U64, P, U32, P, U32, ctypes.POINTER(U32), P]),
            "ah_load_genomes_2bit": (I32, [P, P, U64, P, U64, P, U32, P, ctypes.POINTER(U32), P]),
            "ah_load_genomes_2bit_ex": (I32, [P, P, U64, P, U64, P, U32, P, U32, ctypes.POINTER(U32), P]),
            "ah_unload_genomes": (I32, [P, U32]),
            "ah_set_primers": (I32, [P, ctypes.c_char_p, ctypes.c_char_p, ctypes.POINTER(PcrParams),
                                     ctypes.POINTER(U32)]),
            "ah_set_nn_table": (I32, [P, U32, P]),
            "ah_scan": (I32, [P, U32, P, U32, P, U64, ctypes.POINTER(U64), P]),
            "ah_tm": (I32, [P, U32, P, U32, P, U64, P, P, P]),
            "ah_pair": (I32, [P, U32, P, U32, P, P, U64, P, U64, ctypes.POINTER(U64), P]),
            "ah_fetch": (I32, [P, U32, P, U64, P, U64, P, P]),
            "ah_set_profiling": (I32, [P, I32]),
            "ah_get_profile": (I32, [P, ctypes.c_char_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(U64),
                                     ctypes.POINTER(U64)]),
            "ah_run": (I32, [P, U32, P, U32, ctypes.POINTER(RunOut), P]),
            "ah_run_begin": (I32, [P, U32, P, U32, ctypes.POINTER(RunOut), P, P]),
            "ah_tm_sweep": (I32, [P, U32, P, U32, P, U64, P, U64, P, U32, P, ctypes.POINTER(U64), P]),
            "ah_amplitypes": (I32, [P, U32, P, U64, P, P, U64, ctypes.POINTER(U64), ctypes.POINTER(U64), ctypes.POINTER(U64), P]),
            "ah_generate_bases": (I32, [P, U64, P, U64, P, P, U64, U64, U64, P, P]),
            "ah_run_end": (I32, [P]),
            "ah_serve_start": (I32, [P, U32, ctypes.POINTER(ServeConfig), ctypes.POINTER(P)]),
            "ah_serve_submit": (I32, [P, ctypes.POINTER(Request), ctypes.POINTER(U64)]),
            "ah_serve_wait": (I32, [P, U64, ctypes.POINTER(RequestInfo), P, U64, P, U64, P, U64, P]),
            "ah_serve_stop": (I32, [P]),
            "ah_hmm_build": (I32, [P, P, P, U64, ctypes.POINTER(U32)]),
            "ah_hmm_tables": (I32, [P, U32, ctypes.POINTER(U64), ctypes.POINTER(U64), P, P]),
            "ah_hmm_score": (I32, [P, U32, U32, P, U64, P, P]),
            "ah_hmm_forward": (I32, [P, U32, U32, P, U64, P, P]),
            "ah_hmm_free": (I32, [P, U32]),
            "ah_tune_scan": (I32, [P, U32, P, U32, U64, ctypes.POINTER(TuneResult), P]),
            "ah_pair_noalloc": (I32, [P, U32, P, P, U64, P, U64, ctypes.POINTER(U64), P]),
            "ah_debug_compile_scan": (I32, [ctypes.c_char_p, ctypes.c_char_p, I32, I32, I32, I32, ctypes.c_char_p, S]),
            "ah_debug_hmm_profile": (I32, [P, P, U64, U64, ctypes.POINTER(U64), ctypes.POINTER(U64), P, P]),
            "ah_debug_scan_source": (I32, [ctypes.c_char_p, ctypes.c_char_p, I32, I32, I32, I32, ctypes.c_char_p, S]),
            "ah_debug_scan_stall": (I32, [P, I32]),
            "ah_debug_pipe_rates": (I32, [P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(x):
    """Raw address of a numpy array or torch tensor (None -> NULL)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return ctypes.c_void_p(x.data_ptr())
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return ctypes.c_void_p(x.ctypes.data)
    if isinstance(x, int):
        return ctypes.c_void_p(x)
    raise TypeError(f"unsupported buffer type {type(x)}")


def _stream(s):
    if s is None:
        return None
    if hasattr(s, "cuda_stream"):
        return ctypes.c_void_p(s.cuda_stream)
    return ctypes.c_void_p(int(s))


def pcr_params(d: dict) -> PcrParams:
    return PcrParams(int(d["k"]), int(d.get("clamp", 0)), int(d["min_len"]), int(d["max_len"]),
                     float(d.get("tm_min", float("-inf"))), float(d.get("dnac1_nM", 250.0)),
                     float(d.get("dnac2_nM", 25.0)), float(d.get("Na_mM", 50.0)), float(d.get("K_mM", 0.0)),
                     float(d.get("Tris_mM", 0.0)), float(d.get("Mg_mM", 0.0)), float(d.get("dNTPs_mM", 0.0)),
                     int(d.get("saltcorr", 5)), 0)


# ---------------------------------------------------------------- ABI calls
class Context:
    """One ah_ctx.  Methods carry the ABI's names and arguments."""

    def __init__(self, device: int = 0, mem_budget_bytes: int = 0):
        self._lib = lib()
        h = ctypes.c_void_p()
        st = self._lib.ah_create(device, mem_budget_bytes, ctypes.byref(h))
        if st != AH_OK:
            raise AHError(st, self._lib.ah_last_error(None).decode())
        self.h = h

    def close(self):
        for srv in list(getattr(self, "_servers", ())):
            srv.stop()
        if getattr(self, "h", None):
            self._lib.ah_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _check(self, st: int, needed: int | None = None):
        if st != AH_OK:
            raise AHError(st, self._lib.ah_last_error(self.h).decode(), needed)

    def last_error(self) -> str:
        return self._lib.ah_last_error(self.h).decode()

    def device_bytes(self) -> int:
        return int(self._lib.ah_device_bytes(self.h))

    def debug_scan_stall(self, on: bool):
        """Test aid: make later scans take their timeout path (each warp's first
        slice waits on a barrier that nothing completes; 20 us limit)."""
        self._check(self._lib.ah_debug_scan_stall(self.h, 1 if on else 0))

    def ah_set_profiling(self, enable):
        """0/False off, 1/True stage events and host sections, 2 host sections only,
        3 events on the pack and scan stages only, and host sections."""
        self._check(self._lib.ah_set_profiling(self.h, int(enable)))

    def ah_get_profile(self, stage: str | None):
        """(milliseconds, kernel launches, calls) of one stage, or totals for None."""
        ms, l, k = ctypes.c_double(), ctypes.c_uint64(), ctypes.c_uint64()
        self._check(self._lib.ah_get_profile(self.h, stage.encode() if stage else None, ctypes.byref(ms),
                                             ctypes.byref(l), ctypes.byref(k)))
        return ms.value, l.value, k.value

    def ah_load_genomes(self, seq, n_bases: int, contig_off: np.ndarray, contig_genome: np.ndarray,
                        stream=None, reversed: bool = False, host_async: bool = False) -> int:
        """reversed: pack every contig reversed (the decoy collection).  host_async:
        a host seq's copies are queued, not waited for (AH_LOAD_HOST_ASYNC): keep it
        unchanged until a synchronising call on the set has returned."""
        contig_off = np.ascontiguousarray(contig_off, dtype=np.uint64)
        contig_genome = np.ascontiguousarray(contig_genome, dtype=np.uint32)
        sid = ctypes.c_uint32()
        flags = (AH_LOAD_REVERSED if reversed else 0) | (AH_LOAD_HOST_ASYNC if host_async else 0)
        self._check(self._lib.ah_load_genomes_ex(self.h, _ptr(seq), n_bases, _ptr(contig_off), len(contig_off) - 1,
                                                 _ptr(contig_genome), flags, ctypes.byref(sid), _stream(stream)))
        return sid.value

    def ah_load_genomes_2bit(self, codes, n_bases: int, gaps: np.ndarray, contig_off: np.ndarray,
                             contig_genome: np.ndarray, stream=None, host_async: bool = False) -> int:
        """Load from 2-bit codes (encode_2bit) and the no-base runs (gaps: (n, 2) uint64);
        host_async as ah_load_genomes (the codes and gaps stay unchanged meanwhile)."""
        gaps = np.ascontiguousarray(gaps, dtype=np.uint64).reshape(-1, 2)
        contig_off = np.ascontiguousarray(contig_off, dtype=np.uint64)
        contig_genome = np.ascontiguousarray(contig_genome, dtype=np.uint32)
        sid = ctypes.c_uint32()
        self._check(self._lib.ah_load_genomes_2bit_ex(self.h, _ptr(codes), n_bases,
                                                      _ptr(gaps) if len(gaps) else None, len(gaps),
                                                      _ptr(contig_off), len(contig_off) - 1, _ptr(contig_genome),
                                                      AH_LOAD_HOST_ASYNC if host_async else 0, ctypes.byref(sid),
                                                      _stream(stream)))
        return sid.value

    def ah_unload_genomes(self, set_id: int):
        self._check(self._lib.ah_unload_genomes(self.h, set_id))

    def ah_set_primers(self, fwd: str, rev: str, params: dict) -> int:
        pid = ctypes.c_uint32()
        p = pcr_params(params)
        self._check(self._lib.ah_set_primers(self.h, fwd.encode(), rev.encode(), ctypes.byref(p), ctypes.byref(pid)))
        return pid.value

    def ah_set_nn_table(self, pair_id: int, table: NNTable | None):
        self._check(self._lib.ah_set_nn_table(self.h, pair_id, ctypes.byref(table) if table is not None else None))

    def ah_scan(self, set_id: int, pair_ids, out, cap: int, stream=None) -> int:
        ids = np.ascontiguousarray(pair_ids, dtype=np.uint32)
        n = ctypes.c_uint64()
        st = self._lib.ah_scan(self.h, set_id, _ptr(ids), len(ids), _ptr(out), cap, ctypes.byref(n), _stream(stream))
        self._check(st, n.value)
        return n.value

    def ah_run(self, set_id: int, pair_ids, out: RunOut, stream=None) -> RunOut:
        ids = np.ascontiguousarray(pair_ids, dtype=np.uint32)
        st = self._lib.ah_run(self.h, set_id, _ptr(ids), len(ids), ctypes.byref(out), _stream(stream))
        self._check(st, out.n_sites)
        return out

    def ah_run_begin(self, set_id: int, pair_ids, out: RunOut, stream=None, scan_done=None):
        """Queue a run (see ah_run_end); scan_done: a torch.cuda.Event (or raw cudaEvent_t) recorded
        after the scan.  `out` and its buffers must stay alive until ah_run_end."""
        ids = np.ascontiguousarray(pair_ids, dtype=np.uint32)
        self._pending_ids = ids  # kept alive with the queued run
        ev = None
        if scan_done is not None:
            if hasattr(scan_done, "cuda_event"):
                if not scan_done.cuda_event:  # torch creates its event on first use
                    scan_done.record()
                ev = ctypes.c_void_p(scan_done.cuda_event)
            else:
                ev = ctypes.c_void_p(int(scan_done))
        self._check(self._lib.ah_run_begin(self.h, set_id, _ptr(ids), len(ids), ctypes.byref(out), _stream(stream), ev))

    def ah_tm_sweep(self, set_id: int, pair_ids, sites, amplicons, thresholds, stream=None):
        """Per threshold: (amplicons, FF/RR amplicons, genomes amplified), and the set's genome count."""
        ids = np.ascontiguousarray(pair_ids, dtype=np.uint32)
        thr = np.ascontiguousarray(thresholds, dtype=np.float64)
        rows = np.zeros((len(thr), 3), dtype=np.uint64)
        ng = ctypes.c_uint64()
        n_s = len(sites) if isinstance(sites, np.ndarray) else sites.numel() // 16
        n_a = len(amplicons) if isinstance(amplicons, np.ndarray) else amplicons.numel() // 28
        self._check(self._lib.ah_tm_sweep(self.h, set_id, _ptr(ids), len(ids), _ptr(sites) if n_s else None, n_s,
                                          _ptr(amplicons) if n_a else None, n_a, _ptr(thr), len(thr), _ptr(rows),
                                          ctypes.byref(ng), _stream(stream)))
        return rows, ng.value

    def amplitypes(self, set_id: int, amplicons: np.ndarray, stream=None):
        """(variant id per amplicon, rows [genome, amplitype, n_amplicons, n_variants] per genome with
        amplicons, number of variants, number of amplitypes) -- size query, then the call."""
        n = len(amplicons)
        variant = np.zeros(max(n, 1), dtype=np.uint32)
        nr, nv, nt = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        st = self._lib.ah_amplitypes(self.h, set_id, _ptr(amplicons) if n else None, n, None, None, 0,
                                     ctypes.byref(nr), ctypes.byref(nv), ctypes.byref(nt), _stream(stream))
        if st not in (AH_OK, AH_ERR_OVERFLOW):
            self._check(st)
        rows = np.zeros((max(nr.value, 1), 4), dtype=np.uint32)
        self._check(self._lib.ah_amplitypes(self.h, set_id, _ptr(amplicons) if n else None, n, _ptr(variant),
                                            _ptr(rows), nr.value, ctypes.byref(nr), ctypes.byref(nv),
                                            ctypes.byref(nt), _stream(stream)))
        return variant[:n], rows[:nr.value], nv.value, nt.value

    def generate_bases(self, coll, base0: int, n: int, out, stream=None, tables=None):
        """Bases [base0, base0 + n) of a countergen collection into device memory `out` (torch uint8).
        tables: the collection's segments and patches already on the device (device_tables());
        the call is then stream-ordered, else host slices are passed and the call waits."""
        if tables is not None:
            segs, ns, pp, pb, npch = tables
            self._check(self._lib.ah_generate_bases(self.h, coll.seed, _ptr(segs), ns, _ptr(pp) if npch else None,
                                                    _ptr(pb) if npch else None, npch, base0, n, _ptr(out),
                                                    _stream(stream)))
            return
        ends = coll.segments["end"]
        s0 = int(np.searchsorted(ends, base0, side="right"))  # the segments that hold the range
        s1 = min(len(ends), int(np.searchsorted(ends, base0 + max(n, 1) - 1, side="right")) + 1)
        segs = np.ascontiguousarray(coll.segments[s0:s1])
        pp = np.ascontiguousarray(coll.patch_pos, dtype=np.uint64)
        pb = np.ascontiguousarray(coll.patch_bytes, dtype=np.uint8)
        lo, hi = np.searchsorted(pp, base0), np.searchsorted(pp, base0 + n)  # the patches in range
        pp, pb = np.ascontiguousarray(pp[lo:hi]), np.ascontiguousarray(pb[lo:hi])
        self._check(self._lib.ah_generate_bases(self.h, coll.seed, _ptr(segs), len(segs), _ptr(pp) if len(pp) else None,
                                                _ptr(pb) if len(pb) else None, len(pp), base0, n, _ptr(out),
                                                _stream(stream)))

    @staticmethod
    def device_tables(coll):
        """A collection's segments and patches as device tensors (for generate_bases)."""
        import torch
        segs = torch.from_numpy(np.ascontiguousarray(coll.segments).view(np.uint8).copy()).cuda()
        pp = torch.from_numpy(np.ascontiguousarray(coll.patch_pos, dtype=np.uint64).view(np.uint8).copy()).cuda()
        pb = torch.from_numpy(np.ascontiguousarray(coll.patch_bytes, dtype=np.uint8).copy()).cuda()
        return segs, len(coll.segments), pp, pb, len(coll.patch_pos)

    def ah_run_end(self, out: RunOut) -> RunOut:
        self._check(self._lib.ah_run_end(self.h), out.n_sites)
        return out

    def run(self, set_id: int, pair_ids, tm_filter: bool = True, caps=(0, 0, 0)) -> dict:
        """The whole path into numpy arrays (host buffers).  caps are capacity
        hints (sites, amplicons, sequence bytes); when too small the call is
        repeated with the reported counts."""
        for _ in range(2):
            sites = np.zeros(max(caps[0], 1), dtype=SITE_DTYPE)
            tm = np.zeros(max(caps[0], 1), dtype=np.float32)
            ps = np.zeros(max(caps[0], 1), dtype=np.uint8)
            amps = np.zeros(max(caps[1], 1), dtype=AMPLICON_DTYPE)
            seq = np.zeros(max(caps[2], 1), dtype=np.uint8)
            offs = np.zeros(max(caps[1], 1) + 1, dtype=np.uint64)
            o = RunOut(sites.ctypes.data, caps[0], 0, tm.ctypes.data, ps.ctypes.data, amps.ctypes.data, caps[1], 0,
                       seq.ctypes.data, caps[2], 0, offs.ctypes.data, 1 if tm_filter else 0, 0)
            ids = np.ascontiguousarray(pair_ids, dtype=np.uint32)
            st = self._lib.ah_run(self.h, set_id, _ptr(ids), len(ids), ctypes.byref(o), None)
            if st == AH_OK:
                n, m, q = o.n_sites, o.n_amplicons, o.n_seq
                return dict(sites=sites[:n], tm=tm[:n], pass_=ps[:n], amps=amps[:m], seqs=seq[:q].tobytes(),
                            offs=offs[:m + 1])
            if st != AH_ERR_OVERFLOW:
                self._check(st)
            caps = (o.n_sites, o.n_amplicons, o.n_seq)
        raise AHError(AH_ERR_OVERFLOW, "ah_run: counts changed between calls")

    def ah_tune_scan(self, set_id: int, pair_ids, sample_tiles: int = 0, stream=None) -> dict:
        ids = np.ascontiguousarray(pair_ids, dtype=np.uint32)
        r = TuneResult()
        self._check(self._lib.ah_tune_scan(self.h, set_id, _ptr(ids), len(ids), sample_tiles, ctypes.byref(r),
                                           _stream(stream)))
        return {f: getattr(r, f) for f, _ in TuneResult._fields_ if f != "reserved"}

    def ah_tm(self, set_id: int, pair_ids, sites, n: int, tm_out, pass_out=None, stream=None):
        ids = np.ascontiguousarray(pair_ids, dtype=np.uint32)
        self._check(self._lib.ah_tm(self.h, set_id, _ptr(ids), len(ids), _ptr(sites), n, _ptr(tm_out),
                                    _ptr(pass_out), _stream(stream)))

    def ah_pair(self, set_id: int, pair_ids, sites, passed, n: int, out, cap: int, stream=None) -> int:
        ids = np.ascontiguousarray(pair_ids, dtype=np.uint32)
        m = ctypes.c_uint64()
        st = self._lib.ah_pair(self.h, set_id, _ptr(ids), len(ids), _ptr(sites), _ptr(passed), n, _ptr(out), cap,
                               ctypes.byref(m), _stream(stream))
        self._check(st, m.value)
        return m.value

    def ah_fetch(self, set_id: int, amplicons, n: int, seq_out, cap: int, offsets_out, stream=None):
        self._check(self._lib.ah_fetch(self.h, set_id, _ptr(amplicons), n, _ptr(seq_out), cap, _ptr(offsets_out),
                                       _stream(stream)))

    # ------------------------------------------------ profile HMM
    def hmm_build(self, seqs) -> int:
        """Profile from training sequences (list of str or bytes) -> profile id."""
        data = b"".join(x.encode() if isinstance(x, str) else bytes(x) for x in seqs)
        off = np.zeros(len(seqs) + 1, dtype=np.uint64)
        off[1:] = np.cumsum([len(x) for x in seqs])
        buf = np.frombuffer(data, dtype=np.uint8).copy() if data else np.zeros(1, np.uint8)
        hid = ctypes.c_uint32()
        self._check(self._lib.ah_hmm_build(self.h, _ptr(buf), _ptr(off), len(seqs), ctypes.byref(hid)))
        return hid.value

    def hmm_tables(self, hmm_id: int):
        """(m, reference index, t[(m + 1), 3, 3], e[(m + 1), 4]) as float32 arrays."""
        m, ref = ctypes.c_uint64(), ctypes.c_uint64()
        self._check(self._lib.ah_hmm_tables(self.h, hmm_id, ctypes.byref(m), ctypes.byref(ref), None, None))
        t = np.zeros((m.value + 1, 3, 3), dtype=np.float32)
        e = np.zeros((m.value + 1, 4), dtype=np.float32)
        self._check(self._lib.ah_hmm_tables(self.h, hmm_id, None, None, _ptr(t), _ptr(e)))
        return m.value, ref.value, t, e

    def hmm_score(self, set_id: int, hmm_id: int, amplicons, n: int | None = None, out=None, stream=None,
                  forward: bool = False):
        """Viterbi (or, with forward=True, Forward) log-odds score (bits) of each
        amplicon; numpy float32 unless `out` is given."""
        n = len(amplicons) if n is None else n
        res = np.zeros(n, dtype=np.float32) if out is None else out
        if not isinstance(amplicons, np.ndarray) or amplicons.flags["C_CONTIGUOUS"]:
            a = amplicons
        else:
            a = np.ascontiguousarray(amplicons)
        fn = self._lib.ah_hmm_forward if forward else self._lib.ah_hmm_score
        self._check(fn(self.h, set_id, hmm_id, _ptr(a) if n else None, n, _ptr(res) if n else None,
                       _stream(stream)))
        return res

    def hmm_forward(self, set_id: int, hmm_id: int, amplicons, n: int | None = None, out=None, stream=None):
        """Forward log-odds score (bits) of each amplicon: log2 of the sum over state paths."""
        return self.hmm_score(set_id, hmm_id, amplicons, n, out, stream, forward=True)

    def hmm_free(self, hmm_id: int):
        self._check(self._lib.ah_hmm_free(self.h, hmm_id))

    # ------------------------------------------------ numpy conveniences (host buffers)
    def load(self, seq: np.ndarray, contig_off, contig_genome, stream=None, reversed: bool = False) -> int:
        n = int(contig_off[-1])
        return self.ah_load_genomes(seq, n, contig_off, contig_genome, stream, reversed)

    def scan(self, set_id: int, pair_ids) -> np.ndarray:
        """Sites as a numpy structured array (size query, then the call)."""
        try:
            n = self.ah_scan(set_id, pair_ids, None, 0)
        except AHError as e:
            if e.status != AH_ERR_OVERFLOW:
                raise
            n = e.needed
        out = np.zeros(n, dtype=SITE_DTYPE)
        if n:
            m = self.ah_scan(set_id, pair_ids, out, n)
            assert m == n
        return out

    def tm(self, set_id: int, pair_ids, sites: np.ndarray):
        tm = np.zeros(len(sites), dtype=np.float32)
        ps = np.zeros(len(sites), dtype=np.uint8)
        self.ah_tm(set_id, pair_ids, np.ascontiguousarray(sites), len(sites), tm, ps)
        return tm, ps

    def pair(self, set_id: int, pair_ids, sites: np.ndarray, passed: np.ndarray | None = None) -> np.ndarray:
        sites = np.ascontiguousarray(sites)
        ids = np.ascontiguousarray(pair_ids, dtype=np.uint32)
        m = ctypes.c_uint64()
        st = self._lib.ah_pair(self.h, set_id, _ptr(ids), len(ids), _ptr(sites), _ptr(passed), len(sites), None, 0,
                               ctypes.byref(m), None)
        if st not in (AH_OK, AH_ERR_OVERFLOW):
            self._check(st)
        out = np.zeros(m.value, dtype=AMPLICON_DTYPE)
        if m.value:
            k = self.ah_pair(set_id, pair_ids, sites, passed, len(sites), out, m.value)
            assert k == m.value
        return out

    def fetch(self, set_id: int, amplicons: np.ndarray):
        amplicons = np.ascontiguousarray(amplicons)
        offs = np.zeros(len(amplicons) + 1, dtype=np.uint64)
        st = self._lib.ah_fetch(self.h, set_id, _ptr(amplicons), len(amplicons), None, 0, _ptr(offs), None)
        if st not in (AH_OK, AH_ERR_OVERFLOW):
            self._check(st)
        total = int(offs[-1])
        out = np.zeros(max(total, 1), dtype=np.uint8)
        self.ah_fetch(set_id, amplicons, len(amplicons), out, total, offs)
        return out[:total].tobytes(), offs


class Server:
    """ah_serve_*: continuous batching of requests over one resident genome set.
    The context belongs to the server's worker thread until stop()."""

    def __init__(self, ctx: Context, set_id: int, mem_budget: int = 1 << 30, max_batch: int = 64):
        self._lib = ctx._lib
        self.ctx = ctx
        cfg = ServeConfig(int(mem_budget), int(max_batch), 0)
        h = ctypes.c_void_p()
        ctx._check(self._lib.ah_serve_start(ctx.h, set_id, ctypes.byref(cfg), ctypes.byref(h)))
        self.h = h
        ctx.__dict__.setdefault("_servers", set()).add(self)

    def submit(self, genomes, pair_id: int, k: int, tm_filter: bool = True) -> int:
        g = np.ascontiguousarray(genomes, dtype=np.uint32)
        req = Request(g.ctypes.data if len(g) else None, len(g), int(pair_id), int(k), int(bool(tm_filter)))
        t = ctypes.c_uint64()
        st = self._lib.ah_serve_submit(self.h, ctypes.byref(req), ctypes.byref(t))
        if st != AH_OK:
            raise AHError(st, "ah_serve_submit rejected the request")
        return t.value

    def wait(self, ticket: int, sequences: bool = True):
        """(sites, amplicons, sequences, offsets, info dict) of a submitted request
        (sequences and offsets are None when not asked for)."""
        info = RequestInfo()
        z = np.zeros(1, np.uint64)
        st = self._lib.ah_serve_wait(self.h, ticket, ctypes.byref(info), None, 0, None, 0, None, 0,
                                     _ptr(z) if sequences else None)
        if st == AH_OK:
            return (np.zeros(0, SITE_DTYPE), np.zeros(0, AMPLICON_DTYPE), b"" if sequences else None,
                    z if sequences else None, info.as_dict())
        if st != AH_ERR_OVERFLOW:
            raise AHError(st, f"request {ticket} failed ({STATUS_NAMES.get(info.status, info.status)})")
        sites = np.zeros(info.n_sites, SITE_DTYPE)
        amps = np.zeros(info.n_amplicons, AMPLICON_DTYPE)
        seq = np.zeros(max(info.n_seq, 1), np.uint8) if sequences else None
        offs = np.zeros(info.n_amplicons + 1, np.uint64) if sequences else None
        st = self._lib.ah_serve_wait(self.h, ticket, ctypes.byref(info), _ptr(sites), len(sites), _ptr(amps),
                                     len(amps), _ptr(seq), info.n_seq, _ptr(offs))
        if st != AH_OK:
            raise AHError(st, f"request {ticket}: results could not be read")
        return sites, amps, (seq[:info.n_seq].tobytes() if sequences else None), offs, info.as_dict()

    def stop(self):
        if getattr(self, "h", None):
            self._lib.ah_serve_stop(self.h)
            self.h = None
            self.ctx.__dict__.get("_servers", set()).discard(self)

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.stop()


def debug_hmm_profile(seqs):
    """The library's profile of training sequences, built on the host without a
    context (no GPU needed): (m, reference index, t[(m + 1), 3, 3], e[(m + 1), 4])."""
    data = b"".join(x.encode() if isinstance(x, str) else bytes(x) for x in seqs)
    off = np.zeros(len(seqs) + 1, dtype=np.uint64)
    off[1:] = np.cumsum([len(x) for x in seqs])
    buf = np.frombuffer(data, dtype=np.uint8).copy() if data else np.zeros(1, np.uint8)
    m, ref = ctypes.c_uint64(), ctypes.c_uint64()
    rc = lib().ah_debug_hmm_profile(_ptr(buf), _ptr(off), len(seqs), 0, ctypes.byref(m), ctypes.byref(ref), None, None)
    if rc:
        raise ValueError("no training sequence")
    t = np.zeros((m.value + 1, 3, 3), dtype=np.float32)
    e = np.zeros((m.value + 1, 4), dtype=np.float32)
    rc = lib().ah_debug_hmm_profile(_ptr(buf), _ptr(off), len(seqs), m.value, ctypes.byref(m), ctypes.byref(ref),
                                    _ptr(t), _ptr(e))
    assert rc == 0
    return m.value, ref.value, t, e


def encode_2bit(seq: np.ndarray):
    """ASCII bases -> (2-bit codes, no-base runs) for ah_load_genomes_2bit: base p
    in bits 2 (p % 4) of byte p / 4 (A 0, C 1, G 2, T 3, either case); every
    other letter is no base, listed as (start, length) runs (its code bits 0)."""
    seq = np.ascontiguousarray(seq, dtype=np.uint8)
    lut = np.full(256, 255, dtype=np.uint8)
    for i, ch in enumerate(b"ACGT"):
        lut[ch] = i
        lut[ch + 32] = i
    c = lut[seq]
    bad = c == 255
    c = np.where(bad, 0, c).astype(np.uint8)
    n = len(c)
    pad = np.zeros((-n) % 4, dtype=np.uint8)
    q = np.concatenate([c, pad]).reshape(-1, 4)
    codes = (q[:, 0] | (q[:, 1] << 2) | (q[:, 2] << 4) | (q[:, 3] << 6)).astype(np.uint8)
    edges = np.diff(np.concatenate([[0], bad.view(np.int8), [0]]))
    starts = np.nonzero(edges == 1)[0]
    ends = np.nonzero(edges == -1)[0]
    gaps = np.stack([starts, ends - starts], axis=1).astype(np.uint64) if len(starts) else np.zeros((0, 2), np.uint64)
    return codes, gaps


def debug_pipe_rates():
    """Measured issue rates of the current GPU: (LOP3, 32-bit integer add)
    lane-operations per clock per SM, from the SMs' own cycle counters."""
    out = (ctypes.c_double * 2)()
    rc = lib().ah_debug_pipe_rates(out)
    if rc != 0:
        raise AHError(AH_ERR_CUDA, f"pipe-rate probe failed ({rc})")
    return float(out[0]), float(out[1])


def debug_compile_scan(fwd: str, rev: str, k: int, R: int = 4, arith_pct: int = 0, order: int = 0):
    """Generate and NVRTC-compile the scan kernel of one pair (no GPU needed).
    Returns (ok, log) where the log holds the ptxas register report."""
    buf = ctypes.create_string_buffer(1 << 16)
    rc = lib().ah_debug_compile_scan(fwd.encode(), rev.encode(), k, R, arith_pct, order, buf, len(buf))
    return rc == 0, buf.value.decode(errors="replace")


def debug_scan_source(fwd: str, rev: str, k: int, R: int = 4, arith_pct: int = 0, order: int = 0) -> str:
    """The generated CUDA source of one pair's scan kernel."""
    buf = ctypes.create_string_buffer(1 << 22)
    rc = lib().ah_debug_scan_source(fwd.encode(), rev.encode(), k, R, arith_pct, order, buf, len(buf))
    if rc != 0:
        raise RuntimeError(f"scan source generation failed ({rc})")
    return buf.value.decode()


def scan_lop3_per_word(fwd: str, rev: str, k: int, R: int = 4, arith_pct: int = 0) -> int:
    """Logic-pipe (LOP3) operations the generated hot loop issues per 32-start
    word for one pair, counted in its generated source."""
    src = debug_scan_source(fwd, rev, k, R, arith_pct)
    hot = src[src.index("u32 hg[NGRP * R];"):src.index("__any_sync")]
    return round(hot.count("lop3<") / R)
