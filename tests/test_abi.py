"""Host-side checks of the C ABI library (no GPU needed).

The library loads on a machine without a GPU; these tests make no compute
call.  They check the exported symbols against include/ampliconhunter.h, the
record layouts, and that the scan-kernel generator produces code that NVRTC
compiles for sm_103a across primer lengths, codes and mismatch limits.
"""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2509_13300_gb300 import ah, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return ah.lib()


def header_symbols():
    src = open(os.path.join(ROOT, "include", "ampliconhunter.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)  # drop comments
    return sorted(set(re.findall(r"\b(ah_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_binding_exports():
    assert header_symbols() == sorted(ah.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in header_symbols():
        assert hasattr(lib, name), name


def test_record_layouts_match_header():
    # ah_site 16 bytes, ah_amplicon 28 bytes, ah_pcr_params and ah_nn_table as declared
    assert ah.SITE_DTYPE.itemsize == 16
    assert ah.AMPLICON_DTYPE.itemsize == 28
    assert ctypes.sizeof(ah.PcrParams) == 4 * 4 + 8 * 8 + 4 * 2
    assert ctypes.sizeof(ah.NNTable) == 8 * (256 * 2 + 16 * 2)


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    st = lib.ah_create(0, 0, ctypes.byref(h))
    assert st == ah.AH_ERR_ARG and not h.value
    assert b"device" in lib.ah_last_error(None)


@pytest.mark.parametrize("k", [0, 1, 2, 3, 4, 5, 7, 8, 10, 25])
def test_generated_scan_kernel_compiles(lib, k):
    ok, log = ah.debug_compile_scan("AGRRTTYGATYHTDGYTYAG", "YCNTTCCYTYDYRGTACT", k, 4, 30)
    assert ok, log
    assert "0 bytes spill stores" in log


@pytest.mark.parametrize("fwd,rev", [("ACGTN", "NNNNN"), ("A" * 32, "T" * 32), ("BDHVNRYSWKM", "acgtnrysw")])
def test_generated_scan_kernel_compiles_for_code_mixes(lib, fwd, rev):
    for R in (4, 8):
        ok, log = ah.debug_compile_scan(fwd, rev, 2, R, 0, 1)
        assert ok, log
