"""The C-ABI library loads without a GPU and exports every entry point declared in include/ah.h,
and the Python binding covers each of them (no compute calls: this runs on CPU)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "ah.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[\w\s\*]*?\b(ah_\w+)\s*\(", text, flags=re.M)
    return sorted(set(n for n in names if not n.endswith("_t")))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2511_00170_gb300 import ah

    return ah.load()


def test_header_declares_the_path():
    d = _declared()
    for name in ["ah_pack_batch", "ah_scan_primers", "ah_pair_amplicons", "ah_tm_filter", "ah_extract_barcodes"]:
        assert name in d


def test_library_exports_every_declared_symbol(lib):
    path = os.path.join(ROOT, "paper_2511_00170_gb300", "libah.so")
    syms = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (ah_\w+)$", syms, flags=re.M))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    for n in _declared():
        assert hasattr(lib, n)


def test_binding_covers_the_header(lib):
    from paper_2511_00170_gb300 import ah

    assert set(_declared()) <= set(ah.SIGNATURES)
    for n in _declared():
        assert callable(getattr(ah, n))


def test_library_does_not_need_a_driver_at_load(lib):
    # the driver is reached through the CUDA runtime at run time only
    out = subprocess.run(["ldd", os.path.join(ROOT, "paper_2511_00170_gb300", "libah.so")], capture_output=True,
                         text=True).stdout
    assert "libcuda.so" not in out


def test_no_gpu_context_creation_fails_cleanly(lib):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2511_00170_gb300 import ah

    with pytest.raises(ah.AhError):
        ah.ah_ctx_create(0)
