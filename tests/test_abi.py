"""The C-ABI library builds for sm_103a, loads, and exports every entry point
include/gtadoc.h declares (no GPU needed: no compute call is made)."""
import ctypes
import re
from pathlib import Path

import pytest

from paper_2106_06889_gb300 import _build

HEADER = Path(__file__).resolve().parent.parent / "include" / "gtadoc.h"


def declared():
    text = HEADER.read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gt_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def so():
    return _build.build_gtadoc()


def test_header_declares_entry_points():
    names = declared()
    for must in ("gt_create", "gt_load_grammar", "gt_word_count", "gt_sort", "gt_result_view"):
        assert must in names


def test_library_exports_every_declared_symbol(so):
    lib = ctypes.CDLL(str(so))
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_no_internal_symbols_leak(so):
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", str(so)], capture_output=True, text=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    gt = {n for n in exported if n.startswith("gt_")}
    assert gt == set(declared())


def test_create_without_gpu_fails_loudly(so):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    lib = ctypes.CDLL(str(so))
    h = ctypes.c_void_p()
    rc = lib.gt_create(ctypes.byref(h), 0, ctypes.c_size_t(0))
    assert rc != 0 and not h.value
