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


def test_null_arguments_are_rejected_before_any_device_call(so):
    """Every entry point checks its pointers first and answers GT_EINVAL (1)
    to a missing context, grammar, server, result or output pointer."""
    lib = ctypes.CDLL(str(so))
    P = ctypes.c_void_p
    null = P()
    calls = {
        "gt_create": (null, 0, ctypes.c_size_t(0)),
        "gt_destroy": (null,),
        "gt_sync": (null, null),
        "gt_load_grammar": (null, null, null, null),
        "gt_free_grammar": (null,),
        "gt_grammar_info_get": (null, null),
        "gt_rule_weights": (null, null, null),
        "gt_word_count": (null, null, null),
        "gt_word_count_noalloc": (null, null, null),
        "gt_word_count_batch": (null, null, 1, null),
        "gt_head_tail": (null, null, null, null),
        "gt_sort": (null, 0, null, null),
        "gt_term_vector": (null, 0, null, null),
        "gt_inverted_index": (null, null, null),
        "gt_sequence_count": (null, 0, null, null),
        "gt_ranked_index": (null, 1, null, null),
        "gt_tfidf": (null, null, null),
        "gt_cooccurrence": (null, null, null),
        "gt_run_batch": (null, null, 0, null, null),
        "gt_plan_create": (null, null, 1, null, null),
        "gt_plan_launch": (null, null),
        "gt_plan_result": (null, 0, null, null, null),
        "gt_plan_destroy": (null,),
        "gt_result_view": (null, null, null, null),
        "gt_free_result": (null,),
        "gt_profile_enable": (null, 1),
        "gt_profile_reset": (null,),
        "gt_profile_read": (null, null, null, null, null),
        "gt_set_param": (null, null, ctypes.c_int64(0)),
        "gt_autotune": (null, ctypes.c_uint32(1), 3, null, null),
        "gt_server_create": (null, 4, ctypes.c_size_t(0), null),
        "gt_submit": (null, null, 1, null),
        "gt_poll": (null, ctypes.c_uint64(0), 0, null, null),
        "gt_server_stats": (null, null, null, null, null),
        "gt_server_destroy": (null,),
        "gt_check_bounded_wait": (null, 0, 100, null),
    }
    for name, args in calls.items():
        f = getattr(lib, name)
        f.restype = ctypes.c_int
        assert f(*args) == 1, name
    lib.gt_last_error.restype = ctypes.c_char_p
    lib.gt_last_error.argtypes = [P]
    assert lib.gt_last_error(null) == b"null context"
    lib.gt_kernel_launches.restype = ctypes.c_int64
    assert lib.gt_kernel_launches() == 0


def test_every_entry_point_is_covered_by_the_null_argument_test():
    # entry points that take no pointer to check, or return a value, not a status
    exempt = {"gt_last_error", "gt_kernel_launches"}
    src = Path(__file__).read_text()
    block = src[src.index("calls = {"):src.index("for name, args in calls.items()")]
    covered = set(re.findall(r'"(gt_[a-z_0-9]+)"', block))
    assert set(declared()) - exempt - covered == set()


def test_binding_loads_the_library_and_types_every_entry_point(so):
    from paper_2106_06889_gb300 import binding
    L = binding.lib()
    for name in declared():
        f = getattr(L, name)
        if name not in ("gt_last_error", "gt_kernel_launches"):
            assert f.argtypes is not None and f.restype is ctypes.c_int, name
