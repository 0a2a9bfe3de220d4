"""Thin Python binding of ``libgtadoc.so`` (the ``gt_*`` C ABI of include/gtadoc.h).

Functions carry the C names and only marshal arguments: host arrays become
pointers, torch CUDA tensors become device pointers, a torch stream becomes a
``cudaStream_t``.  Every computation happens in the library's CUDA kernels.
If the library is missing or no GB300 is present the calls raise; nothing
falls back to a CPU path.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from ._build import GTADOC_SO

GT_OK = 0
_CODES = {1: "GT_EINVAL", 2: "GT_ENOMEM", 3: "GT_ECUDA", 4: "GT_ETIMEOUT", 5: "GT_ETABLE_FULL",
          6: "GT_EOVERFLOW", 7: "GT_EBUSY", 8: "GT_ENOTFOUND"}


class GtError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_CODES.get(code, code)}: {msg}")
        self.code = code


class gt_grammar_desc(ctypes.Structure):
    _fields_ = [("num_words", ctypes.c_int32), ("num_rules", ctypes.c_int32), ("num_files", ctypes.c_int32),
                ("rule_off", ctypes.c_void_p), ("sym", ctypes.c_void_p), ("file_off", ctypes.c_void_p),
                ("on_device", ctypes.c_int32)]


class gt_tune_result(ctypes.Structure):
    _fields_ = [("wc_aggregate", ctypes.c_int32), ("wc_slices", ctypes.c_int32), ("file_strategy", ctypes.c_int32),
                ("candidates", ctypes.c_int32), ("wc_ms", ctypes.c_double), ("file_ms", ctypes.c_double)]


class gt_query(ctypes.Structure):
    _fields_ = [("grammar", ctypes.c_void_p), ("kind", ctypes.c_int32), ("param", ctypes.c_int32),
                ("d_counts", ctypes.c_void_p)]


GT_Q_WORD_COUNT, GT_Q_SORT, GT_Q_INVERTED_INDEX, GT_Q_TERM_VECTOR = 0, 1, 2, 3
GT_Q_SEQUENCE_COUNT, GT_Q_RANKED_INDEX, GT_Q_TFIDF, GT_Q_COOCCURRENCE = 4, 5, 6, 7


class gt_grammar_info(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("num_words", "num_rules", "num_files", "num_syms", "num_edges",
                                              "num_root_edges", "depth", "num_tokens", "owned_windows",
                                              "device_bytes", "root_words", "file_pairs", "file_words")]


_lib = None
_P = ctypes.c_void_p


def lib() -> ctypes.CDLL:
    """Load the in-tree CUDA library (built by ``__graft_entry__.build()``)."""
    global _lib
    if _lib is None:
        if not GTADOC_SO.exists():
            raise RuntimeError(f"{GTADOC_SO} is not built; run __graft_entry__.build() (needs nvcc)")
        L = ctypes.CDLL(str(GTADOC_SO))
        sig = {
            "gt_create": [ctypes.POINTER(_P), ctypes.c_int, ctypes.c_size_t],
            "gt_destroy": [_P],
            "gt_sync": [_P, _P],
            "gt_load_grammar": [_P, ctypes.POINTER(gt_grammar_desc), _P, ctypes.POINTER(_P)],
            "gt_free_grammar": [_P],
            "gt_grammar_info_get": [_P, ctypes.POINTER(gt_grammar_info)],
            "gt_rule_weights": [_P, _P, _P],
            "gt_word_count": [_P, _P, _P],
            "gt_word_count_noalloc": [_P, _P, _P],
            "gt_word_count_batch": [_P, _P, ctypes.c_int, _P],
            "gt_sort": [_P, ctypes.c_int, _P, ctypes.POINTER(_P)],
            "gt_inverted_index": [_P, _P, ctypes.POINTER(_P)],
            "gt_term_vector": [_P, ctypes.c_int, _P, ctypes.POINTER(_P)],
            "gt_sequence_count": [_P, ctypes.c_int, _P, ctypes.POINTER(_P)],
            "gt_ranked_index": [_P, ctypes.c_int, _P, ctypes.POINTER(_P)],
            "gt_tfidf": [_P, _P, ctypes.POINTER(_P)],
            "gt_cooccurrence": [_P, _P, ctypes.POINTER(_P)],
            "gt_head_tail": [_P, _P, _P, _P],
            "gt_result_view": [_P, ctypes.c_char_p, ctypes.POINTER(_P), ctypes.POINTER(ctypes.c_int64)],
            "gt_free_result": [_P],
            "gt_profile_enable": [_P, ctypes.c_int],
            "gt_set_param": [_P, ctypes.c_char_p, ctypes.c_int64],
            "gt_autotune": [_P, ctypes.c_uint32, ctypes.c_int, _P, _P],
            "gt_run_batch": [_P, _P, ctypes.c_int, _P, _P],
            "gt_plan_create": [_P, _P, ctypes.c_int, _P, ctypes.POINTER(_P)],
            "gt_plan_launch": [_P, _P],
            "gt_plan_result": [_P, ctypes.c_int, ctypes.c_char_p, ctypes.POINTER(_P), ctypes.POINTER(ctypes.c_int64)],
            "gt_plan_destroy": [_P],
            "gt_server_create": [_P, ctypes.c_int, ctypes.c_size_t, ctypes.POINTER(_P)],
            "gt_submit": [_P, _P, ctypes.c_int, ctypes.POINTER(ctypes.c_uint64)],
            "gt_poll": [_P, ctypes.c_uint64, ctypes.c_int, _P, ctypes.POINTER(ctypes.c_int64)],
            "gt_server_stats": [_P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_uint64)],
            "gt_server_destroy": [_P],
            "gt_check_bounded_wait": [_P, ctypes.c_int, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)],
            "gt_profile_reset": [_P],
            "gt_profile_read": [_P, ctypes.c_char_p, ctypes.POINTER(ctypes.c_double),
                                ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)],
        }
        for name, args in sig.items():
            f = getattr(L, name, None)
            if f is None:
                raise RuntimeError(f"{GTADOC_SO} does not export {name}; rebuild it with __graft_entry__.build()")
            f.argtypes = args
            f.restype = ctypes.c_int
        L.gt_kernel_launches.argtypes = []
        L.gt_kernel_launches.restype = ctypes.c_int64
        L.gt_last_error.argtypes = [_P]
        L.gt_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _check(rc: int, ctx=None):
    if rc != GT_OK:
        msg = lib().gt_last_error(ctx).decode() if ctx else ""
        raise GtError(rc, msg)


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _dptr(t) -> ctypes.c_void_p:
    """Device pointer of a contiguous torch CUDA tensor."""
    if not (t.is_cuda and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


@dataclass
class Context:
    handle: ctypes.c_void_p
    device: int


@dataclass
class GrammarHandle:
    handle: ctypes.c_void_p
    ctx: Context
    num_words: int
    num_rules: int
    num_files: int


@dataclass
class ResultHandle:
    handle: ctypes.c_void_p
    ctx: Context


# ---- context ----------------------------------------------------------------

def gt_create(device: int = 0, pool_bytes: int = 0) -> Context:
    h = _P()
    _check(lib().gt_create(ctypes.byref(h), device, pool_bytes))
    return Context(h, device)


def gt_destroy(ctx: Context) -> None:
    _check(lib().gt_destroy(ctx.handle))


def gt_sync(ctx: Context, stream=None) -> None:
    _check(lib().gt_sync(ctx.handle, _stream(stream)), ctx.handle)


# ---- grammar ------------------------------------------------------------------

def gt_load_grammar(ctx: Context, grammar, stream=None) -> GrammarHandle:
    """Load a grammar (host numpy arrays, or torch CUDA tensors).

    ``grammar`` needs ``num_words``, ``rule_off`` (int64), ``sym`` (int32) and
    ``file_off`` (int64).
    """
    ro, sy, fo = grammar.rule_off, grammar.sym, grammar.file_off
    on_device = hasattr(sy, "is_cuda") and sy.is_cuda
    if on_device:
        ptrs = [_dptr(ro), _dptr(sy), _dptr(fo)]
        nr, nf = ro.shape[0] - 1, fo.shape[0] - 1
        keep = (ro, sy, fo)
    else:
        ro = np.ascontiguousarray(ro, dtype=np.int64)
        sy = np.ascontiguousarray(sy, dtype=np.int32)
        fo = np.ascontiguousarray(fo, dtype=np.int64)
        ptrs = [ctypes.c_void_p(a.ctypes.data) for a in (ro, sy, fo)]
        nr, nf = ro.shape[0] - 1, fo.shape[0] - 1
        keep = (ro, sy, fo)
    desc = gt_grammar_desc(int(grammar.num_words), int(nr), int(nf), ptrs[0], ptrs[1], ptrs[2], int(on_device))
    h = _P()
    _check(lib().gt_load_grammar(ctx.handle, ctypes.byref(desc), _stream(stream), ctypes.byref(h)), ctx.handle)
    del keep
    return GrammarHandle(h, ctx, int(grammar.num_words), int(nr), int(nf))


def gt_free_grammar(g: GrammarHandle) -> None:
    _check(lib().gt_free_grammar(g.handle))


def gt_grammar_info_get(g: GrammarHandle) -> dict:
    info = gt_grammar_info()
    _check(lib().gt_grammar_info_get(g.handle, ctypes.byref(info)))
    return {n: int(getattr(info, n)) for n, _ in gt_grammar_info._fields_}


# ---- analytics ----------------------------------------------------------------

def gt_rule_weights(g: GrammarHandle, d_weights, stream=None) -> None:
    _check(lib().gt_rule_weights(g.handle, _dptr(d_weights), _stream(stream)), g.ctx.handle)


def gt_word_count(g: GrammarHandle, d_counts, stream=None) -> None:
    _check(lib().gt_word_count(g.handle, _dptr(d_counts), _stream(stream)), g.ctx.handle)


def gt_word_count_batch(gs, d_counts, stream=None) -> None:
    """Word counts of several grammars (one context) in one fused launch sequence."""
    n = len(gs)
    if n == 0 or n != len(d_counts):
        raise ValueError("need one output buffer per grammar")
    hs = (ctypes.c_void_p * n)(*[g.handle.value for g in gs])
    ps = (ctypes.c_void_p * n)(*[_dptr(t).value for t in d_counts])
    _check(lib().gt_word_count_batch(ctypes.cast(hs, ctypes.c_void_p), ctypes.cast(ps, ctypes.c_void_p), n,
                                     _stream(stream)), gs[0].ctx.handle)


def gt_word_count_noalloc(g: GrammarHandle, d_counts, stream=None) -> None:
    _check(lib().gt_word_count_noalloc(g.handle, _dptr(d_counts), _stream(stream)), g.ctx.handle)


def gt_head_tail(g: GrammarHandle, d_head, d_tail, stream=None) -> None:
    _check(lib().gt_head_tail(g.handle, _dptr(d_head), _dptr(d_tail), _stream(stream)), g.ctx.handle)


def _result_call(fn, g: GrammarHandle, *args, stream=None) -> ResultHandle:
    h = _P()
    _check(fn(g.handle, *args, _stream(stream), ctypes.byref(h)), g.ctx.handle)
    return ResultHandle(h, g.ctx)


def gt_sort(g: GrammarHandle, order: int = 0, stream=None) -> ResultHandle:
    return _result_call(lib().gt_sort, g, order, stream=stream)


def gt_inverted_index(g: GrammarHandle, stream=None) -> ResultHandle:
    return _result_call(lib().gt_inverted_index, g, stream=stream)


def gt_term_vector(g: GrammarHandle, top_k: int = 0, stream=None) -> ResultHandle:
    return _result_call(lib().gt_term_vector, g, top_k, stream=stream)


def gt_sequence_count(g: GrammarHandle, per_file: int = 0, stream=None) -> ResultHandle:
    return _result_call(lib().gt_sequence_count, g, per_file, stream=stream)


def gt_ranked_index(g: GrammarHandle, n: int = 3, stream=None) -> ResultHandle:
    return _result_call(lib().gt_ranked_index, g, n, stream=stream)


def gt_tfidf(g: GrammarHandle, stream=None) -> ResultHandle:
    return _result_call(lib().gt_tfidf, g, stream=stream)


def gt_cooccurrence(g: GrammarHandle, stream=None) -> ResultHandle:
    return _result_call(lib().gt_cooccurrence, g, stream=stream)


# ---- results ------------------------------------------------------------------

_TYPESTR = {"word": "<i4", "file": "<i4", "count": "<u8", "key": "<u8", "offsets": "<i8", "tfidf": "<f8"}


class _DeviceArray:
    """Zero-copy view of a library-owned device buffer for torch.as_tensor."""

    def __init__(self, ptr: int, n: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False),
                                         "version": 3, "strides": None}


def gt_result_view(r: ResultHandle, field: str):
    """(device pointer, length) of one result field."""
    p = _P()
    n = ctypes.c_int64()
    _check(lib().gt_result_view(r.handle, field.encode(), ctypes.byref(p), ctypes.byref(n)), r.ctx.handle)
    return int(p.value or 0), int(n.value)


def result_tensor(r: ResultHandle, field: str):
    """A torch CUDA tensor viewing one result field (valid until gt_free_result)."""
    import torch
    ptr, n = gt_result_view(r, field)
    ts = _TYPESTR[field]
    if ts == "<u8":
        ts = "<i8"  # counts and keys are < 2^63; torch's int64 views them losslessly
    if n == 0 or ptr == 0:
        empty = {"<i4": torch.int32, "<f8": torch.float64}.get(ts, torch.int64)
        return torch.empty(0, dtype=empty, device="cuda")
    return torch.as_tensor(_DeviceArray(ptr, n, ts), device="cuda")


def result_numpy(r: ResultHandle, field: str) -> np.ndarray:
    t = result_tensor(r, field).cpu().numpy()
    return t.astype(np.uint64) if _TYPESTR[field] == "<u8" else t


def gt_free_result(r: ResultHandle) -> None:
    _check(lib().gt_free_result(r.handle))


# ---- profiling ------------------------------------------------------------------

def gt_profile_enable(ctx: Context, on: bool = True) -> None:
    _check(lib().gt_profile_enable(ctx.handle, int(on)))


def gt_profile_reset(ctx: Context) -> None:
    _check(lib().gt_profile_reset(ctx.handle))


def gt_profile_read(ctx: Context, phase: str):
    """(total device ms, timed spans, kernels launched) of one phase."""
    ms, sp, la = ctypes.c_double(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib().gt_profile_read(ctx.handle, phase.encode(), ctypes.byref(ms), ctypes.byref(sp), ctypes.byref(la)),
           ctx.handle)
    return float(ms.value), int(sp.value), int(la.value)


def gt_kernel_launches() -> int:
    return int(lib().gt_kernel_launches())


def gt_check_bounded_wait(ctx: Context, publish: bool, polls: int) -> int:
    """The bounded look-back wait on one warp: the prefix it obtained (7) when
    its predecessor publishes; GtError(GT_ETIMEOUT) when it never does."""
    p = ctypes.c_int64()
    _check(lib().gt_check_bounded_wait(ctx.handle, int(publish), polls, ctypes.byref(p)), ctx.handle)
    return int(p.value)


def gt_set_param(ctx: Context, name: str, value: int) -> None:
    _check(lib().gt_set_param(ctx.handle, name.encode(), int(value)), ctx.handle)


def gt_autotune(g: GrammarHandle, kinds, reps: int = 3, stream=None) -> dict:
    """kinds: iterable of GT_Q_* kinds (empty clears the grammar's choices)."""
    mask = 0
    for k in kinds:
        mask |= 1 << int(k)
    res = gt_tune_result()
    _check(lib().gt_autotune(g.handle, mask, int(reps), _stream(stream), ctypes.byref(res)), g.ctx.handle)
    return {n: getattr(res, n) for n, _ in gt_tune_result._fields_}


def _query_array(queries):
    n = len(queries)
    arr = (gt_query * max(n, 1))()
    for i, (gh, kind, param, counts) in enumerate(queries):
        arr[i].grammar = gh.handle.value if isinstance(gh.handle, ctypes.c_void_p) else gh.handle
        arr[i].kind = int(kind)
        arr[i].param = int(param)
        arr[i].d_counts = _dptr(counts).value if counts is not None else None
    return arr


def gt_run_batch(ctx: Context, queries, stream=None):
    """queries: list of (GrammarHandle, kind, param, counts_tensor_or_None).
    Returns a list with a ResultHandle (or None for word counts) per query."""
    n = len(queries)
    arr = _query_array(queries)
    outs = (ctypes.c_void_p * max(n, 1))()
    _check(lib().gt_run_batch(ctx.handle, ctypes.cast(arr, ctypes.c_void_p), n, _stream(stream),
                              ctypes.cast(outs, ctypes.c_void_p)), ctx.handle)
    return [ResultHandle(ctypes.c_void_p(outs[i]), ctx) if outs[i] else None for i in range(n)]


# ---- plans: a batch captured once as a CUDA graph ---------------------------------

@dataclass
class Plan:
    handle: ctypes.c_void_p
    ctx: Context
    keep: object  # the query array and its tensors stay referenced while the plan exists


def gt_plan_create(ctx: Context, queries, stream=None) -> Plan:
    arr = _query_array(queries)
    h = _P()
    _check(lib().gt_plan_create(ctx.handle, ctypes.cast(arr, ctypes.c_void_p), len(queries), _stream(stream),
                                ctypes.byref(h)), ctx.handle)
    return Plan(h, ctx, (arr, [q[3] for q in queries]))


def gt_plan_launch(p: Plan, stream=None) -> None:
    _check(lib().gt_plan_launch(p.handle, _stream(stream)), p.ctx.handle)


def plan_result_numpy(p: Plan, i: int, field: str) -> np.ndarray:
    """Field of query i's result from the plan's last launch, copied to host."""
    import torch
    ptr, n = _P(), ctypes.c_int64()
    _check(lib().gt_plan_result(p.handle, i, field.encode(), ctypes.byref(ptr), ctypes.byref(n)), p.ctx.handle)
    ts = _TYPESTR[field]
    if n.value == 0:
        return np.zeros(0, dtype=np.dtype(ts))
    t = torch.as_tensor(_DeviceArray(int(ptr.value), int(n.value), "<i8" if ts == "<u8" else ts), device="cuda")
    a = t.cpu().numpy()
    return a.astype(np.uint64) if ts == "<u8" else a


def gt_plan_destroy(p: Plan) -> None:
    _check(lib().gt_plan_destroy(p.handle))


# ---- serving --------------------------------------------------------------------

@dataclass
class Server:
    handle: ctypes.c_void_p
    ctx: Context


def gt_server_create(ctx: Context, slots: int = 4, mem_budget: int = 0) -> Server:
    h = _P()
    _check(lib().gt_server_create(ctx.handle, slots, mem_budget, ctypes.byref(h)), ctx.handle)
    return Server(h, ctx)


def gt_submit(sv: Server, queries) -> int:
    """queries: list of (GrammarHandle, kind, param, counts_tensor_or_None)."""
    arr = _query_array(queries)
    t = ctypes.c_uint64()
    _check(lib().gt_submit(sv.handle, ctypes.cast(arr, ctypes.c_void_p), len(queries), ctypes.byref(t)),
           sv.ctx.handle)
    return int(t.value)


def gt_poll(sv: Server, ticket: int, nq: int, wait: bool = True):
    """(results or None while running, latency in ns)."""
    outs = (ctypes.c_void_p * max(nq, 1))()
    lat = ctypes.c_int64()
    rc = lib().gt_poll(sv.handle, ticket, int(wait), ctypes.cast(outs, ctypes.c_void_p), ctypes.byref(lat))
    if rc == 7 and not wait:  # GT_EBUSY: still running
        return None, None
    _check(rc, sv.ctx.handle)
    return [ResultHandle(ctypes.c_void_p(outs[i]), sv.ctx) if outs[i] else None for i in range(nq)], int(lat.value)


def gt_server_stats(sv: Server) -> dict:
    a, b, c, d = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_uint64()
    _check(lib().gt_server_stats(sv.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d)))
    return {"waiting": a.value, "inflight": b.value, "max_inflight": c.value, "mem_in_use": d.value}


def gt_server_destroy(sv: Server) -> None:
    _check(lib().gt_server_destroy(sv.handle))
