#!/usr/bin/env python3
"""Benchmark: uncompressed tokens/s analysed on a grammar-compressed corpus.

One step = one pass of the workload's analytics over the resident compressed
corpus (weights, traversal, reduction, canonical output), through the gt_* C
ABI.  Default workload (the headline): 64 files, ~50M tokens, Zipf(s=1.0)
over 500k words, 5% repeated passages, one shared Sequitur grammar; word
count + inverted index + term vector in one batch.  The 500M-token one-file
corpus with nested repeats (3-word sequence count + sort) is measured the
same way and reported under ``extras``.

Prints ONE JSON line (rank 0).  ``--impl reference`` times the CPU oracle on
the host cores instead (the reference arm).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "multi64_50m": {"analytics": ["word_count", "inverted_index", "term_vector"],
                    "desc": "64 files, log-uniform 10k-2M tokens (~50M), Zipf s=1.0, V=500k, 5% repeated "
                            "passages, one Sequitur grammar"},
    "nested_500m": {"analytics": ["sequence_count", "sort"],
                    "desc": "one file of 500M tokens, Zipf s=1.05, V=1M, nested repeats (passages of passages, "
                            "depth 6) on 50% of the tokens, one Sequitur grammar (16 shards)"},
}
METRIC = "uncompressed tokens/s analysed (word count, 3-gram count); p50/p99 query ms"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    def __init__(self, device: int):
        self.proc = None
        try:
            import torch
            index = "GPU-" + str(torch.cuda.get_device_properties(device).uuid)
        except Exception:
            index = str(device)
        self.path = os.path.join(tempfile.gettempdir(), f"gtadoc_clocks_{os.getpid()}.csv")
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
        try:
            os.remove(self.path)
        except OSError:
            pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# Algorithmic bytes (the bytes the method must move; intermediates excluded)
# ---------------------------------------------------------------------------

def step_bytes(workload: str, info: dict, out: dict) -> int:
    """Bytes one step of the workload must move, by the per-unit figures of
    the hot-path measurement plan:
      word count:  4 B per body symbol + 8 B per DAG edge + 8 B per rule
                   weight + 8 B per word count;
      per file:    + 8 B per (file, rule) weight + 12 B per term-vector pair
                   + 4 B per inverted-index posting (one traversal serves
                   the term vector, the inverted index and the word count);
      3-gram:      4 B per body symbol + 8 B per rule weight + 16 B per rule
                   of head/tail words + 32 B per owned window (one table
                   update) + 16 B per distinct 3-gram;
      sort:        the word count's bytes + 12 B per distinct word."""
    G, E, R, V = info["num_syms"], info["num_edges"], info["num_rules"], info["num_words"]
    wc = 4 * G + 8 * E + 8 * R + 8 * V
    if workload == "multi64_50m":
        return wc + 8 * info["file_pairs"] + 12 * out["tv_pairs"] + 4 * out["ii_postings"]
    seq = 4 * G + 8 * R + 16 * R + 32 * info["owned_windows"] + 16 * out["distinct_3grams"]
    return seq + wc + 12 * out["distinct_words"]


def kernel_bytes(workload: str, info: dict, out: dict) -> dict:
    """Per timed single-kernel phase: (kernel, bytes of the method's own input
    or output that kernel moves).  chunk_sort_kernel<0>: the root symbols it
    reads (4 B each); tv_hist_kernel: the term-vector pairs it writes (12 B
    each); chunk_sort_kernel<1>: the per-file rule weights (4 B per (file,
    rule) pair) and the rule bodies (4 B per rule symbol) it reads;
    wc_partition_kernel and sg_scatter_kernel: the symbol stream (4 B per body
    symbol).  On the 3-gram workload the rows of owned windows
    (8 B key + 4 B weight) stand in for the per-window table updates of the
    paper's sequence support (Section IV-D): radix_downsweep_kernel<4> and sg_scatter_kernel read and write
    every row once per launch (24 B), sg_reduce_kernel reads them (12 B) and
    writes the distinct 3-grams (16 B each)."""
    G, V = info["num_syms"], info["num_words"]
    root_len = out["root_len"]
    if workload == "multi64_50m":
        return {"chunk_sort_root": ("chunk_sort_kernel<0>", 4 * root_len),
                "tv_hist_kernel": ("tv_hist_kernel", 12 * out["tv_pairs"]),
                "chunk_sort_rules": ("chunk_sort_kernel<1>", 4 * info["file_pairs"] + 4 * (G - root_len)),
                "wc_partition": ("wc_partition_kernel", 4 * G)}
    U = info["owned_windows"]
    return {"radix_pass": ("radix_downsweep_kernel<4>", 24 * U),
            "seq_scatter": ("sg_scatter_kernel", 24 * U),
            "seq_reduce": ("sg_reduce_kernel", 12 * U + 16 * out["distinct_3grams"]),
            "wc_partition": ("wc_partition_kernel", 4 * G)}


PHASES = ("weights", "wc_partition", "wc_hist", "sort_canon", "file_weights", "tv_hist",
          "chunk_sort_root", "chunk_sort_rules", "tv_hist_kernel", "tv_out", "ii_out", "wc_from_files",
          "seq_headtail", "seq_emit", "seq_sort", "radix_pass", "seq_part", "seq_scatter", "seq_fine", "seq_reduce",
          "tv_out", "cooc_rows", "rows_sort")
LOAD_PHASES = ("load_upload", "load_dag", "load_file_layout")


def dist_env():
    """(rank, world size, local rank) of this process under torchrun; one
    process per GPU, 1 process when run directly."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(x: float, world: int, device="cuda") -> float:
    """The largest value of x over all ranks (the job's time is its slowest
    rank's); x itself when there is one rank."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, tokens_per_rank: int, steps: int, seconds: float) -> float:
    """Whole-job tokens/s: every rank analyses its own copy (weak scaling)."""
    return world * tokens_per_rank * steps / seconds


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def step_queries(B, gh, analytics, counts):
    """The workload's analytics as one batch (one traversal per grammar).
    Sort is by word ID (order 0); the sequence count is global."""
    kind = {"word_count": B.GT_Q_WORD_COUNT, "sort": B.GT_Q_SORT, "inverted_index": B.GT_Q_INVERTED_INDEX,
            "term_vector": B.GT_Q_TERM_VECTOR, "sequence_count": B.GT_Q_SEQUENCE_COUNT}
    return [(gh, kind[a], 0, counts if a == "word_count" else None) for a in analytics]


def run_step(B, ctx, qs, stream, keep):
    """Enqueue one step; result handles go to ``keep`` and are released
    after the timed region (freeing waits for the GPU)."""
    keep.extend(r for r in B.gt_run_batch(ctx, qs, stream) if r is not None)


def step_outputs(B, analytics, results) -> dict:
    """Sizes of one step's results (for the algorithmic bytes)."""
    out = {"tv_pairs": 0, "ii_postings": 0, "distinct_3grams": 0, "distinct_words": 0}
    it = iter(results)
    for a in analytics:
        if a == "word_count":
            continue
        r = next(it)
        if a == "term_vector":
            out["tv_pairs"] = B.gt_result_view(r, "word")[1]
        elif a == "inverted_index":
            out["ii_postings"] = B.gt_result_view(r, "file")[1]
        elif a == "sequence_count":
            out["distinct_3grams"] = B.gt_result_view(r, "key")[1]
        elif a == "sort":
            out["distinct_words"] = B.gt_result_view(r, "word")[1]
    return out


def load_timed(B, ctx, g, stream, reps=2):
    """Load the grammar ``reps`` times (the first includes one-time costs),
    keep the last; its wall time from pinned host arrays and its phases
    (upload, DAG build, per-file layout)."""
    import torch
    pinned = {k: torch.from_numpy(np.ascontiguousarray(getattr(g, k))).pin_memory()
              for k in ("rule_off", "sym", "file_off")}

    class HostG:
        num_words = g.num_words
        rule_off = pinned["rule_off"].numpy()
        sym = pinned["sym"].numpy()
        file_off = pinned["file_off"].numpy()

    gh = None
    for _ in range(reps):
        if gh is not None:
            B.gt_free_grammar(gh)
        B.gt_profile_reset(ctx)
        B.gt_profile_enable(ctx, True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        gh = B.gt_load_grammar(ctx, HostG, stream)
        stream.synchronize()
        ms = 1e3 * (time.perf_counter() - t0)
        B.gt_profile_enable(ctx, False)
    ph = {p: B.gt_profile_read(ctx, p)[0] for p in LOAD_PHASES}
    B.gt_profile_reset(ctx)
    load = {"ms": ms, "upload_ms": ph["load_upload"], "dag_ms": ph["load_dag"],
            "file_layout_ms": ph["load_file_layout"],
            "note": "gt_load_grammar from pinned host arrays (timed separately from the step, as the paper "
                    "splits initialisation from traversal); file_layout_ms is the top-down per-file layout "
                    "(<= 64 files) that per-file queries reuse: DAG facts, no counts"}
    return gh, load, pinned, HostG


def measure(B, ctx, workload, g, steps, warmup, world, stream, autotune=True, e2e_steps=3, clocks=True,
            eager=False):
    """Device-timed steps of one workload on a resident grammar, with its
    step-level and dominant-kernel rooflines, phases, load time and the
    end-to-end figure through the public API from host buffers."""
    import torch
    analytics = WORKLOADS[workload]["analytics"]
    gh, load, pinned, HostG = load_timed(B, ctx, g, stream)
    info = B.gt_grammar_info_get(gh)
    N = info["num_tokens"]
    counts = torch.empty(g.num_words, dtype=torch.int64, device="cuda")
    tune = None
    if autotune:
        kinds = [k for a, k in (("word_count", B.GT_Q_WORD_COUNT), ("sort", B.GT_Q_SORT),
                                ("inverted_index", B.GT_Q_INVERTED_INDEX), ("term_vector", B.GT_Q_TERM_VECTOR))
                 if a in analytics]
        tune = B.gt_autotune(gh, kinds, reps=3, stream=stream) if kinds else None
    qs = step_queries(B, gh, analytics, counts)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    keep = []
    with torch.cuda.stream(stream):
        for _ in range(max(warmup, 3)):
            run_step(B, ctx, qs, stream, keep)
        torch.cuda.synchronize()
        outs = step_outputs(B, analytics, keep[-(len(keep) // max(warmup, 3)):])
        for r in keep:
            B.gt_free_result(r)
        keep.clear()
        # ---- the timed step: the batch captured once as a CUDA graph
        # (gt_plan_create) and replayed, one graph launch per step; every
        # launch recomputes every result from the grammar ----
        # (eager: the timed loop launches kernel by kernel instead, for
        # profilers that replay single kernels)
        plan = None if eager else B.gt_plan_create(ctx, qs, stream)

        def step():
            if plan is None:
                run_step(B, ctx, qs, stream, keep)
            else:
                B.gt_plan_launch(plan, stream)

        for _ in range(max(warmup, 3)):
            step()
        torch.cuda.synchronize()
        launches0 = B.gt_kernel_launches()
        barrier()
        torch.cuda.synchronize()
        sampler = ClockSampler(torch.cuda.current_device()) if clocks else None
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("timed_steps")  # lets a profiler select the timed launches
        ev0.record(stream)
        for _ in range(steps):
            step()
        ev1.record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        barrier()
        clk = sampler.stop() if sampler else None
        launches = B.gt_kernel_launches() - launches0
        if plan is not None:
            B.gt_plan_destroy(plan)
        for r in keep:
            B.gt_free_result(r)
        keep.clear()
        # ---- the same step launched kernel by kernel (gt_run_batch) ----
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = B.gt_kernel_launches()
        barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            run_step(B, ctx, qs, stream, keep)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        eager_launches = B.gt_kernel_launches() - l0
        for r in keep:
            B.gt_free_result(r)
        keep.clear()
        # phase timers: a separate pass with CUDA events around every phase
        # (kept out of the timed region; graphs are not replayed while profiling)
        B.gt_profile_reset(ctx)
        B.gt_profile_enable(ctx, True)
        for _ in range(max(3, min(steps, 5))):
            run_step(B, ctx, qs, stream, keep)
        torch.cuda.synchronize()
        B.gt_profile_enable(ctx, False)
        for r in keep:
            B.gt_free_result(r)
        keep.clear()
    ms = max_over_ranks(ev0.elapsed_time(ev1), world)
    ms_step = ms / steps
    ems = max_over_ranks(e0.elapsed_time(e1), world) / steps
    eager_step = {"ms_per_step": ems, "value": job_throughput(world, N, 1, ems / 1e3), "unit": "tokens/s",
                  "kernels_per_step": eager_launches // steps,
                  "note": "gt_run_batch per step: the same kernels launched one by one from the host"}
    phases = {}
    for ph in PHASES:
        tot, spans, la = B.gt_profile_read(ctx, ph)
        if spans:
            phases[ph] = {"ms_per_launch": tot / spans, "spans": spans, "launches": la}
    B.gt_profile_reset(ctx)
    hbm, src = peaks()
    outs["root_len"] = int(g.rule_off[1])
    sb = step_bytes(workload, info, outs)
    kb = kernel_bytes(workload, info, outs)
    # dominant kernel: the single-kernel phase with the largest time per step
    cands = [(phases[p]["ms_per_launch"] * phases[p]["launches"] / phases[p]["spans"], p)
             for p in kb if p in phases and phases[p]["launches"] == phases[p]["spans"]]
    dom = max(cands)[1] if cands else None
    kernel = None
    if dom:
        kname, kbytes = kb[dom]
        kms = phases[dom]["ms_per_launch"]
        kernel = {"kernel": kname, "ms_per_launch": kms, "algorithmic_bytes_per_launch": kbytes,
                  "achieved": kbytes / (kms / 1e3) / 1e9, "frac": kbytes / (kms / 1e3) / 1e9 / hbm,
                  "bytes": "the method's own input or output this kernel moves (intermediates excluded)"}
    achieved = sb / (ms_step / 1e3) / 1e9
    roofline = {"bound": "hbm", "scope": "whole step (every kernel of the step)", "achieved": achieved,
                "peak": hbm, "peak_source": src, "unit": "GB/s", "frac": achieved / hbm, "traffic": None,
                "algorithmic_bytes_per_step": sb, "dominant_kernel": kernel}

    # ---- end to end through the public API with host buffers ----
    e2e = None
    if e2e_steps:
        out_host = torch.empty(g.num_words, dtype=torch.int64).pin_memory()
        h2d = sum(int(v.numel() * v.element_size()) for v in pinned.values())
        host_res = {}  # pinned host buffers for the result fields, sized by the untimed first step

        def e2e_step(sizing):
            """Load from the pinned host arrays, run the step's analytics, copy
            every result back into pinned host memory; returns the bytes read back."""
            nbytes = 0
            gh2 = B.gt_load_grammar(ctx, HostG, stream)
            q2 = step_queries(B, gh2, analytics, counts)
            res = [r for r in B.gt_run_batch(ctx, q2, stream) if r is not None]
            if "word_count" in analytics:
                out_host.copy_(counts, non_blocking=True)
                nbytes += out_host.numel() * out_host.element_size()
            for i, r in enumerate(res):  # every result field back to host memory
                for fld in ("offsets", "word", "key", "count", "file"):
                    try:
                        t = B.result_tensor(r, fld)
                    except B.GtError:
                        continue
                    buf = host_res.get((i, fld))
                    if buf is None or buf.numel() < t.numel():
                        assert sizing, "result sizes change between steps"
                        buf = torch.empty(max(t.numel(), 1), dtype=t.dtype).pin_memory()
                        host_res[(i, fld)] = buf
                    buf[:t.numel()].copy_(t, non_blocking=True)
                    nbytes += t.numel() * t.element_size()
            stream.synchronize()
            for r in res:
                B.gt_free_result(r)
            B.gt_free_grammar(gh2)
            return nbytes

        with torch.cuda.stream(stream):
            e2e_step(True)  # untimed: sizes the pinned result buffers
            torch.cuda.synchronize()
            d2h_res = 0
            t0 = time.perf_counter()
            for _ in range(e2e_steps):
                d2h_res += e2e_step(False)
            e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, world)
        e2e = {"value": job_throughput(world, N, 1, e2e_s), "unit": "tokens/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h_res // e2e_steps, "ms_per_step": 1e3 * e2e_s,
               "note": "gt_load_grammar from pinned host arrays + the step's analytics + every result copied back "
                       "into pinned host memory (one untimed step first sizes those buffers)"}
    B.gt_free_grammar(gh)
    return {"value": job_throughput(world, N, steps, ms / 1e3), "ms_per_step": ms_step, "tokens": N,
            "info": info, "outputs": outs, "roofline": roofline, "phases": phases, "load": load, "e2e": e2e,
            "gpu_launches": launches, "clocks": clk, "autotune": tune, "eager_step": eager_step}


# ---------------------------------------------------------------------------
# Serving: continuous batching against the plain path, same arrivals
# ---------------------------------------------------------------------------

SERVING = {"corpora": 48, "tokens": (1_000_000, 64_000_000), "queries": 10_000, "slots": 8,
           "mem_budget": 12 << 30}


def serving_bench(B, ctx, cfg=SERVING, seed=7):
    """Resident corpora; mix 40% word count / 30% inverted index / 30% 3-gram
    count, corpus chosen uniformly.  Plain = one query at a time on one
    stream, each waited for; served = the continuous-batching server (slots,
    admission by estimated memory footprint under a budget).  Both see the
    same Poisson arrivals at 50/80/95% of the server's saturated rate, and
    each latency is from arrival to completion."""
    import torch
    from paper_2106_06889_gb300.corpus import load_serving_set
    gs = load_serving_set(cfg["corpora"], cfg["tokens"])
    hs = [B.gt_load_grammar(ctx, g) for g in gs]
    ntok = [int(B.gt_grammar_info_get(h)["num_tokens"]) for h in hs]
    nq = cfg["queries"]
    rng = np.random.default_rng(seed)
    kinds = rng.choice([B.GT_Q_WORD_COUNT, B.GT_Q_INVERTED_INDEX, B.GT_Q_SEQUENCE_COUNT], size=nq,
                       p=[0.4, 0.3, 0.3])
    which = rng.integers(0, len(gs), size=nq)
    bufs = [torch.empty(g.num_words, dtype=torch.int64, device="cuda") for g in gs]

    def q(i):
        k = int(kinds[i])
        return [(hs[which[i]], k, 0, bufs[which[i]] if k == B.GT_Q_WORD_COUNT else None)]

    tokens = sum(ntok[which[i]] for i in range(nq))
    st = torch.cuda.Stream()

    def plain(arrivals):
        """One query at a time; a query arriving while another runs waits."""
        lats, t_start = np.zeros(nq), time.perf_counter()
        for i in range(nq):
            if arrivals is not None:
                delay = t_start + arrivals[i] - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
            out = B.gt_run_batch(ctx, q(i), st)
            st.synchronize()
            done = time.perf_counter()
            lats[i] = 1e3 * (done - (t_start + arrivals[i] if arrivals is not None else done))
            for r in out:
                if r is not None:
                    B.gt_free_result(r)
        return time.perf_counter() - t_start, lats

    sv = B.gt_server_create(ctx, slots=cfg["slots"], mem_budget=cfg["mem_budget"])

    def served(arrivals):
        """Submissions follow the arrivals; a client thread collects each
        request as it completes and frees its results (results nobody has
        collected stay allocated: they are outside the server's budget)."""
        import threading
        tickets, lats, late, failed = [0] * nq, np.zeros(nq), np.zeros(nq), []
        submitted = threading.Semaphore(0)

        def collect():
            try:
                for i in range(nq):
                    submitted.acquire()
                    if tickets[i] == 0:  # the submitting thread stopped
                        return
                    out, lat = B.gt_poll(sv, tickets[i], 1, wait=True)
                    lats[i] = lat / 1e6 + late[i]
                    for r in out:
                        if r is not None:
                            B.gt_free_result(r)
            except BaseException as e:  # re-raised by the submitting thread
                failed.append(e)

        th = threading.Thread(target=collect)
        t_start = time.perf_counter()
        th.start()
        try:
            for i in range(nq):
                if failed:
                    break
                if arrivals is not None:
                    delay = t_start + arrivals[i] - time.perf_counter()
                    if delay > 0:
                        time.sleep(delay)
                    # latency counts from the arrival, also when submission lags it
                    late[i] = max(0.0, 1e3 * (time.perf_counter() - (t_start + arrivals[i])))
                tickets[i] = B.gt_submit(sv, q(i))
                submitted.release()
        finally:
            submitted.release()  # wakes the collector if a submission was missing
            th.join()
        if failed:
            raise failed[0]
        return time.perf_counter() - t_start, lats

    for i in range(min(50, nq)):  # warm-up (graphs, pools)
        for r in B.gt_run_batch(ctx, q(i), st):
            if r is not None:
                B.gt_free_result(r)
    st.synchronize()
    t_plain, _ = plain(None)
    served(None)  # warm-up
    t_sat, _ = served(None)
    cap_qps = nq / t_sat
    rates = []
    for frac in (0.5, 0.8, 0.95):
        lam = frac * cap_qps
        arr = np.cumsum(rng.exponential(1.0 / lam, size=nq))
        row = {"load": frac, "offered_qps": lam}
        for name, fn in (("served", served), ("plain", plain)):
            t, lats = fn(arr)
            row[name] = {"achieved_qps": nq / t, "p50_ms": float(np.percentile(lats, 50)),
                         "p99_ms": float(np.percentile(lats, 99))}
        rates.append(row)
    stats = B.gt_server_stats(sv)
    B.gt_server_destroy(sv)
    # word counts of every resident corpus: fused launch sequences (64 grammars
    # each at most) against one call per corpus (both device-timed on one stream)
    fused = {}
    with torch.cuda.stream(st):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for mode in ("per_corpus", "fused", "per_corpus", "fused"):  # second round is timed
            ev0.record(st)
            for _ in range(10):
                if mode == "fused":
                    B.gt_word_count_batch(hs, bufs, st)
                else:
                    for h, b in zip(hs, bufs):
                        B.gt_word_count(h, b, st)
            ev1.record(st)
            st.synchronize()
            fused[mode] = ev0.elapsed_time(ev1) / 10
    for h in hs:
        B.gt_free_grammar(h)
    return {"corpora": len(gs), "corpus_tokens_total": int(sum(ntok)), "tokens_range": list(cfg["tokens"]),
            "queries_per_rate": nq, "slots": cfg["slots"], "mem_budget_bytes": cfg["mem_budget"],
            "mix": "40% word count / 30% inverted index / 30% 3-gram count, corpus uniform",
            "saturated": {"plain_qps": nq / t_plain, "plain_tokens_per_s": tokens / t_plain,
                          "served_qps": cap_qps, "served_tokens_per_s": tokens / t_sat,
                          "max_inflight": stats["max_inflight"]},
            "poisson": rates, "word_count_all_corpora_ms": fused}


def small_word_count(B, ctx, reps=200):
    """Word count on the 200k-token single-file corpus, where launch latency
    dominates: per-query time with the launch sequence replayed from a CUDA
    graph against launched kernel by kernel."""
    import torch
    from paper_2106_06889_gb300.corpus import load_config
    g, _ = load_config("wc_single_200k")
    gh = B.gt_load_grammar(ctx, g)
    out = torch.empty(g.num_words, dtype=torch.int64, device="cuda")
    st = torch.cuda.Stream()
    res = {}
    for use in (1, 0):
        B.gt_set_param(ctx, "use_graphs", use)
        with torch.cuda.stream(st):
            for _ in range(5):
                B.gt_word_count(gh, out, st)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            for _ in range(reps):
                B.gt_word_count(gh, out, st)
            b.record(st)
            torch.cuda.synchronize()
        res["graph_us" if use else "direct_us"] = 1e3 * a.elapsed_time(b) / reps
    B.gt_set_param(ctx, "use_graphs", 1)
    B.gt_free_grammar(gh)
    res["tokens"] = 200_000
    return res


def many_files(B, ctx, reps=3):
    """100k small files in one grammar: ranked inverted index over words and
    over 3-word keys, and term vector + inverted index, all by the bottom-up
    per-file strategy.  Device time per query, results freed outside the
    timed region."""
    import torch
    from paper_2106_06889_gb300.corpus import load_config
    g, _ = load_config("files100k")
    gh = B.gt_load_grammar(ctx, g)
    info = B.gt_grammar_info_get(gh)
    N = info["num_tokens"]
    st = torch.cuda.Stream()
    out = {"tokens": N, "files": info["num_files"], "grammar_symbols": info["num_syms"]}
    cases = {"ranked_index_words": lambda: [B.gt_ranked_index(gh, 1, st)],
             "ranked_index_3grams": lambda: [B.gt_ranked_index(gh, 3, st)],
             "term_vector_inverted_index": lambda: B.gt_run_batch(
                 ctx, [(gh, B.GT_Q_TERM_VECTOR, 0, None), (gh, B.GT_Q_INVERTED_INDEX, 0, None)], st)}
    with torch.cuda.stream(st):
        for name, fn in cases.items():
            for r in fn():  # warm-up
                B.gt_free_result(r)
            ts = []
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
                res = fn()
                e1.record(st)
                st.synchronize()
                ts.append(e0.elapsed_time(e1))
                for r in res:
                    B.gt_free_result(r)
            ms = float(np.median(ts))
            out[name] = {"ms_per_query": ms, "tokens_per_s": N / (ms / 1e3)}
    B.gt_free_grammar(gh)
    return out


def sequence_paths(B, ctx, g, stream, reps=3):
    """The global 3-word count by the one-row-per-window LSD radix sort (the
    default, with scatter tiles of 2048 and of 4096 keys) and by the
    sample-sort buckets, on the same grammar."""
    import torch
    gh = B.gt_load_grammar(ctx, g, stream)
    out = {}
    with torch.cuda.stream(stream):
        for name, path, items, pf in (("bucketed", 2, 8, 0), ("radix_sort_tile4096", 1, 16, 0),
                                      ("radix_sort_prefetch", 1, 8, 1), ("radix_sort", 1, 8, 0)):
            B.gt_set_param(ctx, "seq_path", path)
            B.gt_set_param(ctx, "radix_items", items)
            B.gt_set_param(ctx, "radix_prefetch", pf)
            B.gt_free_result(B.gt_sequence_count(gh, 0, stream))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            keep = []
            e0.record(stream)
            for _ in range(reps):
                keep.append(B.gt_sequence_count(gh, 0, stream))
            e1.record(stream)
            torch.cuda.synchronize()
            for r in keep:
                B.gt_free_result(r)
            out[name + "_ms"] = e0.elapsed_time(e1) / reps
    B.gt_set_param(ctx, "seq_path", 1)
    B.gt_free_grammar(gh)
    return out


def uncompressed_baseline(B, ctx, workload, stream, steps=5):
    """The workload's step on the uncompressed token stream: the same corpus
    as a root-only grammar (no rules), run by the same kernels - the GPU
    uncompressed-analytics baseline the paper compares G-TADOC with (it
    reports 2x on average).  Device time per step, inputs resident."""
    from paper_2106_06889_gb300.corpus import load_config, root_only_grammar
    _, c = load_config(workload, keep_tokens=True)
    g = root_only_grammar(c.tokens, c.file_lens, c.num_words)
    del c
    m = measure(B, ctx, workload, g, steps, 3, 1, stream, autotune=False, e2e_steps=0, clocks=False)
    return {"value": m["value"], "unit": "tokens/s", "ms_per_step": m["ms_per_step"],
            "grammar_symbols": m["info"]["num_syms"], "load_ms": m["load"]["ms"],
            "note": "the corpus as a root-only grammar: every token is a root symbol, no rules"}


# ---------------------------------------------------------------------------
# CPU baseline: the oracle (test infrastructure) on the host cores
# ---------------------------------------------------------------------------

ORACLE_CALLS = {  # the oracle's form of each analytic of a step
    "word_count": lambda orc, g: orc.word_count(g),
    "inverted_index": lambda orc, g: orc.inverted_index(g),
    "term_vector": lambda orc, g: orc.term_vector(g, 0),
    "sequence_count": lambda orc, g: orc.sequence_count(g, 0),
    "sort": lambda orc, g: orc.sort_words(g, 0),
}


def sample_grammar(g, k):
    """The first k files, or for a one-file corpus its first k root symbols."""
    from paper_2106_06889_gb300.corpus import prefix_files, root_prefix
    return prefix_files(g, k) if g.num_files > 1 else root_prefix(g, k)


def oracle_sample(g, analytics, budget_s: float = 20.0):
    """Time the CPU oracle, one core, running a step's analytics on a bounded
    sample of the workload (a prefix of its files, or of its one file's root
    symbols), grown geometrically until one run takes >= budget/4 seconds.
    Returns (tokens/s, sample description, tokens, seconds)."""
    import oracle
    many = g.num_files > 1
    k, limit = (1, g.num_files) if many else (1 << 16, int(g.file_off[1]))
    while True:
        sub = sample_grammar(g, k)
        t0 = time.perf_counter()
        for a in analytics:
            ORACLE_CALLS[a](oracle, sub)
        dt = time.perf_counter() - t0
        if dt > budget_s / 4 or k >= limit:
            break
        k = min(limit, k * 2)
    ntok = int(oracle.word_count(sub).astype(np.int64).sum())
    what = (f"the first {k} of {g.num_files} files" if many
            else f"the first {k} of {int(g.file_off[1])} root symbols of its one file")
    return ntok / dt, what, ntok, dt


_POOL_G = None


def _pool_init(g):
    global _POOL_G
    _POOL_G = g


def _pool_ping(_):
    return os.getpid()


def _pool_part(args):
    """One worker's share of the file-split oracle: its files' analytics."""
    a, b, analytics = args
    import oracle
    from paper_2106_06889_gb300.corpus import file_range
    sub = file_range(_POOL_G, a, b)
    files = oracle.expand_files(sub)
    out = {}
    if "word_count" in analytics:
        out["word_count"] = oracle.word_count_text(files, sub.num_words)
    if "term_vector" in analytics:
        out["term_vector"] = oracle.term_vector_text(files)
    if "inverted_index" in analytics:
        out["inverted_index"] = oracle.inverted_index_text(files, sub.num_words)
    return a, out


def oracle_file_split(g, analytics, workers: int):
    """The oracle split by file over `workers` processes (the coarse-grained,
    file-level parallelism of the CPU baseline the paper compares against),
    partial results merged in the parent.  Every file of the workload; the
    pool is started (spawn) before the timed region.  Returns (tokens/s,
    workers used, seconds) or None if the workload has one file."""
    import multiprocessing as mp
    F = g.num_files
    if F < 2 or not set(analytics) <= {"word_count", "term_vector", "inverted_index"}:
        return None
    workers = max(1, min(workers, F))
    size = np.diff(np.asarray(g.file_off, np.int64))
    ends = np.cumsum(size)
    cuts = [0] + sorted(set(int(np.searchsorted(ends, ends[-1] * k / workers)) + 1
                            for k in range(1, workers))) + [F]
    ranges = [(a, b) for a, b in zip(cuts, cuts[1:]) if b > a]
    with mp.get_context("spawn").Pool(len(ranges), initializer=_pool_init, initargs=(g,)) as pool:
        pool.map(_pool_ping, range(len(ranges)))
        t0 = time.perf_counter()
        parts = pool.map(_pool_part, [(a, b, analytics) for a, b in ranges])
        merged = merge_file_split(parts, analytics, g.num_words)
        dt = time.perf_counter() - t0
    ntok = int(merged["word_count"].sum()) if "word_count" in merged else int(merged["term_vector"][2].sum())
    return ntok / dt, len(ranges), dt, ntok


def merge_file_split(parts, analytics, V):
    """Whole-corpus results from per-file-range parts ((first file, results)):
    word counts summed, term vectors concatenated in file order, inverted
    index postings regrouped by word with files ascending."""
    parts = sorted(parts, key=lambda p: p[0])
    merged = {}
    if "word_count" in analytics:
        merged["word_count"] = np.sum([p["word_count"] for _, p in parts], axis=0)
    if "term_vector" in analytics:
        offs, ws, cs, base = [np.zeros(1, np.int64)], [], [], 0
        for _, p in parts:
            o, w, c = p["term_vector"]
            offs.append(o[1:] + base)
            base += int(o[-1])
            ws.append(w)
            cs.append(c)
        merged["term_vector"] = (np.concatenate(offs), np.concatenate(ws), np.concatenate(cs))
    if "inverted_index" in analytics:
        wl, fl = [], []
        for a, p in parts:
            o, f = p["inverted_index"]
            wl.append(np.repeat(np.arange(V, dtype=np.int64), np.diff(o)))
            fl.append(f.astype(np.int64) + a)
        w, f = np.concatenate(wl), np.concatenate(fl)
        order = np.argsort(w, kind="stable")  # files of each word stay ascending
        merged["inverted_index"] = (np.concatenate([[0], np.cumsum(np.bincount(w, minlength=V))]),
                                    f[order].astype(np.int32))
    return merged


def cpu_baselines(g, analytics, budget_s=20.0):
    rate, what, ntok, dt = oracle_sample(g, analytics, budget_s)
    nproc = os.cpu_count() or 1
    cpu = {"value": rate, "unit": "tokens/s", "cores": 1, "kind": "oracle", "nproc": nproc,
           "sample": f"{' + '.join(analytics)} on {what} ({ntok} tokens), {dt:.1f} s"}
    par = oracle_file_split(g, analytics, nproc)
    if par:
        cpu["file_split"] = {"value": par[0], "unit": "tokens/s", "cores": par[1], "kind": "oracle split by file",
                             "sample": f"every file ({par[3]} tokens), {par[2]:.1f} s, partial results merged"}
    else:
        cpu["file_split"] = {"value": None, "note": "one file: nothing to split by file"}
    return cpu


# ---------------------------------------------------------------------------
# main
# ---------------------------------------------------------------------------

def workload_config(args, g) -> dict:
    """The line's config: what the workload is (both arms print the same)."""
    wl = WORKLOADS[args.workload]
    return {"workload": args.workload, "analytics": wl["analytics"], "desc": wl["desc"], "scale": args.scale,
            "l2": f"inputs larger than L2 (symbol array {4 * len(g.sym) / 1e6:.0f} MB > 129 MB)"}


def reference_arm(args, rank):
    """The oracle as it stands, one core, a bounded sample of the workload per
    step (rank 0 only)."""
    from paper_2106_06889_gb300.corpus import load_config
    if rank != 0:
        return
    wl = WORKLOADS[args.workload]
    g, _ = load_config(args.workload, scale=args.scale)
    runs = []
    for i in range(args.warmup + args.steps):
        r = oracle_sample(g, wl["analytics"], budget_s=4.0)
        if i >= args.warmup:
            runs.append(r)
    v = statistics.median(r[0] for r in runs)
    s = runs[0]
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "tokens/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * s[3],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic", "config": workload_config(args, g),
            "cpu_baseline": {"value": v, "unit": "tokens/s", "cores": 1, "kind": "oracle", "nproc": os.cpu_count(),
                             "sample": f"{' + '.join(wl['analytics'])} on {s[1]} ({s[2]} tokens) per step"},
            "e2e": {"value": v, "unit": "tokens/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def workload_summary(m: dict) -> dict:
    """The figures of one measured workload for the JSON line."""
    info = m["info"]
    return {"value": m["value"], "unit": "tokens/s", "ms_per_step": m["ms_per_step"],
            "roofline": m["roofline"], "phases": m["phases"], "load_ms": m["load"], "e2e": m["e2e"],
            "gpu_launches": m["gpu_launches"], "outputs": m["outputs"], "eager_step": m["eager_step"],
            "grammar": {k: info[k] for k in ("num_tokens", "num_syms", "num_rules", "num_files", "num_edges",
                                             "depth", "owned_windows", "file_pairs")}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gtadoc", choices=["gtadoc", "reference"])
    ap.add_argument("--workload", default="multi64_50m", choices=list(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end legs (used for profiling runs)")
    ap.add_argument("--no-extras", action="store_true", help="skip every secondary measurement")
    ap.add_argument("--no-c3", action="store_true", help="skip the 500M-token 3-gram workload in the extras")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving (p50/p99) measurement")
    ap.add_argument("--no-autotune", action="store_true", help="time the default launch configuration")
    ap.add_argument("--eager", action="store_true",
                    help="time the step launched kernel by kernel instead of as one graph (profiling captures)")
    ap.add_argument("--scale", type=float, default=1.0,
                    help="corpus scale for profiling captures of a smaller case (1.0 = the workload as stated)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    rank, world, local = dist_env()
    if args.impl == "reference":
        reference_arm(args, rank)
        return

    import torch
    from paper_2106_06889_gb300 import binding as B
    from paper_2106_06889_gb300.corpus import load_config

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    wl = WORKLOADS[args.workload]
    g, _ = load_config(args.workload, scale=args.scale)  # every rank analyses its own resident copy (weak scaling)
    ctx = B.gt_create(local)
    stream = torch.cuda.Stream()
    m = measure(B, ctx, args.workload, g, args.steps, args.warmup, world, stream,
                autotune=not args.no_autotune, e2e_steps=0 if args.no_e2e else max(2, min(args.steps, 5)),
                eager=args.eager)
    extras = {}

    def fresh(fn):
        """Run fn on a context of its own, destroyed afterwards (a context's
        stream-ordered pool keeps what a large workload allocated).  A failing
        extra is reported in the line as {"error": ...} and on stderr, and the
        headline still prints."""
        c = B.gt_create(local)
        try:
            return fn(c)
        except Exception as e:
            import traceback
            traceback.print_exc()
            return {"error": f"{type(e).__name__}: {e}"}
        finally:
            torch.cuda.synchronize()
            B.gt_destroy(c)

    def against(unc, value):
        if "value" in unc:
            unc["compressed_over_uncompressed"] = value / unc["value"]
        return unc

    if not args.no_extras and world == 1:
        extras["sequence_count_paths"] = {"corpus": args.workload, **sequence_paths(B, ctx, g, stream)}
        unc = fresh(lambda c: uncompressed_baseline(B, c, args.workload, stream))
        extras["uncompressed_baseline"] = {args.workload: against(unc, m["value"])}
        extras["small_word_count"] = fresh(lambda c: small_word_count(B, c))
        extras["many_files"] = fresh(lambda c: many_files(B, c))
        other = "nested_500m" if args.workload != "nested_500m" else None
        if other and not args.no_c3:
            g3, _ = load_config(other)

            def c3(c):
                m3 = measure(B, c, other, g3, max(3, min(args.steps, 10)), 3, world, stream, autotune=False,
                             e2e_steps=0 if args.no_e2e else 2, clocks=False)
                return {"m3": m3, "paths": sequence_paths(B, c, g3, stream)}

            r3 = fresh(c3)
            if "error" in r3:
                extras[other] = r3
            else:
                m3 = r3["m3"]
                x = {"workload": other, "desc": WORKLOADS[other]["desc"], "analytics": WORKLOADS[other]["analytics"],
                     **workload_summary(m3), "sequence_count_paths": r3["paths"]}
                unc = fresh(lambda c: uncompressed_baseline(B, c, other, stream, steps=3))
                extras["uncompressed_baseline"][other] = against(unc, m3["value"])
                if not args.no_cpu_baseline:
                    x["cpu_baseline"] = cpu_baselines(g3, WORKLOADS[other]["analytics"])
                extras[other] = x
            del g3
    serving = None
    if rank == 0 and world == 1 and not args.no_serving and not args.no_extras:
        serving = fresh(lambda c: serving_bench(B, c))
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baselines(g, wl["analytics"])
    if rank == 0:
        info = m["info"]
        line = {"metric": METRIC, "value": m["value"], "unit": "tokens/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": m["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
                "config": workload_config(args, g),
                "execution": "gt_plan: the step's batch captured once as a CUDA graph, one graph launch per "
                             "step recomputing every result (eager_step: the same batch by gt_run_batch)",
                "grammar": {"tokens": m["tokens"], "grammar_symbols": info["num_syms"], "rules": info["num_rules"],
                            "files": info["num_files"]},
                "autotune": m["autotune"],
                "roofline": m["roofline"], "load_ms": m["load"], "phases": m["phases"], "outputs": m["outputs"],
                "eager_step": m["eager_step"],
                "extras": extras, "serving": serving, "cpu_baseline": cpu, "e2e": m["e2e"],
                "gpu_launches": m["gpu_launches"], "clocks": m["clocks"]}
        print(json.dumps(line))
    B.gt_destroy(ctx)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
