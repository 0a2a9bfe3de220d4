"""Host-side arithmetic of bench.py: the algorithmic bytes of a step and of
each timed kernel, the bounded oracle samples, and the file-split oracle
whose merged results must equal the single-process oracle's."""
import sys
from pathlib import Path

import numpy as np
import pytest

sys.path.insert(0, str(Path(__file__).resolve().parent.parent))
import bench  # noqa: E402
import oracle  # noqa: E402
from paper_2106_06889_gb300.corpus import make_corpus, sequitur  # noqa: E402

INFO = {"num_syms": 1000, "num_words": 500_000, "num_files": 64, "num_edges": 70, "num_rules": 40,
        "file_pairs": 20, "owned_windows": 1100}
OUT = {"tv_pairs": 90, "ii_postings": 90, "distinct_3grams": 700, "distinct_words": 300, "root_len": 400}


def test_step_bytes_per_workload():
    wc = 4 * 1000 + 8 * 70 + 8 * 40 + 8 * 500_000
    assert bench.step_bytes("multi64_50m", INFO, OUT) == wc + 8 * 20 + 12 * 90 + 4 * 90
    seq = 4 * 1000 + 8 * 40 + 16 * 40 + 32 * 1100 + 16 * 700
    assert bench.step_bytes("nested_500m", INFO, OUT) == seq + wc + 12 * 300


def test_kernel_bytes_count_only_the_methods_own_data():
    kb = bench.kernel_bytes("multi64_50m", INFO, OUT)
    assert kb["chunk_sort_root"] == ("chunk_sort_kernel<0>", 4 * 400)
    assert kb["tv_hist_kernel"] == ("tv_hist_kernel", 12 * 90)
    # the rule-word chunks read every (file, rule) weight and the rule bodies
    assert kb["chunk_sort_rules"] == ("chunk_sort_kernel<1>", 4 * 20 + 4 * 600)
    assert kb["wc_partition"] == ("wc_partition_kernel", 4 * 1000)
    kb = bench.kernel_bytes("nested_500m", INFO, OUT)
    assert kb["radix_pass"] == ("radix_downsweep_kernel<4>", 24 * 1100)  # rows read and written once a pass
    assert kb["seq_scatter"] == ("sg_scatter_kernel", 24 * 1100)
    assert kb["seq_reduce"] == ("sg_reduce_kernel", 12 * 1100 + 16 * 700)


def small_grammar(lens, seed=5):
    rng = np.random.default_rng(seed)
    lens = np.array(lens, np.int64)
    toks = rng.integers(0, 50, size=int(lens.sum())).astype(np.int32)
    return sequitur(toks, lens, 50), toks


def test_cpu_baseline_runs_the_step_analytics_on_a_prefix():
    g, _ = small_grammar([400, 300, 500, 200])
    rate, what, ntok, dt = bench.oracle_sample(g, ["word_count", "inverted_index", "term_vector"], budget_s=0.0)
    # a zero budget stops after the first prefix: one file, its tokens counted
    assert what.startswith("the first 1 of 4 files") and ntok == 400 and dt > 0 and rate == ntok / dt
    rate, what, ntok, dt = bench.oracle_sample(g, ["sequence_count"], budget_s=1e9)
    # an unbounded budget grows the prefix to every file
    assert what.startswith("the first 4 of 4 files") and ntok == 1400


def test_one_file_sample_is_a_root_prefix():
    g, toks = small_grammar([200_000])
    sub = bench.sample_grammar(g, 1000)
    e = oracle.expand_files(sub)[0]
    assert sub.num_files == 1 and int(sub.file_off[1]) == 1000
    assert np.array_equal(e, toks[:e.shape[0]])
    rate, what, ntok, dt = bench.oracle_sample(g, ["sequence_count", "sort"], budget_s=0.0)
    # a zero budget stops at the first sample: 2^16 root symbols and the words they expand to
    assert what.startswith(f"the first {1 << 16} of {int(g.file_off[1])} root symbols")
    assert ntok == int(oracle.word_count(bench.sample_grammar(g, 1 << 16)).sum())


def test_file_split_oracle_merges_to_the_oracle():
    m = make_corpus("multi64_50m", scale=0.002)  # 64 files
    g = sequitur(m.tokens, m.file_lens, m.num_words)
    analytics = ["word_count", "inverted_index", "term_vector"]
    rate, workers, dt, ntok = bench.oracle_file_split(g, analytics, 3)
    assert workers == 3 and ntok == int(m.file_lens.sum()) and rate > 0
    assert bench.oracle_file_split(small_grammar([500])[0], analytics, 3) is None  # one file


def test_file_split_merge_is_exact():
    """bench's merge of per-file-range parts (computed in-process, out of
    order) equals the oracle on the whole corpus."""
    m = make_corpus("multi64_50m", scale=0.002)
    g = sequitur(m.tokens, m.file_lens, m.num_words)
    bench._pool_init(g)
    analytics = ["word_count", "inverted_index", "term_vector"]
    parts = [bench._pool_part((a, b, analytics)) for a, b in ((21, 64), (0, 20), (20, 21))]
    merged = bench.merge_file_split(parts, analytics, g.num_words)
    assert np.array_equal(merged["word_count"], oracle.word_count(g))
    for got, want in zip(merged["inverted_index"], oracle.inverted_index(g)):
        assert np.array_equal(got, want)
    for got, want in zip(merged["term_vector"], oracle.term_vector(g)):
        assert np.array_equal(got, want)
