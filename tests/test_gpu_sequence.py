"""GPU parity through the C ABI for head/tail-based sequence counting (global
and per file) and the ranked inverted index (3-word keys and words),
bit-exact against the CPU oracle."""
import json
from pathlib import Path

import numpy as np
import pytest

import oracle
from paper_2106_06889_gb300 import binding as B
from paper_2106_06889_gb300.corpus import (sequitur, make_corpus, root_only_grammar, refactor_grammar, prefix_files,
                                           load_config)
from tests.test_oracle_pins import tiny_cases, grammar_from_rules

pytestmark = pytest.mark.gpu
GOLDEN = Path(__file__).parent / "golden"


@pytest.fixture(scope="module")
def ctx():
    c = B.gt_create(0)
    yield c
    B.gt_destroy(c)


def grammars():
    out = [(n, g) for n, g, _, _ in tiny_cases(seed=51, count=20)]
    fx = json.loads((GOLDEN / "headtail_section4c.json").read_text())
    out.append(("paper_headtail", grammar_from_rules(fx["num_words"], fx["rules"], fx["file_off"])))
    m = make_corpus("multi64_50m", scale=0.004)  # 64 files, ~200k tokens
    g = sequitur(m.tokens, m.file_lens, m.num_words)
    out.append(("multi200k", g))
    out.append(("multi200k_refac", refactor_grammar(g, np.random.default_rng(9), rounds=2, frac=0.1)))
    out.append(("multi200k_root", root_only_grammar(m.tokens, m.file_lens, m.num_words)))
    n = make_corpus("nested_500m", scale=0.0006)  # one file, ~300k tokens, deep nesting
    out.append(("nested300k", sequitur(n.tokens, n.file_lens, n.num_words)))
    out.append(("empty_files", grammar_from_rules(5, [[0, 6, 1, 6], [2, 3]], [0, 0, 2, 2, 4, 4])))
    out.append(("short_files", grammar_from_rules(5, [[0, 1, 6, 2], [3, 4]], [0, 1, 2, 3, 4])))
    out.append(("unit_rules", grammar_from_rules(4, [[5, 1, 6, 5, 2, 7], [0], [3, 5], [6, 6]], [0, 2, 6])))
    return out


GRAMMARS = grammars()
IDS = [n for n, _ in GRAMMARS]


@pytest.mark.parametrize("name,g", GRAMMARS, ids=IDS)
def test_sequence_count(ctx, name, g):
    gh = B.gt_load_grammar(ctx, g)
    r = B.gt_sequence_count(gh, 0)
    k, c = oracle.sequence_count(g, 0)
    assert np.array_equal(B.result_numpy(r, "key"), k)
    assert np.array_equal(B.result_numpy(r, "count"), c)
    B.gt_free_result(r)
    r = B.gt_sequence_count(gh, 1)
    f, k, c = oracle.sequence_count(g, 1)
    assert np.array_equal(B.result_numpy(r, "file"), f)
    assert np.array_equal(B.result_numpy(r, "key"), k)
    assert np.array_equal(B.result_numpy(r, "count"), c)
    B.gt_free_result(r)
    B.gt_free_grammar(gh)


@pytest.mark.parametrize("n", [1, 3])
@pytest.mark.parametrize("name,g", GRAMMARS, ids=IDS)
def test_ranked_index(ctx, name, g, n):
    gh = B.gt_load_grammar(ctx, g)
    r = B.gt_ranked_index(gh, n)
    offs, keys, files, counts = oracle.ranked_index(g, n)
    assert np.array_equal(B.result_numpy(r, "offsets"), offs)
    assert np.array_equal(B.result_numpy(r, "key"), keys)
    assert np.array_equal(B.result_numpy(r, "file"), files)
    assert np.array_equal(B.result_numpy(r, "count"), counts)
    B.gt_free_result(r)
    B.gt_free_grammar(gh)


def test_owned_windows_match_eq1(ctx):
    """Sum of all 3-word counts equals sum_r wt_r * owned_r (the Eq. 1 count)."""
    n = make_corpus("nested_500m", scale=0.0006)
    g = sequitur(n.tokens, n.file_lens, n.num_words)
    gh = B.gt_load_grammar(ctx, g)
    r = B.gt_sequence_count(gh, 0)
    total = int(B.result_numpy(r, "count").astype(np.int64).sum())
    assert total == int(n.tokens.shape[0]) - 2
    B.gt_free_result(r)
    B.gt_free_grammar(gh)


def test_full_size_multifile_sequence_count(ctx):
    """The benchmark's 64-file, ~50M-token corpus: every 3-word count."""
    g, _ = load_config("multi64_50m")
    gh = B.gt_load_grammar(ctx, g)
    r = B.gt_sequence_count(gh, 0)
    k, c = oracle.sequence_count(g, 0)
    assert np.array_equal(B.result_numpy(r, "key"), k)
    assert np.array_equal(B.result_numpy(r, "count"), c)
    B.gt_free_result(r)
    B.gt_free_grammar(gh)


@pytest.mark.parametrize("per_file", [0, 1])
def test_long_runs_across_tiles(ctx, per_file):
    """Runs of one key spanning many 2048-row tiles: a root-only text that
    repeats one word (every window the same key) in three files, plus a
    stretch of other words, so runs end inside, at and past tile edges."""
    rng = np.random.default_rng(77)
    toks = np.concatenate([np.full(20000, 3, np.int32), rng.integers(0, 9, 5000).astype(np.int32),
                           np.full(4096 + 2, 5, np.int32), np.full(9000, 3, np.int32)])
    lens = np.array([20000, 9098, 9000], np.int64)
    g = root_only_grammar(toks, lens, 10)
    gh = B.gt_load_grammar(ctx, g)
    r = B.gt_sequence_count(gh, per_file)
    want = oracle.sequence_count(g, per_file)
    got = [B.result_numpy(r, k) for k in (("file", "key", "count") if per_file else ("key", "count"))]
    for a, b in zip(got, want):
        assert np.array_equal(a, b)
    B.gt_free_result(r)
    B.gt_free_grammar(gh)
