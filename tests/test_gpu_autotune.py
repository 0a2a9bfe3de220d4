"""gt_autotune: the chosen word-count and per-file configurations are valid,
every analytic stays bit-exact against the oracle under them (direct, graph
replay and batch paths), and kinds = 0 clears the choices."""
import numpy as np
import pytest
import torch

import oracle
from paper_2106_06889_gb300 import binding as B
from paper_2106_06889_gb300.corpus import sequitur, make_corpus

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = B.gt_create(0)
    yield c
    B.gt_destroy(c)


def corpus_grammar(nfiles=None):
    m = make_corpus("multi64_50m", scale=0.004)
    if nfiles is None:
        return sequitur(m.tokens, m.file_lens, m.num_words)
    rng = np.random.default_rng(4)
    cuts = np.sort(rng.integers(0, m.tokens.shape[0] + 1, size=nfiles - 1))
    lens = np.diff(np.concatenate([[0], cuts, [m.tokens.shape[0]]])).astype(np.int64)
    return sequitur(m.tokens, lens, m.num_words)


def check_outputs(ctx, gh, g):
    want = oracle.word_count(g)
    for _ in range(3):  # direct, capture, replay
        out = torch.full((g.num_words,), -1, dtype=torch.int64, device="cuda")
        B.gt_word_count(gh, out)
        B.gt_sync(ctx)
        assert np.array_equal(out.cpu().numpy().astype(np.uint64), want)
    r = B.gt_term_vector(gh, 0)
    offs, w, c = oracle.term_vector(g, 0)
    assert np.array_equal(B.result_numpy(r, "offsets"), offs)
    assert np.array_equal(B.result_numpy(r, "word"), w)
    assert np.array_equal(B.result_numpy(r, "count"), c)
    B.gt_free_result(r)
    r = B.gt_inverted_index(gh)
    offs, f = oracle.inverted_index(g)
    assert np.array_equal(B.result_numpy(r, "offsets"), offs)
    assert np.array_equal(B.result_numpy(r, "file"), f)
    B.gt_free_result(r)


def test_autotune_64_files(ctx):
    g = corpus_grammar()
    gh = B.gt_load_grammar(ctx, g)
    try:
        res = B.gt_autotune(gh, [B.GT_Q_WORD_COUNT, B.GT_Q_TERM_VECTOR], reps=2)
        assert res["wc_aggregate"] in (0, 1)
        assert 1 <= res["wc_slices"] <= 64
        assert res["file_strategy"] in (1, 2)
        assert res["candidates"] >= 4  # >= 2 word-count shapes x 2, plus 2 strategies
        assert res["wc_ms"] > 0 and res["file_ms"] > 0
        check_outputs(ctx, gh, g)
        cleared = B.gt_autotune(gh, [])
        assert cleared["candidates"] == 0 and cleared["file_strategy"] == 0
        check_outputs(ctx, gh, g)
    finally:
        B.gt_free_grammar(gh)


def test_autotune_many_files_picks_bottom_up(ctx):
    g = corpus_grammar(nfiles=150)
    gh = B.gt_load_grammar(ctx, g)
    try:
        res = B.gt_autotune(gh, [B.GT_Q_INVERTED_INDEX], reps=1)
        assert res["file_strategy"] == 2 and res["candidates"] == 1
        assert res["wc_ms"] == 0
        check_outputs(ctx, gh, g)
    finally:
        B.gt_free_grammar(gh)


def test_autotune_rejects_bad_reps(ctx):
    g = corpus_grammar()
    gh = B.gt_load_grammar(ctx, g)
    try:
        with pytest.raises(B.GtError) as e:
            B.gt_autotune(gh, [B.GT_Q_WORD_COUNT], reps=0)
        assert e.value.code == 1
    finally:
        B.gt_free_grammar(gh)
