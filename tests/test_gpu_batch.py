"""gt_run_batch: several analytics over several grammars in one call give the
same results as the oracle (and as one-query-at-a-time calls)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2106_06889_gb300 import binding as B
from paper_2106_06889_gb300.corpus import sequitur, make_corpus, prefix_files

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = B.gt_create(0)
    yield c
    B.gt_destroy(c)


def test_mixed_batch_two_grammars(ctx):
    m = make_corpus("multi64_50m", scale=0.004)
    g1 = sequitur(m.tokens, m.file_lens, m.num_words)
    g2 = prefix_files(g1, 5)
    c = make_corpus("wc_single_200k", scale=0.5)
    g3 = sequitur(c.tokens, c.file_lens, c.num_words)
    hs = [B.gt_load_grammar(ctx, g) for g in (g1, g2, g3)]
    wc = [torch.empty(g.num_words, dtype=torch.int64, device="cuda") for g in (g1, g2, g3)]
    qs = [(hs[0], B.GT_Q_TERM_VECTOR, 0, None), (hs[0], B.GT_Q_WORD_COUNT, 0, wc[0]),
          (hs[1], B.GT_Q_INVERTED_INDEX, 0, None), (hs[0], B.GT_Q_INVERTED_INDEX, 0, None),
          (hs[2], B.GT_Q_SORT, 1, None), (hs[0], B.GT_Q_TERM_VECTOR, 4, None),
          (hs[2], B.GT_Q_WORD_COUNT, 0, wc[2]), (hs[1], B.GT_Q_SORT, 0, None),
          (hs[0], B.GT_Q_INVERTED_INDEX, 0, None),
          # a word count with an inverted index and no full term vector: summed from the files' pieces
          (hs[1], B.GT_Q_WORD_COUNT, 0, wc[1])]
    outs = B.gt_run_batch(ctx, qs)
    gs = {id(hs[0]): g1, id(hs[1]): g2, id(hs[2]): g3}
    for (gh, kind, param, counts), r in zip(qs, outs):
        g = gs[id(gh)]
        if kind == B.GT_Q_WORD_COUNT:
            assert r is None
            torch.cuda.synchronize()
            assert np.array_equal(counts.cpu().numpy().astype(np.uint64), oracle.word_count(g))
        elif kind == B.GT_Q_SORT:
            w, cnt = oracle.sort_words(g, param)
            assert np.array_equal(B.result_numpy(r, "word"), w) and np.array_equal(B.result_numpy(r, "count"), cnt)
        elif kind == B.GT_Q_TERM_VECTOR:
            offs, w, cnt = oracle.term_vector(g, param)
            assert np.array_equal(B.result_numpy(r, "offsets"), offs)
            assert np.array_equal(B.result_numpy(r, "word"), w) and np.array_equal(B.result_numpy(r, "count"), cnt)
        else:
            offs, f = oracle.inverted_index(g)
            assert np.array_equal(B.result_numpy(r, "offsets"), offs) and np.array_equal(B.result_numpy(r, "file"), f)
        if r is not None:
            B.gt_free_result(r)
    for h in hs:
        B.gt_free_grammar(h)


def test_batch_rejects_bad_query(ctx):
    c = make_corpus("wc_single_200k", scale=0.1)
    g = sequitur(c.tokens, c.file_lens, c.num_words)
    h = B.gt_load_grammar(ctx, g)
    with pytest.raises(B.GtError):
        B.gt_run_batch(ctx, [(h, B.GT_Q_WORD_COUNT, 0, None)])  # word count needs an output buffer
    with pytest.raises(B.GtError):
        B.gt_run_batch(ctx, [(h, 99, 0, None)])
    B.gt_free_grammar(h)


def test_plan_replays_the_batch(ctx):
    """A batch captured as one CUDA graph (gt_plan): every launch gives the
    oracle's results (word count into the caller's buffer, term vector,
    inverted index, TF-IDF, sequence count, sort), launch after launch."""
    import torch
    m = make_corpus("multi64_50m", scale=0.004)
    g = sequitur(m.tokens, m.file_lens, m.num_words)
    gh = B.gt_load_grammar(ctx, g)
    counts = torch.empty(g.num_words, dtype=torch.int64, device="cuda")
    qs = [(gh, B.GT_Q_WORD_COUNT, 0, counts), (gh, B.GT_Q_TERM_VECTOR, 0, None), (gh, B.GT_Q_INVERTED_INDEX, 0, None),
          (gh, B.GT_Q_TFIDF, 0, None), (gh, B.GT_Q_SEQUENCE_COUNT, 0, None), (gh, B.GT_Q_SORT, 1, None)]
    p = B.gt_plan_create(ctx, qs)
    try:
        wc = oracle.word_count(g)
        tv = oracle.term_vector(g, 0)
        ii = oracle.inverted_index(g)
        tf = oracle.tfidf(g)
        sq = oracle.sequence_count(g, 0)
        so = oracle.sort_words(g, 1)
        for launch in range(3):
            counts.fill_(-1)
            B.gt_plan_launch(p)
            assert np.array_equal(B.plan_result_numpy(p, 1, "word"), tv[1]), launch
            assert np.array_equal(B.plan_result_numpy(p, 1, "count"), tv[2])
            assert np.array_equal(B.plan_result_numpy(p, 2, "offsets"), ii[0])
            assert np.array_equal(B.plan_result_numpy(p, 2, "file"), ii[1])
            np.testing.assert_allclose(B.plan_result_numpy(p, 3, "tfidf"), tf[2], rtol=1e-15, atol=0)
            assert np.array_equal(B.plan_result_numpy(p, 4, "key"), sq[0])
            assert np.array_equal(B.plan_result_numpy(p, 4, "count"), sq[1])
            assert np.array_equal(B.plan_result_numpy(p, 5, "word"), so[0])
            assert np.array_equal(counts.cpu().numpy().astype(np.uint64), wc)
    finally:
        B.gt_plan_destroy(p)
        B.gt_free_grammar(gh)
