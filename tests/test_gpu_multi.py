"""Fused multi-grammar word count (gt_word_count_batch, and gt_run_batch over
several grammars): every grammar's counts equal the oracle's and the
single-grammar path's, bit for bit."""
import numpy as np
import pytest
import torch

import oracle
from paper_2106_06889_gb300 import binding as B
from paper_2106_06889_gb300.corpus import sequitur, make_corpus, root_only_grammar
from tests.test_oracle_pins import tiny_cases, grammar_from_rules

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = B.gt_create(0)
    yield c
    B.gt_destroy(c)


def mixed_grammars():
    out = [g for _, g, _, _ in tiny_cases(seed=61, count=8)]
    c = make_corpus("wc_single_200k")
    out.append(sequitur(c.tokens, c.file_lens, c.num_words))
    m = make_corpus("multi64_50m", scale=0.004)
    out.append(sequitur(m.tokens, m.file_lens, m.num_words))
    out.append(root_only_grammar(m.tokens[:5000], np.array([2000, 3000], np.int64), m.num_words))
    n = make_corpus("nested_500m", scale=0.0004)
    out.append(sequitur(n.tokens, n.file_lens, n.num_words))
    out.append(grammar_from_rules(5, [[], [0, 1]], [0, 0, 0]))  # no symbols in the root
    out.append(grammar_from_rules(4, [[5, 1, 6, 5, 2, 7], [0], [3, 5], [6, 6]], [0, 2, 6]))
    return out


MIXED = mixed_grammars()


def test_word_count_batch_matches_oracle(ctx):
    hs = [B.gt_load_grammar(ctx, g) for g in MIXED]
    try:
        outs = [torch.full((g.num_words,), -1, dtype=torch.int64, device="cuda") for g in MIXED]
        for rep in range(2):
            for o in outs:
                o.fill_(-1)
            B.gt_word_count_batch(hs, outs)
            B.gt_sync(ctx)
            for g, o in zip(MIXED, outs):
                assert np.array_equal(o.cpu().numpy().astype(np.uint64), oracle.word_count(g)), rep
    finally:
        for h in hs:
            B.gt_free_grammar(h)


def test_word_count_batch_over_64_grammars(ctx):
    gs = [g for _, g, _, _ in tiny_cases(seed=62, count=40)]
    gs = (gs * 2)[:70]  # 70 grammars: two fused sequences (64 + 6)
    hs = [B.gt_load_grammar(ctx, g) for g in gs]
    try:
        outs = [torch.empty(g.num_words, dtype=torch.int64, device="cuda") for g in gs]
        B.gt_word_count_batch(hs, outs)
        B.gt_sync(ctx)
        for g, o in zip(gs, outs):
            assert np.array_equal(o.cpu().numpy().astype(np.uint64), oracle.word_count(g))
    finally:
        for h in hs:
            B.gt_free_grammar(h)


def test_run_batch_fuses_grammars(ctx):
    """Word counts and sorts of several grammars in one gt_run_batch call."""
    gs = MIXED[-6:]
    hs = [B.gt_load_grammar(ctx, g) for g in gs]
    try:
        outs = [torch.empty(g.num_words, dtype=torch.int64, device="cuda") for g in gs]
        qs = [(h, B.GT_Q_WORD_COUNT, 0, o) for h, o in zip(hs, outs)]
        qs += [(h, B.GT_Q_SORT, 1, None) for h in hs[:3]]
        res = B.gt_run_batch(ctx, qs)
        B.gt_sync(ctx)
        for g, o in zip(gs, outs):
            assert np.array_equal(o.cpu().numpy().astype(np.uint64), oracle.word_count(g))
        for g, r in zip(gs[:3], res[len(gs):]):
            w, c = oracle.sort_words(g, 1)
            assert np.array_equal(B.result_numpy(r, "word"), w)
            assert np.array_equal(B.result_numpy(r, "count"), c)
            B.gt_free_result(r)
    finally:
        for h in hs:
            B.gt_free_grammar(h)


def test_word_count_batch_rejects_mixed_contexts(ctx):
    other = B.gt_create(0)
    try:
        g = MIXED[0]
        h1, h2 = B.gt_load_grammar(ctx, g), B.gt_load_grammar(other, g)
        outs = [torch.empty(g.num_words, dtype=torch.int64, device="cuda") for _ in range(2)]
        with pytest.raises(B.GtError) as e:
            B.gt_word_count_batch([h1, h2], outs)
        assert e.value.code == 1
        B.gt_free_grammar(h1)
        B.gt_free_grammar(h2)
    finally:
        B.gt_destroy(other)
