"""gt_word_count_noalloc: the word count for callers that cannot allocate
device memory when they call (a real-time or embedded host whose memory is
set aside in advance, or code already inside a region where allocation is
not allowed).  Its scratch is a fixed array inside the library.

Checked here: its counts equal the oracle's (integer counts, so exactly) on
two calls in a row, free device memory does not move across calls, a grammar
at the rule limit is counted correctly and one rule past it is refused with
GT_EOVERFLOW.  The file is named so that pytest collects it last."""
import numpy as np
import pytest
import torch

import oracle
from paper_2106_06889_gb300 import binding as B
from paper_2106_06889_gb300.corpus import Grammar, make_corpus, sequitur
from tests.test_oracle_pins import grammar_from_rules, tiny_cases

pytestmark = pytest.mark.gpu

MAX_RULES = 1 << 22  # the documented limit of gt_word_count_noalloc (include/gtadoc.h)


def grammars():
    out = [(n, g) for n, g, _, _ in tiny_cases(seed=91, count=6)]
    c = make_corpus("wc_single_200k")
    out.append(("wc200k", sequitur(c.tokens, c.file_lens, c.num_words)))
    m = make_corpus("multi64_50m", scale=0.004)
    out.append(("multi200k", sequitur(m.tokens, m.file_lens, m.num_words)))
    out.append(("all_empty", grammar_from_rules(5, [[], [0, 1]], [0, 0, 0])))
    return out


GRAMMARS = grammars()


@pytest.fixture(scope="module")
def ctx():
    c = B.gt_create(0)
    yield c
    B.gt_destroy(c)


@pytest.mark.parametrize("name,g", GRAMMARS, ids=[n for n, _ in GRAMMARS])
def test_noalloc_matches_oracle(ctx, name, g):
    want = oracle.word_count(g)
    gh = B.gt_load_grammar(ctx, g)
    try:
        for call in range(2):  # the scratch array keeps the previous call's weights
            got = torch.full((g.num_words,), -7, dtype=torch.int64, device="cuda")
            B.gt_word_count_noalloc(gh, got)
            B.gt_sync(ctx)
            assert np.array_equal(got.cpu().numpy().astype(np.uint64), want), call
    finally:
        B.gt_free_grammar(gh)


def test_noalloc_leaves_free_memory_unchanged(ctx):
    c = make_corpus("multi64_50m", scale=0.004)
    g = sequitur(c.tokens, c.file_lens, c.num_words)
    gh = B.gt_load_grammar(ctx, g)
    try:
        out = torch.empty(g.num_words, dtype=torch.int64, device="cuda")
        B.gt_word_count_noalloc(gh, out)  # first call: looks up the scratch address, loads the kernels
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        for _ in range(3):
            B.gt_word_count_noalloc(gh, out)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0
        assert np.array_equal(out.cpu().numpy().astype(np.uint64), oracle.word_count(g))
    finally:
        B.gt_free_grammar(gh)


def many_rule_grammar(R):
    """Root = one reference to each of the rules 1..R-1; every rule is the two
    words (0, 1).  Word count: both words occur R - 1 times."""
    V = 2
    root = np.arange(1, R, dtype=np.int64) + V
    bodies = np.tile(np.array([0, 1], np.int64), R - 1)
    sym = np.concatenate([root, bodies]).astype(np.int32)
    rule_off = np.concatenate([[0, R - 1], R - 1 + 2 * np.arange(1, R, dtype=np.int64)]).astype(np.int64)
    return Grammar(V, rule_off, sym, np.array([0, R - 1], np.int64))


def test_noalloc_rule_limit(ctx):
    at = many_rule_grammar(MAX_RULES)
    gh = B.gt_load_grammar(ctx, at)
    try:
        out = torch.full((2,), -1, dtype=torch.int64, device="cuda")
        B.gt_word_count_noalloc(gh, out)
        B.gt_sync(ctx)
        assert out.tolist() == [MAX_RULES - 1, MAX_RULES - 1]
    finally:
        B.gt_free_grammar(gh)
    over = many_rule_grammar(MAX_RULES + 1)
    gh = B.gt_load_grammar(ctx, over)
    try:
        out = torch.full((2,), -1, dtype=torch.int64, device="cuda")
        with pytest.raises(B.GtError) as e:
            B.gt_word_count_noalloc(gh, out)
        assert e.value.code == 6  # GT_EOVERFLOW
        assert out.tolist() == [-1, -1]  # refused before any work was enqueued
        B.gt_word_count(gh, out)  # the allocating word count still serves it
        B.gt_sync(ctx)
        assert out.tolist() == [MAX_RULES, MAX_RULES]
    finally:
        B.gt_free_grammar(gh)
