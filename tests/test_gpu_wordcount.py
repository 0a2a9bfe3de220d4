"""GPU parity through the C ABI: rule weights, word count, sort, head/tail and
load-time facts, compared element by element with the CPU oracle (bit-exact:
all of it is integer work)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2106_06889_gb300 import binding as B
from paper_2106_06889_gb300.corpus import (Grammar, sequitur, make_corpus, load_config, root_only_grammar,
                                           refactor_grammar)
from tests.test_oracle_pins import tiny_cases, grammar_from_rules

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = B.gt_create(0)
    yield c
    B.gt_destroy(c)


def small_grammars():
    out = [(n, g) for n, g, _, _ in tiny_cases(seed=21, count=24)]
    c = make_corpus("wc_single_200k")
    g = sequitur(c.tokens, c.file_lens, c.num_words)
    out.append(("wc200k", g))
    out.append(("wc200k_refac", refactor_grammar(g, np.random.default_rng(1), rounds=2, frac=0.1)))
    out.append(("wc200k_root", root_only_grammar(c.tokens, c.file_lens, c.num_words)))
    m = make_corpus("multi64_50m", scale=0.01)  # 64 files, ~500k tokens: many tiles, ragged tail
    out.append(("multi500k", sequitur(m.tokens, m.file_lens, m.num_words)))
    # edge cases: empty files, all files empty, one word, one-word rules
    out.append(("empty_files", grammar_from_rules(5, [[0, 6, 1, 6], [2, 3]], [0, 0, 2, 2, 4, 4])))
    out.append(("all_empty", grammar_from_rules(5, [[], [0, 1]], [0, 0, 0])))
    out.append(("one_word", grammar_from_rules(1, [[0]], [0, 1])))
    out.append(("unit_rules", grammar_from_rules(4, [[5, 1, 6, 5, 2, 7], [0], [3, 5], [6, 6]], [0, 2, 6])))
    return out


SMALL = small_grammars()
IDS = [n for n, _ in SMALL]


def word_count_gpu(ctx, g):
    gh = B.gt_load_grammar(ctx, g)
    try:
        out = torch.full((g.num_words,), -1, dtype=torch.int64, device="cuda")
        B.gt_word_count(gh, out)
        B.gt_sync(ctx)
        return out.cpu().numpy().astype(np.uint64)
    finally:
        B.gt_free_grammar(gh)


@pytest.mark.parametrize("name,g", SMALL, ids=IDS)
def test_word_count(ctx, name, g):
    assert np.array_equal(word_count_gpu(ctx, g), oracle.word_count(g))


@pytest.mark.parametrize("name,g", SMALL, ids=IDS)
def test_rule_weights(ctx, name, g):
    gh = B.gt_load_grammar(ctx, g)
    wt = torch.full((g.num_rules,), -1, dtype=torch.int64, device="cuda")
    B.gt_rule_weights(gh, wt)
    B.gt_sync(ctx)
    assert np.array_equal(wt.cpu().numpy().astype(np.uint64), oracle.rule_weights(g))
    B.gt_free_grammar(gh)


@pytest.mark.parametrize("name,g", [x for x in SMALL if x[0] != "wc200k_root"][:30],
                         ids=[x[0] for x in SMALL if x[0] != "wc200k_root"][:30])
def test_head_tail(ctx, name, g):
    if g.num_rules > 3000:
        pytest.skip("oracle head/tail expands every rule; kept to small grammars")
    gh = B.gt_load_grammar(ctx, g)
    h = torch.empty(2 * g.num_rules, dtype=torch.int32, device="cuda")
    t = torch.empty(2 * g.num_rules, dtype=torch.int32, device="cuda")
    B.gt_head_tail(gh, h, t)
    B.gt_sync(ctx)
    oh, ot = oracle.head_tail(g)
    assert np.array_equal(h.cpu().numpy().reshape(-1, 2), oh)
    assert np.array_equal(t.cpu().numpy().reshape(-1, 2), ot)
    B.gt_free_grammar(gh)


def test_head_tail_200k(ctx):
    c = make_corpus("wc_single_200k")
    g = sequitur(c.tokens, c.file_lens, c.num_words)
    gh = B.gt_load_grammar(ctx, g)
    h = torch.empty(2 * g.num_rules, dtype=torch.int32, device="cuda")
    t = torch.empty(2 * g.num_rules, dtype=torch.int32, device="cuda")
    B.gt_head_tail(gh, h, t)
    B.gt_sync(ctx)
    oh, ot = oracle.head_tail(g)
    assert np.array_equal(h.cpu().numpy().reshape(-1, 2), oh)
    assert np.array_equal(t.cpu().numpy().reshape(-1, 2), ot)
    B.gt_free_grammar(gh)


@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("name,g", SMALL[-10:], ids=IDS[-10:])
def test_sort(ctx, name, g, order):
    gh = B.gt_load_grammar(ctx, g)
    r = B.gt_sort(gh, order)
    w, c = oracle.sort_words(g, order)
    assert np.array_equal(B.result_numpy(r, "word"), w)
    assert np.array_equal(B.result_numpy(r, "count"), c)
    B.gt_free_result(r)
    B.gt_free_grammar(gh)


@pytest.mark.parametrize("name,g", SMALL[-10:], ids=IDS[-10:])
def test_load_facts(ctx, name, g):
    gh = B.gt_load_grammar(ctx, g)
    info = B.gt_grammar_info_get(gh)
    assert info["num_tokens"] == int(oracle.word_count(g).astype(np.int64).sum())
    if g.num_rules <= 3000:
        assert info["owned_windows"] == int(oracle.owned_windows(g).sum())
    assert info["num_syms"] == g.num_syms
    B.gt_free_grammar(gh)


def test_repeat_calls_are_identical(ctx):
    _, g = SMALL[-7]
    gh = B.gt_load_grammar(ctx, g)
    outs = []
    for _ in range(3):
        o = torch.empty(g.num_words, dtype=torch.int64, device="cuda")
        B.gt_word_count(gh, o)
        outs.append(o)
    B.gt_sync(ctx)
    assert all(torch.equal(outs[0], o) for o in outs[1:])
    B.gt_free_grammar(gh)


@pytest.mark.parametrize("bad", ["cycle", "range", "root_ref", "empty_rule", "file_off"])
def test_invalid_grammar_rejected(ctx, bad):
    V = 4
    if bad == "cycle":
        g = grammar_from_rules(V, [[5, 0], [6, 1], [5, 2]], [0, 2])
    elif bad == "range":
        g = grammar_from_rules(V, [[0, 9]], [0, 2])
    elif bad == "root_ref":
        g = grammar_from_rules(V, [[0, 5], [4, 1]], [0, 2])
    elif bad == "empty_rule":
        g = Grammar(V, np.array([0, 2, 2], np.int64), np.array([0, 1], np.int32), np.array([0, 2], np.int64))
    else:
        g = grammar_from_rules(V, [[0, 1]], [0, 3])
    with pytest.raises(B.GtError) as e:
        B.gt_load_grammar(ctx, g)
    assert e.value.code == 1  # GT_EINVAL


def test_full_size_multifile_word_count(ctx):
    """64 files, ~50M tokens (the benchmark's corpus): every count equals the oracle's."""
    g, _ = load_config("multi64_50m")
    got = word_count_gpu(ctx, g)
    assert np.array_equal(got, oracle.word_count(g))


def test_graph_replay_matches(ctx):
    """Word counts replayed from a captured CUDA graph equal direct launches and
    the oracle, across calls and after the buffer is reused."""
    c = make_corpus("wc_single_200k")
    g = sequitur(c.tokens, c.file_lens, c.num_words)
    gh = B.gt_load_grammar(ctx, g)
    want = oracle.word_count(g)
    out = torch.empty(g.num_words, dtype=torch.int64, device="cuda")
    for i in range(4):  # call 1 direct, call 2 captures, calls 3-4 replay
        out.fill_(-7)
        before = B.gt_kernel_launches()
        B.gt_word_count(gh, out)
        B.gt_sync(ctx)
        assert B.gt_kernel_launches() > before
        assert np.array_equal(out.cpu().numpy().astype(np.uint64), want), i
    B.gt_set_param(ctx, "use_graphs", 0)
    out.fill_(-7)
    B.gt_word_count(gh, out)
    B.gt_sync(ctx)
    assert np.array_equal(out.cpu().numpy().astype(np.uint64), want)
    B.gt_set_param(ctx, "use_graphs", 1)
    B.gt_free_grammar(gh)


def test_graph_cache_bounded_by_lru(ctx):
    """More output buffers than the per-grammar graph cache holds (8): every
    call, captured, replayed or after an eviction, gives the oracle's counts."""
    c = make_corpus("wc_single_200k", scale=0.25)
    g = sequitur(c.tokens, c.file_lens, c.num_words)
    gh = B.gt_load_grammar(ctx, g)
    want = oracle.word_count(g)
    outs = [torch.empty(g.num_words, dtype=torch.int64, device="cuda") for _ in range(12)]
    for rnd in range(3):  # buffer k: direct, captured, replayed or re-captured after eviction
        for k, out in enumerate(outs):
            out.fill_(-3)
            B.gt_word_count(gh, out)
        B.gt_sync(ctx)
        for k, out in enumerate(outs):
            assert np.array_equal(out.cpu().numpy().astype(np.uint64), want), (rnd, k)
    B.gt_free_grammar(gh)
