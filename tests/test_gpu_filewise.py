"""GPU parity through the C ABI for the per-file analytics (term vector, with
and without top-k, and inverted index), bit-exact against the CPU oracle."""
import numpy as np
import pytest

import oracle
from paper_2106_06889_gb300 import binding as B
from paper_2106_06889_gb300.corpus import (sequitur, make_corpus, load_config, root_only_grammar, refactor_grammar,
                                           prefix_files)
from tests.test_oracle_pins import tiny_cases, grammar_from_rules

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = B.gt_create(0)
    yield c
    B.gt_destroy(c)


def grammars():
    out = [(n, g) for n, g, _, _ in tiny_cases(seed=33, count=20)]
    m = make_corpus("multi64_50m", scale=0.01)  # 64 files, ~500k tokens
    g = sequitur(m.tokens, m.file_lens, m.num_words)
    out.append(("multi500k", g))
    out.append(("multi500k_refac", refactor_grammar(g, np.random.default_rng(5), rounds=2, frac=0.1)))
    out.append(("multi500k_root", root_only_grammar(m.tokens, m.file_lens, m.num_words)))
    out.append(("multi500k_8files", prefix_files(g, 8)))
    out.append(("empty_files", grammar_from_rules(5, [[0, 6, 1, 6], [2, 3]], [0, 0, 2, 2, 4, 4])))
    out.append(("all_empty", grammar_from_rules(5, [[], [0, 1]], [0, 0, 0])))
    out.append(("unit_rules", grammar_from_rules(4, [[5, 1, 6, 5, 2, 7], [0], [3, 5], [6, 6]], [0, 2, 6])))
    return out


def heavy_parents_grammar(seed=12, F=8, H=3000, C=1500, V=4000):
    """Rules with many parents: B = (w0 w1) is used by H rules A_k = (B w_k),
    and A_0 by C rules C_j = (A_0 w_j); the root's files reference every A_k
    and C_j (round robin) and some words.  B's per-file weights sum over
    several thousand parent edges (more than one edge task), A_0's over
    1,500 plus the root's references."""
    rng = np.random.default_rng(seed)
    B_, A0, C0 = 1, 2, 2 + H
    rules = [None, [0, 1]]
    rules += [[V + B_, 2 + k % (V - 2)] for k in range(H)]
    rules += [[V + A0, 2 + j % (V - 2)] for j in range(C)]
    refs = [V + A0 + k for k in range(H)] + [V + C0 + j for j in range(C)]
    files = [[] for _ in range(F)]
    for i, r in enumerate(refs):
        files[i % F].append(r)
    for f in range(F):
        extra = rng.choice(refs, size=200).tolist() + rng.integers(0, V, size=100).tolist()
        body = files[f] + extra
        rng.shuffle(body)
        files[f] = body
    rules[0] = [x for b in files for x in b]
    off = np.concatenate([[0], np.cumsum([len(b) for b in files])])
    return grammar_from_rules(V, rules, off)


GRAMMARS = grammars() + [("heavy_parents", heavy_parents_grammar())]
IDS = [n for n, _ in GRAMMARS]


def check_tv(gh, g, k):
    r = B.gt_term_vector(gh, k)
    offs, w, c = oracle.term_vector(g, k)
    assert np.array_equal(B.result_numpy(r, "offsets"), offs)
    assert np.array_equal(B.result_numpy(r, "word"), w)
    assert np.array_equal(B.result_numpy(r, "count"), c)
    B.gt_free_result(r)


def check_ii(gh, g):
    r = B.gt_inverted_index(gh)
    offs, f = oracle.inverted_index(g)
    assert np.array_equal(B.result_numpy(r, "offsets"), offs)
    assert np.array_equal(B.result_numpy(r, "file"), f)
    B.gt_free_result(r)


@pytest.mark.parametrize("name,g", GRAMMARS, ids=IDS)
def test_term_vector(ctx, name, g):
    gh = B.gt_load_grammar(ctx, g)
    for k in (0, 1, 3):
        check_tv(gh, g, k)
    B.gt_free_grammar(gh)


@pytest.mark.parametrize("name,g", GRAMMARS, ids=IDS)
def test_inverted_index(ctx, name, g):
    gh = B.gt_load_grammar(ctx, g)
    check_ii(gh, g)
    B.gt_free_grammar(gh)


def test_full_size_multifile_tv_ii(ctx):
    """64 files, ~50M tokens (the benchmark's corpus): the whole term vector
    and inverted index equal the oracle's."""
    g, _ = load_config("multi64_50m")
    gh = B.gt_load_grammar(ctx, g)
    check_tv(gh, g, 0)
    check_ii(gh, g)
    check_tv(gh, g, 10)
    B.gt_free_grammar(gh)
