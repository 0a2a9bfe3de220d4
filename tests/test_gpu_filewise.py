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


GRAMMARS = grammars()
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
