"""TF-IDF and word co-occurrence through the C ABI against the oracle: both
per-file strategies for TF-IDF (top-down for few files, bottom-up forced and
for many files), the 3-word-window derivation of co-occurrence on grammars
with short, empty and one-word files, and both through gt_run_batch.

TF-IDF values are float64: count * ln(F / df).  The quotient and the product
are correctly rounded on both sides; the logarithms (CUDA's and numpy's)
are each within 1 ulp, so the values agree to a few ulp: rtol = 1e-15
(about 4.5 ulp).  Words, offsets and counts are compared exactly."""
import numpy as np
import pytest
import torch

import oracle
from paper_2106_06889_gb300 import binding as B
from paper_2106_06889_gb300.corpus import make_corpus, sequitur, refactor_grammar
from tests.test_oracle_pins import grammar_from_rules, tiny_cases

pytestmark = pytest.mark.gpu
RTOL = 1e-15


@pytest.fixture
def ctx():
    c = B.gt_create(0)
    yield c
    B.gt_destroy(c)


def cases():
    out = [(n, g) for n, g, _, _ in tiny_cases(seed=33, count=10)]
    m = make_corpus("multi64_50m", scale=0.004)
    g = sequitur(m.tokens, m.file_lens, m.num_words)
    out.append(("multi200k", g))
    out.append(("multi200k_refac", refactor_grammar(g, np.random.default_rng(3), rounds=2, frac=0.1)))
    fs = make_corpus("files_short", scale=0.002)  # 200 files: bottom-up
    out.append(("files200", sequitur(fs.tokens, fs.file_lens, fs.num_words)))
    out.append(("short_files", grammar_from_rules(5, [[0, 1, 6, 2], [3, 4]], [0, 1, 2, 3, 4])))
    out.append(("empty_files", grammar_from_rules(5, [[0, 6, 1, 6], [2, 3]], [0, 0, 2, 2, 4, 4])))
    out.append(("unit_rules", grammar_from_rules(4, [[5, 1, 6, 5, 2, 7], [0], [3, 5], [6, 6]], [0, 2, 6])))
    out.append(("one_word_files", grammar_from_rules(4, [[0, 5, 1], [2]], [0, 1, 2, 3])))
    return out


CASES = cases()
IDS = [n for n, _ in CASES]


def check_tfidf(r, g):
    offs, words, vals = oracle.tfidf(g)
    assert np.array_equal(B.result_numpy(r, "offsets"), offs)
    assert np.array_equal(B.result_numpy(r, "word"), words)
    got = B.result_numpy(r, "tfidf")
    assert got.dtype == np.float64
    np.testing.assert_allclose(got, vals, rtol=RTOL, atol=0)
    assert np.array_equal(got == 0.0, vals == 0.0)  # words in every file: exactly 0


@pytest.mark.parametrize("strategy", [0, 2])
@pytest.mark.parametrize("name,g", CASES, ids=IDS)
def test_tfidf(ctx, name, g, strategy):
    B.gt_set_param(ctx, "file_strategy", strategy)  # 0: automatic (top-down up to 64 files), 2: bottom-up
    gh = B.gt_load_grammar(ctx, g)
    try:
        r = B.gt_tfidf(gh)
        check_tfidf(r, g)
        B.gt_free_result(r)
    finally:
        B.gt_free_grammar(gh)


@pytest.mark.parametrize("name,g", CASES, ids=IDS)
def test_cooccurrence(ctx, name, g):
    gh = B.gt_load_grammar(ctx, g)
    try:
        k, c = oracle.cooccurrence(g)
        for _ in range(2):
            r = B.gt_cooccurrence(gh)
            assert np.array_equal(B.result_numpy(r, "key"), k) and np.array_equal(B.result_numpy(r, "count"), c)
            B.gt_free_result(r)
    finally:
        B.gt_free_grammar(gh)


def test_batch_shares_the_term_vector_traversal(ctx):
    m = make_corpus("multi64_50m", scale=0.004)
    g = sequitur(m.tokens, m.file_lens, m.num_words)
    gh = B.gt_load_grammar(ctx, g)
    try:
        qs = [(gh, B.GT_Q_TERM_VECTOR, 0, None), (gh, B.GT_Q_TFIDF, 0, None), (gh, B.GT_Q_INVERTED_INDEX, 0, None),
              (gh, B.GT_Q_COOCCURRENCE, 0, None)]
        res = B.gt_run_batch(ctx, qs)
        o, w, c = oracle.term_vector(g, 0)
        assert np.array_equal(B.result_numpy(res[0], "word"), w) and np.array_equal(B.result_numpy(res[0], "count"), c)
        check_tfidf(res[1], g)
        io, fl = oracle.inverted_index(g)
        assert np.array_equal(B.result_numpy(res[2], "offsets"), io) and np.array_equal(B.result_numpy(res[2], "file"), fl)
        k, cc = oracle.cooccurrence(g)
        assert np.array_equal(B.result_numpy(res[3], "key"), k) and np.array_equal(B.result_numpy(res[3], "count"), cc)
        for r in res:
            B.gt_free_result(r)
    finally:
        B.gt_free_grammar(gh)


def test_bounded_wait_gives_up_and_the_context_stays_usable(ctx):
    """A look-back whose predecessor never publishes gives up after its poll
    limit with GT_ETIMEOUT (no hang, no fault); with the predecessor's prefix
    published it returns it; the context keeps working afterwards."""
    with pytest.raises(B.GtError) as e:
        B.gt_check_bounded_wait(ctx, False, 2000)
    assert "GT_ETIMEOUT" in str(e.value)
    assert B.gt_check_bounded_wait(ctx, True, 2000) == 7
    g = grammar_from_rules(5, [[0, 6, 1], [2, 3]], [0, 3])  # rule 1 = symbol 6
    gh = B.gt_load_grammar(ctx, g)
    out = torch.empty(5, dtype=torch.int64, device="cuda")
    B.gt_word_count(gh, out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy().astype(np.uint64), oracle.word_count(g))
    B.gt_free_grammar(gh)
