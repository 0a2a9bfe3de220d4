"""GPU parity through the C ABI for the bottom-up per-file strategy (Section
IV-A; selected for many files, Section V-C): term vector, inverted index,
per-file sequence count and ranked index, bit-exact against the CPU oracle,
forced on grammars of any file count and chosen automatically beyond 64
files."""
import numpy as np
import pytest
import torch

import oracle
from paper_2106_06889_gb300 import binding as B
from paper_2106_06889_gb300.corpus import sequitur, make_corpus, refactor_grammar, root_only_grammar
from tests.test_oracle_pins import tiny_cases, grammar_from_rules

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = B.gt_create(0)
    yield c
    B.gt_destroy(c)


def split_files(tokens, nfiles, rng):
    """Cut one token stream into `nfiles` files of random (possibly zero) lengths."""
    cuts = np.sort(rng.integers(0, tokens.shape[0] + 1, size=nfiles - 1))
    return np.diff(np.concatenate([[0], cuts, [tokens.shape[0]]])).astype(np.int64)


def grammars():
    out = [(n, g) for n, g, _, _ in tiny_cases(seed=71, count=12)]
    rng = np.random.default_rng(17)
    nest = make_corpus("nested_500m", scale=0.0004)  # ~200k tokens, deep nesting
    for nf in (3, 65, 300):
        lens = split_files(nest.tokens, nf, rng)
        out.append((f"nested_{nf}files", sequitur(nest.tokens, lens, nest.num_words)))
    m = make_corpus("multi64_50m", scale=0.004)  # 64 files, ~200k tokens
    g = sequitur(m.tokens, m.file_lens, m.num_words)
    out.append(("multi200k", g))
    out.append(("multi200k_refac", refactor_grammar(g, np.random.default_rng(3), rounds=2, frac=0.1)))
    out.append(("multi200k_root", root_only_grammar(m.tokens, m.file_lens, m.num_words)))
    out.append(("empty_files", grammar_from_rules(5, [[0, 6, 1, 6], [2, 3]], [0, 0, 2, 2, 4, 4])))
    out.append(("all_empty", grammar_from_rules(5, [[], [0, 1]], [0, 0, 0])))
    out.append(("short_files", grammar_from_rules(5, [[0, 1, 6, 2], [3, 4]], [0, 1, 2, 3, 4])))
    out.append(("unit_rules", grammar_from_rules(4, [[5, 1, 6, 5, 2, 7], [0], [3, 5], [6, 6]], [0, 2, 6])))
    return out


GRAMMARS = grammars()
IDS = [n for n, _ in GRAMMARS]


def check_all(ctx, g):
    gh = B.gt_load_grammar(ctx, g)
    try:
        for k in (0, 1, 3):
            r = B.gt_term_vector(gh, k)
            offs, w, c = oracle.term_vector(g, k)
            assert np.array_equal(B.result_numpy(r, "offsets"), offs), k
            assert np.array_equal(B.result_numpy(r, "word"), w), k
            assert np.array_equal(B.result_numpy(r, "count"), c), k
            B.gt_free_result(r)
        r = B.gt_inverted_index(gh)
        offs, f = oracle.inverted_index(g)
        assert np.array_equal(B.result_numpy(r, "offsets"), offs)
        assert np.array_equal(B.result_numpy(r, "file"), f)
        B.gt_free_result(r)
        r = B.gt_sequence_count(gh, 1)
        f, k, c = oracle.sequence_count(g, 1)
        assert np.array_equal(B.result_numpy(r, "file"), f)
        assert np.array_equal(B.result_numpy(r, "key"), k)
        assert np.array_equal(B.result_numpy(r, "count"), c)
        B.gt_free_result(r)
        for n in (1, 3):
            r = B.gt_ranked_index(gh, n)
            offs, keys, files, counts = oracle.ranked_index(g, n)
            assert np.array_equal(B.result_numpy(r, "offsets"), offs), n
            assert np.array_equal(B.result_numpy(r, "key"), keys), n
            assert np.array_equal(B.result_numpy(r, "file"), files), n
            assert np.array_equal(B.result_numpy(r, "count"), counts), n
            B.gt_free_result(r)
    finally:
        B.gt_free_grammar(gh)


@pytest.mark.parametrize("local", [1, 0], ids=["smem_files", "global_sort"])
@pytest.mark.parametrize("name,g", GRAMMARS, ids=IDS)
def test_forced_bottom_up(ctx, name, g, local):
    """Bottom-up forced; word rows either per file in shared memory (files of
    at most 8192 tokens) or by the global (file, word) sort."""
    B.gt_set_param(ctx, "file_strategy", 2)
    B.gt_set_param(ctx, "bu_local", local)
    try:
        check_all(ctx, g)
    finally:
        B.gt_set_param(ctx, "file_strategy", 0)
        B.gt_set_param(ctx, "bu_local", 1)


@pytest.mark.parametrize("name,g", [x for x in GRAMMARS if x[0].startswith("nested_")],
                         ids=[n for n in IDS if n.startswith("nested_")])
def test_auto_strategy(ctx, name, g):
    """Default selection: top-down up to 64 files, bottom-up beyond."""
    check_all(ctx, g)


def test_top_down_beyond_64_files_reported(ctx):
    g = dict(GRAMMARS)["nested_300files"]
    B.gt_set_param(ctx, "file_strategy", 1)
    gh = B.gt_load_grammar(ctx, g)
    try:
        with pytest.raises(B.GtError) as e:
            B.gt_term_vector(gh, 0)
        assert e.value.code == 6  # GT_EOVERFLOW: top-down file masks hold 64 files
    finally:
        B.gt_free_grammar(gh)
        B.gt_set_param(ctx, "file_strategy", 0)


def test_batch_shares_bottom_up_rows(ctx):
    """gt_run_batch over a 300-file grammar: TV, TV top-k, II from one pass."""
    g = dict(GRAMMARS)["nested_300files"]
    gh = B.gt_load_grammar(ctx, g)
    try:
        wc = torch.empty(g.num_words, dtype=torch.int64, device="cuda")
        res = B.gt_run_batch(ctx, [(gh, B.GT_Q_TERM_VECTOR, 0, None), (gh, B.GT_Q_TERM_VECTOR, 5, None),
                                   (gh, B.GT_Q_INVERTED_INDEX, 0, None), (gh, B.GT_Q_WORD_COUNT, 0, wc)])
        for r, k in ((res[0], 0), (res[1], 5)):
            offs, w, c = oracle.term_vector(g, k)
            assert np.array_equal(B.result_numpy(r, "offsets"), offs)
            assert np.array_equal(B.result_numpy(r, "word"), w)
            assert np.array_equal(B.result_numpy(r, "count"), c)
        offs, f = oracle.inverted_index(g)
        assert np.array_equal(B.result_numpy(res[2], "offsets"), offs)
        assert np.array_equal(B.result_numpy(res[2], "file"), f)
        B.gt_sync(ctx)
        assert np.array_equal(wc.cpu().numpy().astype(np.uint64), oracle.word_count(g))
        for r in res:
            if r is not None:
                B.gt_free_result(r)
    finally:
        B.gt_free_grammar(gh)


@pytest.mark.parametrize("name,scale,files", [("files_short", 0.02, 2000), ("files100k", 0.002, 200)])
def test_many_files(ctx, name, scale, files):
    """The many-files workloads (Zipf 1.1 over 200k words): 2000 files of
    100-5000 tokens (per-file shared-memory path) and 200 files of 1k-50k
    tokens (global sort path): ranked index (words and 3-word keys), term
    vector and inverted index."""
    c = make_corpus(name, scale=scale)
    g = sequitur(c.tokens, c.file_lens, c.num_words)
    assert g.num_files == files
    check_all(ctx, g)
