"""The global 3-word sequence count by sample-sort buckets, bit-exact against
the oracle: sizes that span many coarse and fine buckets, hot keys (one key
owning most rows), tiny vocabularies, the in-global-memory reduction of
buckets with more distinct keys than the shared table holds (forced by a
small table), and equality with the radix-sort path it replaced."""
import numpy as np
import pytest

import oracle
from paper_2106_06889_gb300 import binding as B
from paper_2106_06889_gb300.corpus import make_corpus, root_only_grammar, sequitur
from tests.test_oracle_pins import grammar_from_rules, tiny_cases

pytestmark = pytest.mark.gpu


@pytest.fixture
def ctx():
    c = B.gt_create(0)
    B.gt_set_param(c, "seq_path", 2)  # the sample-sort bucket path
    yield c
    B.gt_destroy(c)


def zipf_grammar(n, V, s, seed, files=1, root_only=False):
    rng = np.random.default_rng(seed)
    w = np.arange(1, V + 1, dtype=np.float64) ** (-s)
    toks = rng.choice(V, size=n, p=w / w.sum()).astype(np.int32)
    cuts = np.sort(rng.integers(0, n + 1, size=files - 1))
    lens = np.diff(np.concatenate([[0], cuts, [n]])).astype(np.int64)
    if root_only:
        return root_only_grammar(toks, lens, V)
    return sequitur(toks, lens, V)


def cases():
    out = [(n, g) for n, g, _, _ in tiny_cases(seed=77, count=8)]
    n = make_corpus("nested_500m", scale=0.004)  # one file, 2M tokens, deep DAG: many buckets
    out.append(("nested2m", sequitur(n.tokens, n.file_lens, n.num_words)))
    m = make_corpus("multi64_50m", scale=0.01)  # 64 files, 500k tokens
    out.append(("multi500k", sequitur(m.tokens, m.file_lens, m.num_words)))
    # one word repeated: every window is the same key (a single hot key)
    out.append(("one_key", root_only_grammar(np.zeros(300_000, np.int32), [300_000], 4)))
    # three words, Zipf: 27 keys, each with many rows
    out.append(("v3_zipf", zipf_grammar(400_000, 3, 1.5, 5, files=3)))
    # a steep Zipf over a large vocabulary, no rules: a few hot keys among many
    out.append(("steep_root", zipf_grammar(600_000, 200_000, 1.6, 6, files=7, root_only=True)))
    out.append(("all_empty", grammar_from_rules(5, [[], [0, 1]], [0, 0, 0])))
    return out


CASES = cases()
IDS = [n for n, _ in CASES]


def run(gh):
    r = B.gt_sequence_count(gh, 0)
    k, c = B.result_numpy(r, "key"), B.result_numpy(r, "count")
    B.gt_free_result(r)
    return k, c


@pytest.mark.parametrize("name,g", CASES, ids=IDS)
def test_bucket_count_matches_oracle(ctx, name, g):
    want_k, want_c = oracle.sequence_count(g, 0)
    gh = B.gt_load_grammar(ctx, g)
    try:
        for _ in range(2):  # two runs: the same bytes
            k, c = run(gh)
            assert np.array_equal(k, want_k) and np.array_equal(c, want_c)
    finally:
        B.gt_free_grammar(gh)


SMALL_TABLE = [c for c in CASES if c[0] in ("nested2m", "multi500k", "v3_zipf", "seq0")]


@pytest.mark.parametrize("cap", [2, 40])
@pytest.mark.parametrize("name,g", SMALL_TABLE, ids=[n for n, _ in SMALL_TABLE])
def test_reduction_in_global_memory(ctx, name, g, cap):
    """A small shared table sends (almost) every fine bucket through the
    global-memory sort and run reduction."""
    B.gt_set_param(ctx, "seq_table_cap", cap)
    want_k, want_c = oracle.sequence_count(g, 0)
    gh = B.gt_load_grammar(ctx, g)
    try:
        k, c = run(gh)
        assert np.array_equal(k, want_k) and np.array_equal(c, want_c)
    finally:
        B.gt_free_grammar(gh)


def test_same_as_sort_path(ctx):
    g = CASES[IDS.index("nested2m")][1]
    gh = B.gt_load_grammar(ctx, g)
    try:
        k1, c1 = run(gh)
        B.gt_set_param(ctx, "seq_path", 1)  # the radix-sort path
        k2, c2 = run(gh)
        assert np.array_equal(k1, k2) and np.array_equal(c1, c2)
        assert int(c1.sum(dtype=np.uint64)) == B.gt_grammar_info_get(gh)["num_tokens"] - 2
    finally:
        B.gt_free_grammar(gh)


@pytest.mark.parametrize("name,g", [c for c in CASES if c[0] in ("nested2m", "multi500k", "one_key", "steep_root")],
                         ids=["nested2m", "multi500k", "one_key", "steep_root"])
def test_radix_tile_sizes(name, g):
    """The radix-sort path with tiles of 2048 and of 4096 keys per scatter
    pass ("radix_items" 8 and 16), and with the persistent prefetching
    scatter ("radix_prefetch" 1): the 3-word counts and the word sort equal
    the oracle's; an unsupported size is refused."""
    c = B.gt_create(0)
    try:
        with pytest.raises(B.GtError):
            B.gt_set_param(c, "radix_items", 12)
        B.gt_set_param(c, "seq_path", 1)
        gh = B.gt_load_grammar(c, g)
        want = oracle.sequence_count(g, 0)
        ww, wc = oracle.sort_words(g, 1)
        for items, prefetch in ((8, 0), (16, 0), (8, 1)):
            B.gt_set_param(c, "radix_items", items)
            B.gt_set_param(c, "radix_prefetch", prefetch)
            k, n = run(gh)
            assert np.array_equal(k, want[0]) and np.array_equal(n, want[1]), (items, prefetch)
            r = B.gt_sort(gh, 1)
            assert np.array_equal(B.result_numpy(r, "word"), ww) and np.array_equal(B.result_numpy(r, "count"), wc)
            B.gt_free_result(r)
        B.gt_free_grammar(gh)
    finally:
        B.gt_destroy(c)
