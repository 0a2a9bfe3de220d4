"""Parity at the full sizes of the workloads, in the launch configuration
bench.py times: the 500M-token nested corpus (word count, sort, 3-word
sequence count) and the 100k-file corpus (term vector, inverted index, ranked
index over words and over 3-word keys; bottom-up).

The oracle's definitions are applied to the generator's source text, which
is what each grammar expands to (pinned on CPU, checked here by length).
Where the whole oracle result is cheap it is compared in full; otherwise
sampled keys and files are compared exactly and the rest is checked by
properties that hold at any size."""
import numpy as np
import pytest
import torch

import oracle
from paper_2106_06889_gb300 import binding as B
from paper_2106_06889_gb300.corpus import load_config

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = B.gt_create(0)
    yield c
    B.gt_destroy(c)


def split_files(tokens, lens):
    ends = np.cumsum(lens)
    return np.split(tokens, ends[:-1])


def rows_of_keys(offs, keys, cols, pick):
    """Rows of the ranked index (CSR over ascending keys) for the picked keys."""
    out = [[] for _ in cols]
    ks = []
    for key in np.sort(np.unique(pick)):
        i = np.searchsorted(keys, key)
        if i < keys.shape[0] and keys[i] == key:
            a, b = offs[i], offs[i + 1]
            ks.append(np.full(b - a, key, np.uint64))
            for o, col in zip(out, cols):
                o.append(col[a:b])
    cat = (lambda xs: np.concatenate(xs) if xs else np.zeros(0))
    return cat(ks), [cat(o) for o in out]


def test_nested_500m(ctx):
    g, corpus = load_config("nested_500m", keep_tokens=True)
    toks = corpus.tokens
    N = toks.shape[0]
    files = [toks]
    gh = B.gt_load_grammar(ctx, g)
    try:
        info = B.gt_grammar_info_get(gh)
        assert info["num_tokens"] == N and N >= 500_000_000
        # word count and sort: in full
        out = torch.empty(g.num_words, dtype=torch.int64, device="cuda")
        B.gt_word_count(gh, out)
        B.gt_sync(ctx)
        assert np.array_equal(out.cpu().numpy().astype(np.uint64), oracle.word_count_text(files, g.num_words))
        r = B.gt_sort(gh, 1)
        w, c = oracle.sort_words_text(files, g.num_words, 1)
        assert np.array_equal(B.result_numpy(r, "word"), w)
        assert np.array_equal(B.result_numpy(r, "count"), c)
        B.gt_free_result(r)
        # 3-word sequence count: properties of the whole result ...
        r = B.gt_sequence_count(gh, 0)
        keys, counts = B.result_numpy(r, "key"), B.result_numpy(r, "count")
        B.gt_free_result(r)
        assert np.all(keys[1:] > keys[:-1])
        assert counts.min() > 0 and int(counts.sum(dtype=np.uint64)) == N - 2
        # ... and exact counts of sampled keys: drawn from the result and from
        # windows at random text positions (those must be present)
        rng = np.random.default_rng(500)
        pos = rng.integers(0, N - 2, size=1000)
        from_text = oracle.pack3(toks[pos], toks[pos + 1], toks[pos + 2])
        pick = np.concatenate([rng.choice(keys, size=1000, replace=False), from_text])
        ok, of, oc = oracle.key_file_counts_text(files, pick, 3)
        assert np.all(np.isin(from_text, ok))
        idx = np.searchsorted(keys, ok)
        assert np.all(idx < keys.shape[0]) and np.array_equal(keys[idx], ok)
        assert np.array_equal(counts[idx], oc)
    finally:
        B.gt_free_grammar(gh)


def test_files100k(ctx):
    g, corpus = load_config("files100k", keep_tokens=True)
    files = split_files(corpus.tokens, corpus.file_lens)
    F, V = len(files), g.num_words
    assert F == 100_000
    gh = B.gt_load_grammar(ctx, g)
    rng = np.random.default_rng(100)
    try:
        info = B.gt_grammar_info_get(gh)
        assert info["num_tokens"] == corpus.tokens.shape[0]
        res = B.gt_run_batch(ctx, [(gh, B.GT_Q_TERM_VECTOR, 0, None), (gh, B.GT_Q_INVERTED_INDEX, 0, None)])
        toff, tw, tc = (B.result_numpy(res[0], k) for k in ("offsets", "word", "count"))
        ioff, ifl = B.result_numpy(res[1], "offsets"), B.result_numpy(res[1], "file")
        for r in res:
            B.gt_free_result(r)
        # term vector: every file's counts add up to its length, words ascend
        assert toff.shape[0] == F + 1 and toff[-1] == tw.shape[0]
        nonempty = np.diff(toff) > 0
        sums = np.add.reduceat(tc.astype(np.int64), toff[:-1][nonempty])
        assert np.array_equal(sums, corpus.file_lens[nonempty])
        fid = np.repeat(np.arange(F), np.diff(toff))
        same = fid[1:] == fid[:-1]
        assert np.all(tw[1:][same] > tw[:-1][same])
        # ... and sampled files in full
        for f in rng.choice(F, size=300, replace=False):
            o, w, c = oracle.term_vector_text([files[f]])
            assert np.array_equal(tw[toff[f]:toff[f + 1]], w) and np.array_equal(tc[toff[f]:toff[f + 1]], c)
        # inverted index: the support of the term vector, ascending files per word
        order = np.lexsort((fid, tw))
        assert np.array_equal(ioff, np.concatenate([[0], np.cumsum(np.bincount(tw, minlength=V))]))
        assert np.array_equal(ifl, fid[order])
        # ranked index over words and over 3-word keys: sampled keys exactly
        for n in (1, 3):
            r = B.gt_ranked_index(gh, n)
            offs, keys, rf, rc = (B.result_numpy(r, k) for k in ("offsets", "key", "file", "count"))
            B.gt_free_result(r)
            assert np.all(keys[1:] > keys[:-1]) and offs[-1] == rf.shape[0]
            if n == 1:
                assert int(rc.sum(dtype=np.uint64)) == corpus.tokens.shape[0]
            pick = rng.choice(keys, size=300, replace=False)
            k, (f_, c_) = rows_of_keys(offs, keys, (rf, rc), pick)
            ok, of, oc = oracle.key_file_counts_text(files, pick, n)
            assert np.array_equal(k, ok) and np.array_equal(f_, of) and np.array_equal(c_, oc), n
    finally:
        B.gt_free_grammar(gh)
