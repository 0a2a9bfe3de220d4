"""Parity at the full sizes of the workloads, in the launch configuration
bench.py times: the 500M-token nested corpus (word count, sort and the
3-word sequence count, all compared in full) and the many-files corpus at
its stated file lengths of 1k-50k tokens (term vector and inverted index in
full, ranked index over words and over 3-word keys on 10k sampled keys each;
bottom-up), on 20k of its 100k files so that the oracle finishes in minutes.

The oracle's definitions are applied to the generator's source text, which
is what each grammar expands to (pinned on CPU, checked here by length)."""
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
        # 3-word sequence count: every key and count, by the radix-sort path
        # (default) and by the sample-sort buckets
        want_k, want_c = oracle.sequence_count_text(files, g.num_words, 0)
        for path in (1, 2):
            B.gt_set_param(ctx, "seq_path", path)
            r = B.gt_sequence_count(gh, 0)
            keys, counts = B.result_numpy(r, "key"), B.result_numpy(r, "count")
            B.gt_free_result(r)
            assert np.array_equal(keys, want_k) and np.array_equal(counts, want_c), path
            del keys, counts
        B.gt_set_param(ctx, "seq_path", 1)
    finally:
        B.gt_free_grammar(gh)


def test_files_stated_lengths(ctx):
    """20,000 files of 1k-50k tokens (~250M tokens; the first 20k files of the
    100k-file workload, which bench.py times in full): nearly half of the
    files exceed what one CTA sorts in shared memory, so the bottom-up global
    (file, word) sort runs."""
    g, corpus = load_config("files100k", scale=0.2, keep_tokens=True)
    files = split_files(corpus.tokens, corpus.file_lens)
    F, V = len(files), g.num_words
    assert F == 20_000 and corpus.file_lens.min() >= 1000 and corpus.file_lens.max() <= 50_000
    # log-uniform lengths: ln(50/8.192) / ln(50) = 46% of the files exceed 8,192 words
    assert (corpus.file_lens > 8192).mean() > 0.4
    gh = B.gt_load_grammar(ctx, g)
    rng = np.random.default_rng(100)
    try:
        info = B.gt_grammar_info_get(gh)
        assert info["num_tokens"] == corpus.tokens.shape[0]
        res = B.gt_run_batch(ctx, [(gh, B.GT_Q_TERM_VECTOR, 0, None), (gh, B.GT_Q_INVERTED_INDEX, 0, None)])
        got_tv = [B.result_numpy(res[0], k) for k in ("offsets", "word", "count")]
        got_ii = [B.result_numpy(res[1], k) for k in ("offsets", "file")]
        for r in res:
            B.gt_free_result(r)
        # term vector and inverted index: in full, against the oracle on the text
        for got, want in zip(got_tv, oracle.term_vector_text(files)):
            assert np.array_equal(got, want)
        for got, want in zip(got_ii, oracle.inverted_index_text(files, V)):
            assert np.array_equal(got, want)
        del got_tv, got_ii
        # ranked index over words and over 3-word keys: 10k sampled keys exactly
        for n in (1, 3):
            r = B.gt_ranked_index(gh, n)
            offs, keys, rf, rc = (B.result_numpy(r, k) for k in ("offsets", "key", "file", "count"))
            B.gt_free_result(r)
            assert np.all(keys[1:] > keys[:-1]) and offs[-1] == rf.shape[0]
            if n == 1:
                assert int(rc.sum(dtype=np.uint64)) == corpus.tokens.shape[0]
            pick = rng.choice(keys, size=10_000, replace=False)
            k, (f_, c_) = rows_of_keys(offs, keys, (rf, rc), pick)
            ok, of, oc = oracle.key_file_counts_text(files, pick, n)
            assert np.array_equal(k, ok) and np.array_equal(f_, of) and np.array_equal(c_, oc), n
    finally:
        B.gt_free_grammar(gh)
