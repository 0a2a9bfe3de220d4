"""The serving loop: requests submitted while others run are admitted as slots
and memory free up, overlap on the device, and every result equals the same
query run alone (and the oracle)."""
import threading
import time

import numpy as np
import pytest
import torch

import oracle
from paper_2106_06889_gb300 import binding as B
from paper_2106_06889_gb300.corpus import sequitur, make_corpus, prefix_files

pytestmark = pytest.mark.gpu

KINDS = [B.GT_Q_WORD_COUNT, B.GT_Q_INVERTED_INDEX, B.GT_Q_SEQUENCE_COUNT, B.GT_Q_TERM_VECTOR, B.GT_Q_SORT,
         B.GT_Q_RANKED_INDEX]


@pytest.fixture(scope="module")
def setup():
    ctx = B.gt_create(0)
    m = make_corpus("multi64_50m", scale=0.004)
    g1 = sequitur(m.tokens, m.file_lens, m.num_words)
    g2 = prefix_files(g1, 9)
    n = make_corpus("nested_500m", scale=0.0004)
    g3 = sequitur(n.tokens, n.file_lens, n.num_words)
    gs = [g1, g2, g3]
    hs = [B.gt_load_grammar(ctx, g) for g in gs]
    yield ctx, gs, hs
    for h in hs:
        B.gt_free_grammar(h)
    B.gt_destroy(ctx)


def fields(kind):
    return {B.GT_Q_INVERTED_INDEX: ("offsets", "file"), B.GT_Q_TERM_VECTOR: ("offsets", "word", "count"),
            B.GT_Q_SEQUENCE_COUNT: ("key", "count"), B.GT_Q_SORT: ("word", "count"),
            B.GT_Q_RANKED_INDEX: ("offsets", "key", "file", "count")}[kind]


def param(kind):
    return {B.GT_Q_SORT: 1, B.GT_Q_RANKED_INDEX: 3}.get(kind, 0)


def oracle_of(g, kind):
    if kind == B.GT_Q_WORD_COUNT:
        return (oracle.word_count(g),)
    if kind == B.GT_Q_INVERTED_INDEX:
        return oracle.inverted_index(g)
    if kind == B.GT_Q_TERM_VECTOR:
        return oracle.term_vector(g, 0)
    if kind == B.GT_Q_SEQUENCE_COUNT:
        return oracle.sequence_count(g, 0)
    if kind == B.GT_Q_SORT:
        return oracle.sort_words(g, 1)
    return oracle.ranked_index(g, 3)


def result_arrays(r, kind, counts):
    if kind == B.GT_Q_WORD_COUNT:
        return (counts.cpu().numpy().astype(np.uint64),)
    return tuple(B.result_numpy(r, f) for f in fields(kind))


def test_mixed_requests_equal_alone_and_oracle(setup):
    ctx, gs, hs = setup
    rng = np.random.default_rng(4)
    reqs = []
    for i in range(48):
        gi = int(rng.integers(0, 3))
        kind = KINDS[int(rng.integers(0, len(KINDS)))]
        counts = torch.full((gs[gi].num_words,), -1, dtype=torch.int64, device="cuda") \
            if kind == B.GT_Q_WORD_COUNT else None
        reqs.append((gi, kind, counts))
    # alone: one query at a time through gt_run_batch
    alone = []
    for gi, kind, counts in reqs:
        c = torch.empty_like(counts) if counts is not None else None
        out = B.gt_run_batch(ctx, [(hs[gi], kind, param(kind), c)])
        torch.cuda.synchronize()
        alone.append(result_arrays(out[0], kind, c))
        if out[0] is not None:
            B.gt_free_result(out[0])
    # in the mix: submitted from a second thread at random intervals while
    # earlier requests are still running
    sv = B.gt_server_create(ctx, slots=4)
    tickets = [None] * len(reqs)

    def submit():
        for i, (gi, kind, counts) in enumerate(reqs):
            tickets[i] = B.gt_submit(sv, [(hs[gi], kind, param(kind), counts)])
            time.sleep(float(rng.exponential(0.0005)))

    th = threading.Thread(target=submit)
    th.start()
    th.join()
    mixed = []
    for i, (gi, kind, counts) in enumerate(reqs):
        out, lat = B.gt_poll(sv, tickets[i], 1)
        assert lat > 0
        mixed.append(result_arrays(out[0], kind, counts))
        if out[0] is not None:
            B.gt_free_result(out[0])
    stats = B.gt_server_stats(sv)
    B.gt_server_destroy(sv)
    assert stats["max_inflight"] >= 2  # work really overlapped
    for (gi, kind, _), a, m in zip(reqs, alone, mixed):
        want = oracle_of(gs[gi], kind)
        for x, y, z in zip(a, m, want):
            assert np.array_equal(x, y) and np.array_equal(np.asarray(x), np.asarray(z))


def test_memory_budget_serialises(setup):
    ctx, gs, hs = setup
    sv = B.gt_server_create(ctx, slots=4, mem_budget=1)  # every request alone
    with pytest.raises(B.GtError) as e:
        B.gt_submit(sv, [(hs[0], B.GT_Q_SEQUENCE_COUNT, 0, None)])
    assert e.value.code == 7  # GT_EBUSY: larger than the whole budget
    B.gt_server_destroy(sv)
    # a budget that fits one request at a time
    sv = B.gt_server_create(ctx, slots=4, mem_budget=(3 << 30))
    ts = [B.gt_submit(sv, [(hs[i % 3], B.GT_Q_INVERTED_INDEX, 0, None)]) for i in range(8)]
    for i, t in enumerate(ts):
        out, _ = B.gt_poll(sv, t, 1)
        offs, f = oracle.inverted_index(gs[i % 3])
        assert np.array_equal(B.result_numpy(out[0], "file"), f)
        B.gt_free_result(out[0])
    B.gt_server_destroy(sv)
