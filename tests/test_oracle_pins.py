"""Pins of the CPU oracle against things other than itself (no GPU needed).

* brute force: a recursive pure-Python expansion with dict counting
  (tests/brute.py) on many tiny grammars;
* the source text: the expansion must equal the generator's token stream;
* closed forms: sum of word counts = N, sum of term vectors = word count,
  inverted index = support of the term vectors, sum of 3-gram counts =
  sum_f max(N_f - 2, 0), Eq. 1's owned-window count W + 2S - 2 per rule, and
  sum_r wt_r * owned_r = total 3-gram count;
* grammar independence: Sequitur, root-only and randomly re-factored grammars
  of one token stream give identical outputs;
* the paper's prose examples (tests/golden/);
* planted mistakes in a copy of the oracle must each fail some pin.
"""
import copy
import json
import types
from pathlib import Path

import numpy as np
import pytest

import oracle
from oracle import impl as orc_impl
from paper_2106_06889_gb300.corpus import (Grammar, sequitur, root_only_grammar, refactor_grammar,
                                           make_corpus)
from tests import brute

GOLDEN = Path(__file__).parent / "golden"


def grammar_from_rules(V, rules, file_off):
    lens = [len(b) for b in rules]
    return Grammar(V, np.concatenate([[0], np.cumsum(lens)]).astype(np.int64),
                   np.array([x for b in rules for x in b], np.int32), np.array(file_off, np.int64))


def random_stream(rng, n, V, F):
    toks = rng.integers(0, V, size=n).astype(np.int32)
    # repeat a random phrase to create deep rules
    if n > 20:
        ph = rng.integers(0, V, size=rng.integers(3, 12))
        for _ in range(rng.integers(1, 5)):
            p = rng.integers(0, n - ph.size)
            toks[p:p + ph.size] = ph
    cuts = np.sort(rng.integers(0, n + 1, size=F - 1))
    lens = np.diff(np.concatenate([[0], cuts, [n]])).astype(np.int64)
    return toks, lens


def tiny_cases(seed=7, count=40):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.integers(0, 260))
        V = int(rng.integers(1, 7))
        F = int(rng.integers(1, 5))
        toks, lens = random_stream(rng, n, V, F)
        g = sequitur(toks, lens, V)
        out.append((f"seq{i}", g, toks, lens))
        if i % 3 == 0:
            out.append((f"refac{i}", refactor_grammar(g, rng), toks, lens))
        if i % 5 == 0:
            out.append((f"root{i}", root_only_grammar(toks, lens, V), toks, lens))
    # a grammar with one-word rules and a rule used once (not Sequitur, still valid)
    out.append(("unit_rules", grammar_from_rules(4, [[5, 1, 6, 5, 2, 7], [0], [3, 5], [6, 6]], [0, 2, 6]),
                None, None))
    return out


CASES = tiny_cases()


def split_files(toks, lens):
    offs = np.concatenate([[0], np.cumsum(lens)])
    return [toks[offs[f]:offs[f + 1]].astype(np.int64) for f in range(len(lens))]


# ---------------------------------------------------------------------------
# Pin bodies: each takes the oracle module to check, so that the planted-
# mistake tests below can run them against a broken copy.
# ---------------------------------------------------------------------------

def pin_brute(orc, g):
    files_b, _ = brute.expand_files(g)
    files_o = orc.expand_files(g)
    assert [list(map(int, f)) for f in files_o] == files_b
    assert list(map(int, orc.word_count(g))) == brute.word_count(g)
    for order in (0, 1):
        w, c = orc.sort_words(g, order)
        assert list(zip(map(int, w), map(int, c))) == brute.sort_words(g, order)
    for k in (0, 2):
        offs, w, c = orc.term_vector(g, k)
        got = [list(zip(map(int, w[offs[f]:offs[f + 1]]), map(int, c[offs[f]:offs[f + 1]])))
               for f in range(g.num_files)]
        assert got == [list(x) for x in brute.term_vector(g, k)]
    offs, fl = orc.inverted_index(g)
    assert [list(map(int, fl[offs[w]:offs[w + 1]])) for w in range(g.num_words)] == brute.inverted_index(g)
    k, c = orc.sequence_count(g, 0)
    assert list(zip(map(int, k), map(int, c))) == brute.sequence_count(g, 0)
    f, k, c = orc.sequence_count(g, 1)
    assert list(zip(map(int, f), map(int, k), map(int, c))) == brute.sequence_count(g, 1)
    for n in (1, 3):
        offs, keys, fl, cnt = orc.ranked_index(g, n)
        got = [(int(keys[i]), list(zip(map(int, fl[offs[i]:offs[i + 1]]), map(int, cnt[offs[i]:offs[i + 1]]))))
               for i in range(keys.shape[0])]
        assert got == brute.ranked_index(g, n)
    assert list(map(int, orc.rule_weights(g))) == brute.rule_weights(g)
    h, t = orc.head_tail(g)
    bh, bt = brute.head_tail(g)
    assert [tuple(map(int, x)) for x in h] == bh
    assert [tuple(map(int, x)) for x in t] == bt
    assert list(map(int, orc.owned_windows(g))) == brute.owned_windows(g)
    offs, w, v = orc.tfidf(g)
    got = [list(zip(map(int, w[offs[f]:offs[f + 1]]), map(float, v[offs[f]:offs[f + 1]])))
           for f in range(g.num_files)]
    want = brute.tfidf(g)
    assert [[x[0] for x in f] for f in got] == [[x[0] for x in f] for f in want]
    np.testing.assert_allclose([x[1] for f in got for x in f], [x[1] for f in want for x in f], rtol=1e-15, atol=0)
    k, c = orc.cooccurrence(g)
    assert list(zip(map(int, k), map(int, c))) == brute.cooccurrence(g)


def pin_source(orc, g, toks, lens):
    got = orc.expand_files(g)
    want = split_files(toks, lens)
    assert len(got) == len(want)
    for a, b in zip(got, want):
        assert np.array_equal(a, b)


def pin_closed_forms(orc, g, N_f):
    N = int(sum(N_f))
    wc = orc.word_count(g).astype(np.int64)
    assert int(wc.sum()) == N
    offs, w, c = orc.term_vector(g, 0)
    acc = np.zeros(g.num_words, np.int64)
    np.add.at(acc, w.astype(np.int64), c.astype(np.int64))
    assert np.array_equal(acc, wc)
    assert np.array_equal(np.diff(offs) > 0, np.asarray(N_f) > 0)
    ioffs, ifl = orc.inverted_index(g)
    assert int(ioffs[-1]) == int(offs[-1])  # one posting per (file, word) pair
    assert np.array_equal(np.diff(ioffs) > 0, wc > 0)
    sw, sc = orc.sort_words(g, 1)
    assert np.all(np.diff(sc.astype(np.int64)) <= 0)
    assert sorted(map(int, sw)) == list(map(int, np.nonzero(wc)[0]))
    k, cnt = orc.sequence_count(g, 0)
    assert int(cnt.astype(np.int64).sum()) == int(sum(max(n - 2, 0) for n in N_f))
    assert np.all(k[1:] > k[:-1])
    fr, kr, cr = orc.sequence_count(g, 1)
    assert int(cr.astype(np.int64).sum()) == int(cnt.astype(np.int64).sum())
    # TF-IDF: a word in every file scores 0; one in a single file scores
    # count * ln F; value / count is the same idf in every file of a word
    to, tw, tv = orc.tfidf(g)
    assert np.array_equal(to, offs) and np.array_equal(tw, w)
    F = len(N_f)
    df = np.bincount(w.astype(np.int64), minlength=g.num_words)
    ratio = tv / c.astype(np.float64)
    every = df[w] == F
    assert np.all(tv[every] == 0.0)
    single = df[w] == 1
    np.testing.assert_allclose(tv[single], c[single].astype(np.float64) * np.log(F), rtol=1e-15)
    first = np.full(g.num_words, np.nan)
    first[w[::-1]] = ratio[::-1]  # the idf seen in the word's first file
    np.testing.assert_allclose(ratio, first[w], rtol=1e-15)
    # co-occurrence: pairs at distance 1 and 2 inside files; equal to the
    # 3-word windows' (first, second) and (first, third) pairs plus the last
    # pair of every file of two or more words
    ck, cc = orc.cooccurrence(g)
    assert int(cc.astype(np.int64).sum()) == int(sum(max(n - 1, 0) + max(n - 2, 0) for n in N_f))
    m = np.uint64((1 << 21) - 1)
    a, b3, c3 = kr >> np.uint64(42), (kr >> np.uint64(21)) & m, kr & m
    files = orc.expand_files(g)
    tails = [((np.uint64(t[-2]) << np.uint64(21)) | np.uint64(t[-1])) for t in files if t.shape[0] >= 2]
    pk = np.concatenate([(a << np.uint64(21)) | b3, (a << np.uint64(21)) | c3, np.array(tails, np.uint64)])
    pc = np.concatenate([cr, cr, np.ones(len(tails), np.uint64)]).astype(np.int64)
    u, inv = np.unique(pk, return_inverse=True)
    assert np.array_equal(u, ck) and np.array_equal(np.bincount(inv, weights=pc).astype(np.int64),
                                                    cc.astype(np.int64))


def pin_eq1(orc, g):
    """Eq. 1 with l = 3 and wordSize read as the rule's own words: when every
    child expands to >= 2 words, rule r owns exactly W_r + 2 S_r - 2 windows
    (root: per file, floored at 0 for files shorter than three words)."""
    V = g.num_words
    L = orc.expansion_lengths(g)
    owned = orc.owned_windows(g)
    wt = orc.rule_weights(g).astype(np.int64)
    for r in range(g.num_rules):
        body = g.body(r).astype(np.int64)
        segs = [body] if r else [body[g.file_off[f]:g.file_off[f + 1]] for f in range(g.num_files)]
        if any((L[s - V] < 2) for s in body if s >= V):
            continue
        want = 0
        for seg in segs:
            W = int((seg < V).sum())
            S = int((seg >= V).sum())
            n_words = W + sum(int(L[s - V]) for s in seg if s >= V)
            want += (W + 2 * S - 2) if n_words >= 3 else 0
        assert int(owned[r]) == want, r
    k, cnt = orc.sequence_count(g, 0)
    assert int((wt * owned).sum()) == int(cnt.astype(np.int64).sum())


def outputs(orc, g):
    res = {"wc": orc.word_count(g), "sort0": orc.sort_words(g, 0), "sort1": orc.sort_words(g, 1),
           "tv": orc.term_vector(g, 0), "tv3": orc.term_vector(g, 3), "ii": orc.inverted_index(g),
           "seq": orc.sequence_count(g, 0), "seqf": orc.sequence_count(g, 1),
           "rank3": orc.ranked_index(g, 3), "rank1": orc.ranked_index(g, 1)}
    return res


def same_outputs(a, b):
    for k in a:
        x, y = a[k], b[k]
        xs = x if isinstance(x, tuple) else (x,)
        ys = y if isinstance(y, tuple) else (y,)
        assert len(xs) == len(ys), k
        for u, v in zip(xs, ys):
            assert np.array_equal(np.asarray(u), np.asarray(v)), k


# ---------------------------------------------------------------------------
# Tests
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name,g,toks,lens", CASES, ids=[c[0] for c in CASES])
def test_oracle_matches_brute_force(name, g, toks, lens):
    pin_brute(oracle, g)
    if toks is not None:
        pin_source(oracle, g, toks, lens)


def test_oracle_matches_brute_force_at_the_largest_vocabulary():
    """num_words = 2^21, the most a 21-bit field of a 3-word key holds: word
    IDs at both ends of the range, so a key packing that loses the top bit or
    mixes fields shows in the sequence count and the ranked index."""
    V = 1 << 21
    rng = np.random.default_rng(2021)
    pool = np.array([0, 1, 2, 1 << 20, V - 3, V - 2, V - 1], np.int32)
    toks = pool[rng.integers(0, pool.size, size=300)]
    toks[100:108] = toks[10:18]  # a repeated phrase gives nested rules
    lens = np.array([120, 0, 180], np.int64)
    g = sequitur(toks, lens, V)
    assert g.num_words == V and toks.max() == V - 1
    pin_brute(oracle, g)
    pin_source(oracle, g, toks, lens)


@pytest.mark.parametrize("name,g,toks,lens", [c for c in CASES if c[0].startswith("seq")][:25],
                         ids=[c[0] for c in CASES if c[0].startswith("seq")][:25])
def test_eq1_owned_windows(name, g, toks, lens):
    pin_eq1(oracle, g)


@pytest.fixture(scope="module")
def corpus_200k():
    c = make_corpus("wc_single_200k")
    g = sequitur(c.tokens, c.file_lens, c.num_words)
    return c, g


@pytest.fixture(scope="module")
def corpus_multi():
    c = make_corpus("multi64_50m", scale=0.002)  # 64 files, ~100k tokens
    g = sequitur(c.tokens, c.file_lens, c.num_words)
    return c, g


def test_expansion_equals_source_200k(corpus_200k):
    c, g = corpus_200k
    pin_source(oracle, g, c.tokens, c.file_lens)


def test_closed_forms_200k(corpus_200k):
    c, g = corpus_200k
    pin_closed_forms(oracle, g, list(c.file_lens))
    wt = oracle.rule_weights(g)
    assert int(wt[0]) == 1 and np.all(wt[1:] >= 2)  # rule utility: every rule used twice or more


def test_closed_forms_multifile(corpus_multi):
    c, g = corpus_multi
    assert g.num_files == 64
    pin_source(oracle, g, c.tokens, c.file_lens)
    pin_closed_forms(oracle, g, list(c.file_lens))


def test_grammar_independence(corpus_multi):
    c, g = corpus_multi
    rng = np.random.default_rng(3)
    a = outputs(oracle, g)
    same_outputs(a, outputs(oracle, root_only_grammar(c.tokens, c.file_lens, c.num_words)))
    same_outputs(a, outputs(oracle, refactor_grammar(g, rng, rounds=2, frac=0.15)))


def test_root_only_reduces_to_textbook(corpus_200k):
    c, _ = corpus_200k
    g = root_only_grammar(c.tokens, c.file_lens, c.num_words)
    assert np.array_equal(oracle.word_count(g), np.bincount(c.tokens, minlength=c.num_words).astype(np.uint64))
    t = c.tokens.astype(np.uint64)
    keys = (t[:-2] << np.uint64(42)) | (t[1:-1] << np.uint64(21)) | t[2:]
    k, n = np.unique(keys, return_counts=True)
    ok, oc = oracle.sequence_count(g, 0)
    assert np.array_equal(ok, k) and np.array_equal(oc, n.astype(np.uint64))
    assert int(oracle.rule_weights(g)[0]) == 1


def test_repeated_passage_scales_counts():
    rng = np.random.default_rng(11)
    p = rng.integers(0, 50, size=300).astype(np.int32)
    for k in (1, 2, 5):
        toks = np.tile(p, k)
        g = sequitur(toks, [toks.size], 50)
        assert np.array_equal(oracle.word_count(g).astype(np.int64),
                              k * np.bincount(p, minlength=50))


def test_single_file_inverted_index_trivial(corpus_200k):
    c, g = corpus_200k
    offs, fl = oracle.inverted_index(g)
    assert np.all(fl == 0)
    assert np.array_equal(np.diff(offs), (oracle.word_count(g) > 0).astype(np.int64))


def test_golden_headtail_section4c():
    fx = json.loads((GOLDEN / "headtail_section4c.json").read_text())
    g = grammar_from_rules(fx["num_words"], fx["rules"], fx["file_off"])
    h, t = oracle.head_tail(g)
    assert list(map(int, h[1])) == fx["expect"]["head_R1"]
    assert list(map(int, t[1])) == fx["expect"]["tail_R1"]
    keys, _ = oracle.sequence_count(g, 0)
    for name in ("window_inside_root", "window_cross_root_R1"):
        k = int(oracle.pack3(*fx["expect"][name]))
        assert k in set(map(int, keys)), name
    # the cross-rule window belongs to the parent: the root owns it, R1 does not
    owned = oracle.owned_windows(g)
    assert int(owned[1]) == 2  # R1 only owns windows inside w4..w7
    assert int(owned[0]) == 4  # the root owns <w1,w2,w3>, <w2,w3,w4>, <w3,w4,w5>, <w6,w7,w8>


def test_golden_wordcount_flow_section2a():
    """Fig. 2's bottom-up flow (R2 -> R0, R1; R1 -> R0; R0 merges) computed by
    hand-written table merging equals the oracle's direct count."""
    fx = json.loads((GOLDEN / "wordcount_section2a.json").read_text())
    V = fx["num_words"]
    g = grammar_from_rules(V, fx["rules"], fx["file_off"])
    parents = {}
    for r, body in enumerate(fx["rules"]):
        for s in body:
            if s >= V:
                parents.setdefault(str(s - V), set()).add(r)
    assert {k: sorted(v) for k, v in parents.items()} == fx["expect"]["parents"]

    def local(r):
        t = [0] * V
        for s in fx["rules"][r]:
            if s < V:
                t[s] += 1
        return t

    def merge(dst, src, m):
        return [a + m * b for a, b in zip(dst, src)]

    def mult(p, c):
        return sum(1 for s in fx["rules"][p] if s == V + c)

    t2 = local(2)                                   # step 1: R2's table
    t1 = merge(local(1), t2, mult(1, 2))            # step 2: R1 merges R2
    t0 = merge(merge(local(0), t1, mult(0, 1)), t2, mult(0, 2))  # step 3: R0 merges both
    assert list(map(int, oracle.word_count(g))) == t0


# ---------------------------------------------------------------------------
# Planted mistakes: each broken copy of the oracle must fail some pin.
# ---------------------------------------------------------------------------

def broken_oracle(patch):
    m = types.ModuleType("broken_oracle")
    m.__dict__.update({k: v for k, v in vars(orc_impl).items() if not k.startswith("__")})
    patch(m)
    # re-bind the module globals used by the functions to the patched copy
    for k, v in list(vars(m).items()):
        if isinstance(v, types.FunctionType) and v.__module__ == orc_impl.__name__:
            setattr(m, k, types.FunctionType(v.__code__, m.__dict__, v.__name__, v.__defaults__, v.__closure__))
    return m


def _fails(check):
    try:
        check()
    except (AssertionError, IndexError, ValueError):
        return True
    return False


def _pins(m):
    cases = [c for c in CASES[:30]]
    for name, g, toks, lens in cases:
        pin_brute(m, g)
        if toks is not None:
            pin_source(m, g, toks, lens)
            pin_closed_forms(m, g, list(lens))
            if name.startswith("seq"):
                pin_eq1(m, g)


def test_planted_dropped_last_symbol():
    def patch(m):
        orig = orc_impl.expand_files
        m.expand_files = lambda g: [f[:-1] if f.size else f for f in orig(g)]
    assert _fails(lambda: _pins(broken_oracle(patch)))


def test_planted_windows_cross_files():
    def patch(m):
        def seq(g, per_file=0):
            toks = np.concatenate(orc_impl.expand_files(g))
            k, c = np.unique(orc_impl.file_windows(toks), return_counts=True)
            if per_file:
                return np.zeros(k.shape[0], np.int32), k, c.astype(np.uint64)
            return k, c.astype(np.uint64)
        m.sequence_count = seq
    assert _fails(lambda: _pins(broken_oracle(patch)))


def test_planted_wrong_tie_order():
    def patch(m):
        def sort_words(g, order=0):
            w, c = orc_impl.sort_words(g, 0)
            if order == 1:
                idx = np.lexsort((-w.astype(np.int64), -c.astype(np.int64)))
                w, c = w[idx], c[idx]
            return w, c
        m.sort_words = sort_words
    assert _fails(lambda: _pins(broken_oracle(patch)))


def test_planted_weight_misses_root_edges():
    def patch(m):
        def rule_weights(g):
            wt = orc_impl.rule_weights(g).astype(np.int64)
            V = g.num_words
            root = g.body(0)
            direct = np.bincount(root[root >= V] - V, minlength=g.num_rules)
            wt[1:] -= direct[1:]
            return wt.astype(np.uint64)
        m.rule_weights = rule_weights
    assert _fails(lambda: _pins(broken_oracle(patch)))


def test_planted_swapped_key_fields():
    def patch(m):
        m.pack3 = lambda a, b, c: orc_impl.pack3(c, b, a)
    assert _fails(lambda: _pins(broken_oracle(patch)))


@pytest.mark.parametrize("n", [1, 3])
def test_key_file_counts_match_ranked_index(n):
    """key_file_counts_text (the ranked rows of chosen keys, used for sampled
    checks at full size) equals the ranked index restricted to those keys,
    and is computed from the source text rather than the grammar."""
    rng = np.random.default_rng(11)
    checked = 0
    for name, g, toks, lens in tiny_cases(seed=13, count=12):
        if toks is None or g.num_words > (1 << 21):
            continue
        offs, keys, files, counts = oracle.ranked_index(g, n)
        if keys.shape[0] == 0:
            continue
        pick = rng.choice(keys, size=min(5, keys.shape[0]), replace=False)
        pick = np.append(pick, np.uint64((1 << 63) - 1))  # a key that never occurs
        k, f, c = oracle.key_file_counts_text(split_files(toks, lens), pick, n)
        want_k, want_f, want_c = [], [], []
        for key in np.sort(pick):
            i = np.searchsorted(keys, key)
            if i < keys.shape[0] and keys[i] == key:
                a, b = offs[i], offs[i + 1]
                want_k.append(np.full(b - a, key, np.uint64))
                want_f.append(files[a:b])
                want_c.append(counts[a:b])
        assert np.array_equal(k, np.concatenate(want_k)), name
        assert np.array_equal(f, np.concatenate(want_f)), name
        assert np.array_equal(c, np.concatenate(want_c)), name
        checked += 1
    assert checked >= 5


def test_planted_idf_inverted():
    def patch(m):
        def tfidf_text(files):
            offs, words, counts = m.term_vector_text(files)
            df = np.bincount(words.astype(np.int64))
            return offs, words, counts * np.log(df[words] / np.float64(len(files)))
        m.tfidf_text = tfidf_text
    assert _fails(lambda: _pins(broken_oracle(patch)))


def test_planted_cooccurrence_misses_distance_two():
    def patch(m):
        def cooccurrence_text(files):
            keys = [(np.asarray(t[:-1], np.uint64) << np.uint64(21)) | np.asarray(t[1:], np.uint64)
                    for t in files if len(t) > 1]
            k = np.concatenate(keys) if keys else np.zeros(0, np.uint64)
            u, c = np.unique(k, return_counts=True)
            return u, c.astype(np.uint64)
        m.cooccurrence_text = cooccurrence_text
    assert _fails(lambda: _pins(broken_oracle(patch)))


def test_planted_cooccurrence_across_files():
    def patch(m):
        orig = m.cooccurrence_text
        m.cooccurrence_text = lambda files: orig([np.concatenate(files)] if len(files) else files)
    assert _fails(lambda: _pins(broken_oracle(patch)))
