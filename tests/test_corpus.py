"""The input generator: Sequitur output must expand to its input and keep
Sequitur's invariants (digram uniqueness, rule utility); recipes are seeded."""
import numpy as np
import pytest

from paper_2106_06889_gb300.corpus import sequitur, make_corpus, Grammar
import oracle
from tests import brute


def sequitur_invariants(g: Grammar):
    """(#repeated digrams, #rules used < 2 times, #references to the root)."""
    V = g.num_words
    uses = np.zeros(g.num_rules, np.int64)
    occ = {}
    for r in range(g.num_rules):
        b = g.body(r)
        segs = [b] if r else [b[g.file_off[f]:g.file_off[f + 1]] for f in range(g.num_files)]
        for si, seg in enumerate(segs):
            for i, s in enumerate(seg):
                if s >= V:
                    uses[s - V] += 1
                if i + 1 < len(seg):
                    occ.setdefault((int(seg[i]), int(seg[i + 1])), []).append((r, si, i))
    repeated = 0
    for k, o in occ.items():
        if len(o) >= 3:
            repeated += 1
        elif len(o) == 2:
            (r1, s1, i1), (r2, s2, i2) = o
            if not (r1 == r2 and s1 == s2 and abs(i1 - i2) == 1):  # overlapping "x x x" is allowed
                repeated += 1
    return repeated, int((uses[1:] < 2).sum()), int(uses[0])


@pytest.mark.parametrize("seed", range(60))
def test_sequitur_random_streams(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(0, 400))
    V = int(rng.integers(1, 8))
    F = int(rng.integers(1, 5))
    toks = rng.integers(0, V, size=n).astype(np.int32)
    cuts = np.sort(rng.integers(0, n + 1, size=F - 1))
    lens = np.diff(np.concatenate([[0], cuts, [n]]))
    g = sequitur(toks, lens, V)
    files, _ = brute.expand_files(g)
    offs = np.concatenate([[0], np.cumsum(lens)])
    assert files == [list(map(int, toks[offs[f]:offs[f + 1]])) for f in range(F)]
    assert sequitur_invariants(g) == (0, 0, 0)
    assert np.all(np.diff(g.rule_off)[1:] >= 2)  # every rule body has two or more symbols


def test_sequitur_200k_invariants():
    c = make_corpus("wc_single_200k")
    assert c.tokens.shape[0] == 200_000
    g = sequitur(c.tokens, c.file_lens, c.num_words)
    assert sequitur_invariants(g) == (0, 0, 0)
    assert g.num_syms < 200_000  # it does compress


def test_recipes_are_seeded():
    a = make_corpus("multi64_50m", scale=0.001)
    b = make_corpus("multi64_50m", scale=0.001)
    assert np.array_equal(a.tokens, b.tokens) and np.array_equal(a.file_lens, b.file_lens)
    assert a.file_lens.shape[0] == 64
    assert a.tokens.max() < 500_000


def test_sequitur_rejects_bad_input():
    with pytest.raises(ValueError):
        sequitur(np.array([0, 5], np.int32), [2], 3)  # word id out of range
    with pytest.raises(ValueError):
        sequitur(np.array([0, 1], np.int32), [3], 3)  # lengths do not add up


@pytest.mark.parametrize("name,scale", [("nested_500m", 0.001), ("files100k", 0.001), ("files_short", 0.01),
                                        ("multi64_50m", 0.004)])
@pytest.mark.parametrize("shards", [1, 3, 7])
def test_sharded_sequitur_expands_to_source(name, scale, shards):
    """The shard-parallel build used for the largest corpora encodes the same
    text: expansion equals the source, file by file."""
    from paper_2106_06889_gb300.corpus import sequitur_sharded
    c = make_corpus(name, scale=scale)
    g = sequitur_sharded(c.tokens, c.file_lens, c.num_words, shards)
    files = oracle.expand_files(g)
    assert g.num_files == c.file_lens.shape[0]
    assert [len(f) for f in files] == list(c.file_lens)
    assert np.array_equal(np.concatenate(files), c.tokens)
