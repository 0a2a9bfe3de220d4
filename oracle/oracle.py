"""CPU oracle for text analytics on a TADOC grammar (G-TADOC, arXiv 2106.06889).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
module.  The engine never calls it, and it shares no code with the engine.

Every analytic the paper runs (Section VI: word count, sort, inverted index,
term vector, sequence count, ranked inverted index) is a function of the
token stream of each file; the grammar is only a lossless encoding of that
stream (Section II-A).  So this oracle is the plain definition written out:

1. expand the root back into one token array per file, by substituting every
   rule reference with its body until only words are left;
2. compute each analytic directly on those arrays with library primitives
   (``np.bincount``, ``np.unique``, ``np.lexsort``).

No traversal, no blocking, no reuse of partial results: it is slow on purpose
and meant to be checked against the paper by eye.  Integer results are exact
(int64/uint64).  The readings taken where the paper is silent are:

* word count is global over all files (in the word-count example of Section
  II-A the counts of the whole input end up at the root);
* a 3-word sequence never spans two files (the splitters between files are
  unique symbols and belong to no window);
* 3-word keys pack as ``w1 << 42 | w2 << 21 | w3``;
* sort order 0 is ascending word ID, order 1 is descending count then
  ascending word ID;
* term vector top-k keeps the k largest counts by descending count then
  ascending word ID;
* the ranked inverted index lists, per key, the files with their in-file
  counts by descending count then ascending file.

``rule_weights``, ``head_tail``, ``expansion_lengths`` and ``owned_windows``
give the per-rule quantities the paper's traversals build (Algorithm 1's
accumulated weights, Section IV-C's head/tail buffers, Eq. 1's window bound),
each from its own plain definition.
"""
from __future__ import annotations

import numpy as np

KEY_BITS = 21  # bits per word in a packed 3-word key


# ---------------------------------------------------------------------------
# Expansion (Section II-A: the grammar is a lossless encoding of the files)
# ---------------------------------------------------------------------------

def _substitute_once(g, seq: np.ndarray):
    """Replace every rule reference in ``seq`` by its body (one level).

    Returns the new sequence and, for each element of it, the index of the
    element of ``seq`` it came from.
    """
    V = g.num_words
    is_rule = seq >= V
    rid = np.where(is_rule, seq - V, 0)
    lens = np.where(is_rule, g.rule_off[rid + 1] - g.rule_off[rid], 1).astype(np.int64)
    src = np.repeat(np.arange(seq.shape[0], dtype=np.int64), lens)
    # position of each output element within its source element
    starts = np.cumsum(lens) - lens
    within = np.arange(src.shape[0], dtype=np.int64) - starts[src]
    out = np.where(is_rule[src], g.sym[g.rule_off[rid[src]] + within] if src.size else seq[src], seq[src])
    return out.astype(np.int64), src


def expand_sequence(g, seq) -> np.ndarray:
    """Fully expand a sequence of symbols into words."""
    seq = np.asarray(seq, dtype=np.int64)
    for _ in range(g.num_rules + 1):
        if not (seq >= g.num_words).any():
            return seq
        seq, _ = _substitute_once(g, seq)
    raise ValueError("grammar is cyclic")


def expand_files(g) -> list[np.ndarray]:
    """Token array of every file: expand root body segment file_off[f]:file_off[f+1]."""
    root = g.sym[g.rule_off[0]:g.rule_off[1]].astype(np.int64)
    return [expand_sequence(g, root[g.file_off[f]:g.file_off[f + 1]]) for f in range(g.num_files)]


def expand_rule(g, r: int) -> np.ndarray:
    return expand_sequence(g, g.sym[g.rule_off[r]:g.rule_off[r + 1]])


# ---------------------------------------------------------------------------
# Per-rule quantities built by the paper's traversals
# ---------------------------------------------------------------------------

def rule_weights(g) -> np.ndarray:
    """wt[r] = number of occurrences of rule r in the full derivation.

    This is what Algorithm 1 accumulates top-down (a rule's weight is the sum
    over its parents of parent weight times frequency, the root having weight
    one).  Here it is counted directly: while the root is expanded one level
    at a time, every rule reference met is one occurrence.
    """
    V = g.num_words
    wt = np.zeros(g.num_rules, dtype=np.int64)
    wt[0] = 1
    seq = g.sym[g.rule_off[0]:g.rule_off[1]].astype(np.int64)
    for _ in range(g.num_rules + 1):
        refs = seq[seq >= V] - V
        if refs.size == 0:
            return wt.astype(np.uint64)
        wt += np.bincount(refs, minlength=g.num_rules)
        seq, _ = _substitute_once(g, seq)
    raise ValueError("grammar is cyclic")


def expansion_lengths(g) -> np.ndarray:
    """L[r] = number of words in the expansion of rule r."""
    return np.array([expand_rule(g, r).shape[0] for r in range(g.num_rules)], dtype=np.int64)


def head_tail(g):
    """Head and tail buffers (Section IV-C, Fig. 6): first two and last two
    words of each rule's expansion; -1 pads an expansion of one word."""
    head = np.full((g.num_rules, 2), -1, dtype=np.int64)
    tail = np.full((g.num_rules, 2), -1, dtype=np.int64)
    for r in range(g.num_rules):
        e = expand_rule(g, r)
        k = min(2, e.shape[0])
        head[r, :k] = e[:k]          # (first, second or -1)
        tail[r, 2 - k:] = e[e.shape[0] - k:]  # (second-to-last or -1, last)
    return head.astype(np.int32), tail.astype(np.int32)


def owned_windows(g) -> np.ndarray:
    """Per rule, the 3-word windows of its expansion that are not wholly
    inside the expansion of one body symbol (those a parent must handle
    itself, the cross-rule sequences of Section III-B)."""
    out = np.zeros(g.num_rules, dtype=np.int64)
    V = g.num_words
    for r in range(g.num_rules):
        body = g.sym[g.rule_off[r]:g.rule_off[r + 1]].astype(np.int64)
        segs = [body] if r else [body[g.file_off[f]:g.file_off[f + 1]] for f in range(g.num_files)]
        for seg in segs:
            # which body symbol each word of the expansion came from
            src = np.concatenate([np.full(expand_sequence(g, [s]).shape[0], i, dtype=np.int64)
                                  for i, s in enumerate(seg)]) if seg.size else np.zeros(0, np.int64)
            if src.shape[0] >= 3:
                out[r] += int((src[:-2] != src[2:]).sum())
    return out


# ---------------------------------------------------------------------------
# The six analytics (Section VI)
# ---------------------------------------------------------------------------

# Each analytic is defined on the token arrays of the files (``*_text``); the
# grammar versions apply that definition to the grammar's expansion.

def word_count_text(files, num_words: int) -> np.ndarray:
    toks = np.concatenate(files) if len(files) else np.zeros(0, np.int64)
    return np.bincount(toks, minlength=num_words).astype(np.uint64)


def word_count(g) -> np.ndarray:
    return word_count_text(expand_files(g), g.num_words)


def sort_words_text(files, num_words: int, order: int = 0):
    """(word, count) of every word that occurs; order 0 by word, 1 by count desc."""
    cnt = word_count_text(files, num_words).astype(np.int64)
    words = np.nonzero(cnt)[0]
    counts = cnt[words]
    if order == 1:
        idx = np.lexsort((words, -counts))
        words, counts = words[idx], counts[idx]
    return words.astype(np.int32), counts.astype(np.uint64)


def sort_words(g, order: int = 0):
    return sort_words_text(expand_files(g), g.num_words, order)


def term_vector_text(files, top_k: int = 0):
    """Per file: distinct words with in-file counts (CSR over files)."""
    offs, words, counts = [0], [], []
    for toks in files:
        w, c = np.unique(toks, return_counts=True)
        if top_k > 0:
            idx = np.lexsort((w, -c))[:top_k]
            w, c = w[idx], c[idx]
        words.append(w)
        counts.append(c)
        offs.append(offs[-1] + w.shape[0])
    cat = (lambda xs, dt: np.concatenate(xs).astype(dt) if xs else np.zeros(0, dt))
    return np.array(offs, np.int64), cat(words, np.int32), cat(counts, np.uint64)


def term_vector(g, top_k: int = 0):
    return term_vector_text(expand_files(g), top_k)


def inverted_index_text(files, num_words: int):
    """Per word: ascending list of files containing it (CSR over words)."""
    pairs_w, pairs_f = [], []
    for f, toks in enumerate(files):
        w = np.unique(toks)
        pairs_w.append(w)
        pairs_f.append(np.full(w.shape[0], f, np.int64))
    w = np.concatenate(pairs_w) if pairs_w else np.zeros(0, np.int64)
    f = np.concatenate(pairs_f) if pairs_f else np.zeros(0, np.int64)
    idx = np.lexsort((f, w))
    w, f = w[idx], f[idx]
    offs = np.zeros(num_words + 1, np.int64)
    offs[1:] = np.cumsum(np.bincount(w, minlength=num_words))
    return offs, f.astype(np.int32)


def inverted_index(g):
    return inverted_index_text(expand_files(g), g.num_words)


def pack3(a, b, c) -> np.ndarray:
    a, b, c = (np.asarray(x, dtype=np.uint64) for x in (a, b, c))
    return (a << np.uint64(2 * KEY_BITS)) | (b << np.uint64(KEY_BITS)) | c


def file_windows(toks: np.ndarray) -> np.ndarray:
    """Packed keys of every window of three consecutive words of one file."""
    if toks.shape[0] < 3:
        return np.zeros(0, np.uint64)
    return pack3(toks[:-2], toks[1:-1], toks[2:])


def sequence_count_text(files, num_words: int, per_file: int = 0):
    """Counts of 3-word sequences (Section IV-D, l = 3), windows inside files only."""
    if num_words > (1 << KEY_BITS):
        raise ValueError("3-word keys need num_words <= 2^21")
    if not per_file:
        keys = np.concatenate([file_windows(t) for t in files]) if len(files) else np.zeros(0, np.uint64)
        k, c = np.unique(keys, return_counts=True)
        return k.astype(np.uint64), c.astype(np.uint64)
    fs, ks, cs = [], [], []
    for f, t in enumerate(files):
        k, c = np.unique(file_windows(t), return_counts=True)
        fs.append(np.full(k.shape[0], f, np.int32))
        ks.append(k)
        cs.append(c)
    cat = (lambda xs, dt: np.concatenate(xs).astype(dt) if xs else np.zeros(0, dt))
    return cat(fs, np.int32), cat(ks, np.uint64), cat(cs, np.uint64)


def sequence_count(g, per_file: int = 0):
    return sequence_count_text(expand_files(g), g.num_words, per_file)


def key_file_counts_text(files, keys, n: int = 3):
    """For the given keys (words if n = 1, packed 3-word keys if n = 3): every
    (key, file, count) with count = occurrences of the key in the file > 0,
    in ranked order (key asc, count desc, file asc).  The rows of the ranked
    inverted index restricted to those keys."""
    keys = np.unique(np.asarray(keys, dtype=np.uint64))
    ks, fs = [], []
    for f, t in enumerate(files):
        items = t.astype(np.uint64) if n == 1 else file_windows(t)
        hit = items[np.isin(items, keys)]
        ks.append(hit)
        fs.append(np.full(hit.shape[0], f, np.int64))
    k = np.concatenate(ks) if ks else np.zeros(0, np.uint64)
    f = np.concatenate(fs) if fs else np.zeros(0, np.int64)
    pairs = np.stack([k.astype(np.int64), f], axis=1) if k.shape[0] else np.zeros((0, 2), np.int64)
    if pairs.shape[0]:
        u, c = np.unique(pairs, axis=0, return_counts=True)
    else:
        u, c = pairs, np.zeros(0, np.int64)
    kk, ff = u[:, 0].astype(np.uint64), u[:, 1]
    idx = np.lexsort((ff, -c, kk))
    return kk[idx], ff[idx].astype(np.int32), c[idx].astype(np.uint64)


def ranked_index(g, n: int = 3):
    """Per key (ascending): files with in-file counts, count desc then file asc."""
    if n == 3:
        f, k, c = sequence_count(g, per_file=1)
    elif n == 1:
        offs, w, cnt = term_vector(g)
        f = np.repeat(np.arange(g.num_files, dtype=np.int32), np.diff(offs))
        k, c = w.astype(np.uint64), cnt
    else:
        raise ValueError("n must be 1 or 3")
    idx = np.lexsort((f, -c.astype(np.int64), k))
    f, k, c = f[idx], k[idx], c[idx]
    keys, first = np.unique(k, return_index=True)
    offs = np.append(first, k.shape[0]).astype(np.int64)
    return offs, keys.astype(np.uint64), f.astype(np.int32), c.astype(np.uint64)


# ---------------------------------------------------------------------------
# Advanced analytics on the same traversal (the Introduction and Related Work
# name TF-IDF and word co-occurrence as the analytics that build on these)
# ---------------------------------------------------------------------------

def tfidf_text(files):
    """TF-IDF per file: for every word w of file f, tf = its in-file count and
    idf = ln(F / df(w)), df(w) = the number of files containing w (F = number
    of files).  CSR over files, words ascending, values float64 = tf * idf.
    (Reading: raw counts for tf and the natural log for idf, no smoothing.)"""
    offs, words, counts = term_vector_text(files)
    F = len(files)
    df = np.bincount(words.astype(np.int64), minlength=int(words.max()) + 1 if words.size else 0)
    idf = np.log(np.float64(F) / df[words.astype(np.int64)].astype(np.float64)) if words.size else np.zeros(0)
    return offs, words, counts.astype(np.float64) * idf


def tfidf(g):
    return tfidf_text(expand_files(g))


def cooccurrence_text(files):
    """Word co-occurrence within a window of three words: the ordered pairs
    (t[i], t[j]) with j - i in {1, 2} inside one file, counted.  Keys pack as
    a << 21 | b, ascending; counts uint64."""
    keys = []
    for t in files:
        t = np.asarray(t, dtype=np.uint64)
        for d in (1, 2):
            if t.shape[0] > d:
                keys.append((t[:-d] << np.uint64(KEY_BITS)) | t[d:])
    k = np.concatenate(keys) if keys else np.zeros(0, np.uint64)
    u, c = np.unique(k, return_counts=True)
    return u.astype(np.uint64), c.astype(np.uint64)


def cooccurrence(g):
    return cooccurrence_text(expand_files(g))
