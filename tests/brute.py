"""Brute-force reference for tiny grammars: recursive expansion in plain
Python lists and dict counting.  It shares nothing with ``oracle/`` (which
expands level by level with numpy and counts with sort-based primitives), so
the two agreeing on many random grammars pins the oracle."""
from collections import Counter, defaultdict


def bodies(g):
    return [[int(x) for x in g.sym[g.rule_off[r]:g.rule_off[r + 1]]] for r in range(g.num_rules)]


def expand_files(g):
    V = g.num_words
    B = bodies(g)
    memo = {}

    def ex(r):
        if r not in memo:
            out = []
            for s in B[r]:
                out.extend([s] if s < V else ex(s - V))
            memo[r] = out
        return memo[r]

    root = B[0]
    files = []
    for f in range(g.num_files):
        seg = root[int(g.file_off[f]):int(g.file_off[f + 1])]
        out = []
        for s in seg:
            out.extend([s] if s < V else ex(s - V))
        files.append(out)
    return files, ex


def word_count(g):
    files, _ = expand_files(g)
    c = Counter(t for f in files for t in f)
    return [c.get(w, 0) for w in range(g.num_words)]


def sort_words(g, order):
    wc = word_count(g)
    items = [(w, c) for w, c in enumerate(wc) if c > 0]
    if order == 1:
        items.sort(key=lambda x: (-x[1], x[0]))
    return items


def term_vector(g, top_k=0):
    files, _ = expand_files(g)
    out = []
    for toks in files:
        items = sorted(Counter(toks).items())
        if top_k:
            items = sorted(items, key=lambda x: (-x[1], x[0]))[:top_k]
        out.append(items)
    return out


def inverted_index(g):
    files, _ = expand_files(g)
    ii = defaultdict(list)
    for f, toks in enumerate(files):
        for w in sorted(set(toks)):
            ii[w].append(f)
    return [ii.get(w, []) for w in range(g.num_words)]


def key3(a, b, c):
    return (a << 42) | (b << 21) | c


def windows(toks):
    return [key3(toks[i], toks[i + 1], toks[i + 2]) for i in range(len(toks) - 2)]


def sequence_count(g, per_file=0):
    files, _ = expand_files(g)
    if not per_file:
        c = Counter(k for t in files for k in windows(t))
        return sorted(c.items())
    out = []
    for f, t in enumerate(files):
        for k, n in sorted(Counter(windows(t)).items()):
            out.append((f, k, n))
    return out


def ranked_index(g, n=3):
    files, _ = expand_files(g)
    per = defaultdict(dict)
    for f, t in enumerate(files):
        for k, c in Counter(windows(t) if n == 3 else t).items():
            per[k][f] = c
    return [(k, sorted(per[k].items(), key=lambda x: (-x[1], x[0]))) for k in sorted(per)]


def rule_weights(g):
    """Walk the derivation tree from the root, counting every rule visit."""
    V = g.num_words
    B = bodies(g)
    wt = [0] * g.num_rules
    wt[0] = 1
    stack = [s - V for s in B[0] if s >= V]
    while stack:
        r = stack.pop()
        wt[r] += 1
        stack.extend(s - V for s in B[r] if s >= V)
    return wt


def head_tail(g):
    _, ex = expand_files(g)
    V = g.num_words
    B = bodies(g)
    heads, tails = [], []
    for r in range(g.num_rules):
        e = []
        for s in B[r]:
            e.extend([s] if s < V else ex(s - V))
        heads.append((e[0] if len(e) > 0 else -1, e[1] if len(e) > 1 else -1))
        tails.append((e[-2] if len(e) > 1 else -1, e[-1] if len(e) > 0 else -1))
    return heads, tails


def owned_windows(g):
    """Windows of each rule's expansion that touch two or more body symbols."""
    _, ex = expand_files(g)
    V = g.num_words
    B = bodies(g)
    out = []
    for r in range(g.num_rules):
        segs = [B[r]] if r else [B[0][int(g.file_off[f]):int(g.file_off[f + 1])] for f in range(g.num_files)]
        n = 0
        for seg in segs:
            src = []
            for i, s in enumerate(seg):
                src.extend([i] * (1 if s < V else len(ex(s - V))))
            n += sum(1 for j in range(len(src) - 2) if src[j] != src[j + 2])
        out.append(n)
    return out


def tfidf(g):
    """Per file: (word, count * ln(F / df)) for its words, ascending word."""
    import math
    files, _ = expand_files(g)
    F = len(files)
    df = Counter(w for toks in files for w in set(toks))
    return [[(w, c * math.log(F / df[w])) for w, c in sorted(Counter(toks).items())] for toks in files]


def cooccurrence(g):
    files, _ = expand_files(g)
    c = Counter()
    for t in files:
        for i in range(len(t)):
            for j in (i + 1, i + 2):
                if j < len(t):
                    c[(t[i] << 21) | t[j]] += 1
    return sorted(c.items())
