"""Seeded synthetic corpora and their TADOC compressed form.

This module prepares inputs only.  It draws Zipf-distributed word-ID streams
with injected repeated passages (stand-ins for the paper's datasets A-E of
Section V-A, which are not available here) and compresses them with the
Sequitur compressor in ``sequitur.cpp`` into the rule-grammar form of
Section II-A: a root rule holding every file with unique splitters between
files, plus one rule per repeated phrase.

It contains none of the analytics: both the CUDA engine and the CPU oracle
consume the :class:`Grammar` it returns.
"""
from __future__ import annotations

import ctypes
import hashlib
import json
import os
import threading
from dataclasses import dataclass, field
from pathlib import Path

import numpy as np

from .._build import build_corpus, CORPUS_SO, ROOT

__all__ = ["Grammar", "sequitur", "zipf_tokens", "Corpus", "make_corpus", "CONFIGS", "load_config",
           "root_only_grammar", "refactor_grammar", "prefix_files", "file_range", "root_prefix",
           "serving_corpus", "load_serving",
           "load_serving_set"]


@dataclass
class Grammar:
    """A compressed corpus.

    ``sym`` holds every rule body back to back (``rule_off[r]:rule_off[r+1]``);
    rule 0 is the root, whose body is all files concatenated without
    splitters, file ``f`` being ``file_off[f]:file_off[f+1]`` of that body.
    A symbol ``s < num_words`` is a word; ``s >= num_words`` refers to rule
    ``s - num_words``.
    """

    num_words: int
    rule_off: np.ndarray  # int64 [R+1]
    sym: np.ndarray  # int32 [G]
    file_off: np.ndarray  # int64 [F+1]
    meta: dict = field(default_factory=dict)

    @property
    def num_rules(self) -> int:
        return int(self.rule_off.shape[0] - 1)

    @property
    def num_files(self) -> int:
        return int(self.file_off.shape[0] - 1)

    @property
    def num_syms(self) -> int:
        return int(self.sym.shape[0])

    def body(self, r: int) -> np.ndarray:
        return self.sym[self.rule_off[r]:self.rule_off[r + 1]]

    def save(self, path: Path) -> None:
        np.savez(path, num_words=np.int64(self.num_words), rule_off=self.rule_off, sym=self.sym,
                 file_off=self.file_off, meta=np.array(json.dumps(self.meta)))

    @staticmethod
    def load(path: Path) -> "Grammar":
        z = np.load(path)
        return Grammar(int(z["num_words"]), z["rule_off"], z["sym"], z["file_off"], json.loads(str(z["meta"])))


_lib = None
_lib_lock = threading.Lock()  # sequitur_sharded's threads may load it at once


def _corpus_lib():
    global _lib
    with _lib_lock:
        if _lib is not None:
            return _lib
        so = build_corpus()
        lib = ctypes.CDLL(str(so))
        lib.gtc_sequitur_build.restype = ctypes.c_void_p
        lib.gtc_sequitur_build.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                           ctypes.c_void_p]
        lib.gtc_grammar_sizes.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64),
                                          ctypes.POINTER(ctypes.c_int64)]
        lib.gtc_grammar_export.argtypes = [ctypes.c_void_p] * 4
        lib.gtc_grammar_free.argtypes = [ctypes.c_void_p]
        _lib = lib
    return _lib


def sequitur(tokens: np.ndarray, file_lens, num_words: int) -> Grammar:
    """Compress ``tokens`` (the files back to back) into a Sequitur grammar."""
    tokens = np.ascontiguousarray(tokens, dtype=np.int32)
    file_lens = np.ascontiguousarray(file_lens, dtype=np.int64)
    lib = _corpus_lib()
    h = lib.gtc_sequitur_build(tokens.ctypes.data, tokens.shape[0], num_words, file_lens.shape[0],
                               file_lens.ctypes.data)
    if not h:
        raise ValueError("Sequitur rejected the input (bad token, size mismatch or out of memory)")
    try:
        nr, ns = ctypes.c_int64(), ctypes.c_int64()
        lib.gtc_grammar_sizes(h, ctypes.byref(nr), ctypes.byref(ns))
        rule_off = np.empty(nr.value + 1, np.int64)
        sym = np.empty(ns.value, np.int32)
        file_off = np.empty(file_lens.shape[0] + 1, np.int64)
        lib.gtc_grammar_export(h, rule_off.ctypes.data, sym.ctypes.data, file_off.ctypes.data)
    finally:
        lib.gtc_grammar_free(h)
    return Grammar(int(num_words), rule_off, sym, file_off)


def sequitur_sharded(tokens: np.ndarray, file_lens, num_words: int, shards: int) -> Grammar:
    """Sequitur on ``shards`` contiguous pieces of the text in parallel, the
    piece grammars concatenated into one: the root is the pieces' roots back
    to back, each piece keeps its own rules (renumbered; no rule is shared
    across pieces).  Pieces end at file boundaries when there are several
    files, else at equal token counts.  Used for corpora too large for one
    single-threaded Sequitur run."""
    from concurrent.futures import ThreadPoolExecutor
    tokens = np.ascontiguousarray(tokens, dtype=np.int32)
    file_lens = np.ascontiguousarray(file_lens, dtype=np.int64)
    n = int(tokens.shape[0])
    F = int(file_lens.shape[0])
    shards = max(1, min(shards, F) if F > 1 else shards)
    if F > 1:  # cut at the file boundary nearest to each equal share
        ends = np.cumsum(file_lens)
        cuts = sorted(set(int(np.searchsorted(ends, n * k / shards)) + 1 for k in range(1, shards)))
        fcuts = [0] + [c for c in cuts if 0 < c < F] + [F]
        pieces = [(int(ends[a - 1]) if a else 0, int(ends[b - 1]), file_lens[a:b]) for a, b in zip(fcuts, fcuts[1:])]
    else:
        bounds = [n * k // shards for k in range(shards + 1)]
        pieces = [(a, b, None) for a, b in zip(bounds, bounds[1:]) if b > a]
    with ThreadPoolExecutor(max_workers=len(pieces)) as ex:  # the builder releases the GIL
        parts = list(ex.map(lambda p: sequitur(tokens[p[0]:p[1]], p[2] if p[2] is not None else [p[1] - p[0]],
                                               num_words), pieces))
    V = int(num_words)
    roots, bodies, rule_lens = [], [], []
    file_offs, base_sym, nrules = [], 0, 1
    for part in parts:
        shift = nrules - 1  # rule r >= 1 of the piece becomes rule r + shift
        sym = part.sym.astype(np.int64)
        sym = np.where(sym >= V, sym + shift, sym).astype(np.int32)
        r0 = int(part.rule_off[1])
        roots.append(sym[:r0])
        bodies.append(sym[r0:])
        rule_lens.append(np.diff(part.rule_off[1:]))
        if F > 1:
            file_offs.append(part.file_off[1:] + base_sym)
        base_sym += r0
        nrules += part.num_rules - 1
    root = np.concatenate(roots)
    lens = np.concatenate([[root.shape[0]]] + rule_lens).astype(np.int64)
    rule_off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    file_off = (np.concatenate([[0]] + file_offs) if F > 1 else np.array([0, root.shape[0]])).astype(np.int64)
    return Grammar(V, rule_off, np.concatenate([root] + bodies).astype(np.int32), file_off)


def root_only_grammar(tokens: np.ndarray, file_lens, num_words: int) -> Grammar:
    """The trivial encoding: no rules, the root is the raw text."""
    tokens = np.ascontiguousarray(tokens, dtype=np.int32)
    file_off = np.concatenate([[0], np.cumsum(np.asarray(file_lens, np.int64))]).astype(np.int64)
    return Grammar(int(num_words), np.array([0, tokens.shape[0]], np.int64), tokens.copy(), file_off)


def refactor_grammar(g: Grammar, rng: np.random.Generator, rounds: int = 3, frac: float = 0.2) -> Grammar:
    """Re-encode ``g`` with extra random rules (same expansion, other DAG).

    Each round picks random adjacent symbol pairs inside bodies (never across
    a file boundary of the root) and moves each pair into a fresh rule used
    once.  Rule utility is deliberately not kept: the result is a valid but
    non-Sequitur grammar, which the analytics must handle identically.
    """
    bodies = [list(g.body(r)) for r in range(g.num_rules)]
    V = g.num_words
    root_files = [list(g.body(0)[g.file_off[f]:g.file_off[f + 1]]) for f in range(g.num_files)]
    for _ in range(rounds):
        new_rules = []

        def fold(seq):
            out, i = [], 0
            while i < len(seq):
                if i + 1 < len(seq) and rng.random() < frac:
                    rid = len(bodies) + len(new_rules)
                    new_rules.append([seq[i], seq[i + 1]])
                    out.append(V + rid)
                    i += 2
                else:
                    out.append(seq[i])
                    i += 1
            return out

        root_files = [fold(s) for s in root_files]
        for r in range(1, len(bodies)):
            bodies[r] = fold(bodies[r])
        bodies.extend(new_rules)
    bodies[0] = [x for s in root_files for x in s]
    lens = [len(b) for b in bodies]
    rule_off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    sym = np.array([x for b in bodies for x in b], np.int32)
    file_off = np.concatenate([[0], np.cumsum([len(s) for s in root_files])]).astype(np.int64)
    return Grammar(V, rule_off, sym, file_off)


# ---------------------------------------------------------------------------
# Synthetic Zipf corpora
# ---------------------------------------------------------------------------

def zipf_cdf(V: int, s: float) -> np.ndarray:
    w = np.arange(1, V + 1, dtype=np.float64) ** (-s)
    c = np.cumsum(w)
    return c / c[-1]


def zipf_tokens(rng: np.random.Generator, n: int, cdf: np.ndarray, perm: np.ndarray) -> np.ndarray:
    """n word IDs: Zipf ranks by inverse CDF, mapped to IDs by ``perm``."""
    u = rng.random(n)
    rank = np.searchsorted(cdf, u, side="right")
    np.minimum(rank, cdf.shape[0] - 1, out=rank)
    return perm[rank].astype(np.int32)


def zipf_tokens_chunked(seed: int, n: int, cdf: np.ndarray, perm: np.ndarray, chunk: int = 1 << 24,
                        workers: int | None = None) -> np.ndarray:
    """n word IDs like ``zipf_tokens``, drawn in chunks of ``chunk`` tokens
    from independent streams spawned from ``seed`` and filled by threads (the
    draws release the GIL).  The result depends on seed and n only, not on
    the number of threads."""
    from concurrent.futures import ThreadPoolExecutor
    out = np.empty(n, np.int32)
    nch = (n + chunk - 1) // chunk
    seqs = np.random.SeedSequence([int(seed), 0x5A]).spawn(max(nch, 1))

    def fill(c):
        a, b = c * chunk, min(n, (c + 1) * chunk)
        out[a:b] = zipf_tokens(np.random.default_rng(seqs[c]), b - a, cdf, perm)

    with ThreadPoolExecutor(max_workers=workers or min(16, os.cpu_count() or 1)) as ex:
        list(ex.map(fill, range(nch)))
    return out


def inject(rng: np.random.Generator, base: np.ndarray, pieces) -> np.ndarray:
    """Insert each piece into ``base`` at independent uniform positions."""
    if not pieces:
        return base
    pos = np.sort(rng.integers(0, base.shape[0] + 1, size=len(pieces)))
    order = rng.permutation(len(pieces))
    out, last = [], 0
    for p, k in zip(pos, order):
        out.append(base[last:p])
        out.append(pieces[k])
        last = p
    out.append(base[last:])
    return np.concatenate(out).astype(np.int32)


@dataclass
class Corpus:
    tokens: np.ndarray
    file_lens: np.ndarray
    num_words: int
    meta: dict


def make_corpus(name: str, seed: int | None = None, scale: float = 1.0) -> Corpus:
    """Build one of the named synthetic corpora.

    ``scale`` shrinks token counts (not vocabulary) for quick tests.
    """
    spec = CONFIGS[name]
    seed = spec["seed"] if seed is None else seed
    rng = np.random.default_rng(seed)
    V, s = spec["V"], spec["s"]
    cdf = zipf_cdf(V, s)
    perm = rng.permutation(V).astype(np.int32)
    kind = spec["kind"]
    if kind == "single_passages":
        N = max(int(spec["N"] * scale), 1000)
        plen = spec["passage_len"]
        npass = max(1, int(round(spec["passages"] * min(1.0, scale * 4))))
        pool = [zipf_tokens(rng, plen, cdf, perm) for _ in range(npass)]
        pieces = [p for p in pool for _ in range(spec["copies"])]
        base = zipf_tokens(rng, N - sum(len(p) for p in pieces), cdf, perm)
        toks = inject(rng, base, pieces)
        lens = np.array([toks.shape[0]], np.int64)
    elif kind == "files_passages":
        F = spec["F"]
        lo, hi = spec["len_range"]
        raw = np.exp(rng.uniform(np.log(lo), np.log(hi), size=F))
        lens_t = np.maximum(np.round(raw / raw.sum() * spec["N"] * scale), 0).astype(np.int64)
        plen = spec["passage_len"]
        pool = [zipf_tokens(rng, plen, cdf, perm) for _ in range(spec["passages"])]
        files = []
        for f in range(F):
            target = int(lens_t[f])
            want = int(round(target * spec["passage_frac"] / plen))
            pieces = [pool[i] for i in rng.integers(0, len(pool), size=want)]
            base = zipf_tokens(rng, max(target - want * plen, 0), cdf, perm)
            files.append(inject(rng, base, pieces))
        toks = np.concatenate(files).astype(np.int32)
        lens = np.array([f.shape[0] for f in files], np.int64)
    elif kind == "many_files":
        # `scale` shrinks the number of files, not their lengths
        F = max(2, int(round(spec["F"] * scale)))
        lo, hi = spec["len_range"]
        lens = np.round(np.exp(rng.uniform(np.log(lo), np.log(hi), size=F))).astype(np.int64)
        toks = zipf_tokens_chunked(seed, int(lens.sum()), cdf, perm)
    elif kind == "nested":
        # passages of passages: level 0 phrases of Zipf words, level d items
        # are concatenations of `fanout` level d-1 items; pieces from every
        # level are injected until `inject_frac` of the tokens
        N = max(int(spec["N"] * scale), 1000)
        levels = [[zipf_tokens(rng, spec["phrase_len"], cdf, perm) for _ in range(spec["phrases"])]]
        for _ in range(spec["depth"]):
            prev = levels[-1]
            levels.append([np.concatenate([prev[i] for i in rng.integers(0, len(prev), size=spec["fanout"])])
                           for _ in range(spec["pool"])])
        want = int(N * spec["inject_frac"])
        pieces, got = [], 0
        while got < want:
            lv = int(rng.integers(1, spec["depth"] + 1))
            p = levels[lv][int(rng.integers(0, len(levels[lv])))]
            if got + p.shape[0] > want and pieces:
                break
            pieces.append(p)
            got += p.shape[0]
        base = zipf_tokens(rng, max(N - got, 0), cdf, perm)
        toks = inject(rng, base, pieces)
        lens = np.array([toks.shape[0]], np.int64)
    else:
        raise ValueError(f"unknown corpus kind {kind}")
    meta = {"name": name, "seed": int(seed), "scale": scale, "V": V, "s": s, "N": int(toks.shape[0]),
            "F": int(lens.shape[0])}
    return Corpus(toks, lens, V, meta)


# Shapes follow the paper's workloads (Section V-A): one small file (like
# dataset D), a few large files sharing one grammar (like dataset B).
CONFIGS = {
    "wc_single_200k": dict(kind="single_passages", seed=20210613, N=200_000, V=20_000, s=1.1,
                           passages=50, passage_len=200, copies=4),
    "multi64_50m": dict(kind="files_passages", seed=20210614, N=50_000_000, F=64, len_range=(10_000, 2_000_000),
                        V=500_000, s=1.0, passages=500, passage_len=200, passage_frac=0.05),
    # many files: 100k files of 1k-50k tokens (log-uniform, ~1.25B tokens),
    # Zipf 1.1 over 200k words
    "files100k": dict(kind="many_files", seed=20210616, F=100_000, len_range=(1_000, 50_000), V=200_000, s=1.1),
    # the same shape with files of 100-5000 tokens: every file fits one CTA's
    # shared memory (the per-file bottom-up path for short files)
    "files_short": dict(kind="many_files", seed=20210618, F=100_000, len_range=(100, 5_000), V=200_000, s=1.1),
    # one large file with nested repeats (like dataset E): a deep rule DAG
    "nested_500m": dict(kind="nested", seed=20210615, N=500_000_000, V=1_000_000, s=1.05, phrases=4096,
                        phrase_len=16, depth=6, fanout=4, pool=256, inject_frac=0.5),
}


def serving_corpus(i: int, seed: int = 20210617, tokens_range=(1_000_000, 8_000_000)) -> Corpus:
    """Corpus i of the serving set: size log-uniform in tokens_range, Zipf
    exponent uniform in [1.0, 1.2] over 1M words, files log-uniform in
    [10k, 2M] tokens (at most 64 per corpus)."""
    rng = np.random.default_rng(seed + 7919 * i)
    n = int(np.exp(rng.uniform(np.log(tokens_range[0]), np.log(tokens_range[1]))))
    s_exp = float(rng.uniform(1.0, 1.2))
    V = 1_000_000
    cdf = zipf_cdf(V, s_exp)
    perm = rng.permutation(V).astype(np.int32)
    lens = []
    while sum(lens) < n and len(lens) < 64:
        lens.append(int(np.exp(rng.uniform(np.log(10_000), np.log(2_000_000)))))
    lens = np.array(lens, np.float64)
    lens = np.maximum(np.round(lens / lens.sum() * n), 1).astype(np.int64)
    toks = zipf_tokens(rng, int(lens.sum()), cdf, perm)
    meta = {"name": f"serving{i}", "seed": seed, "V": V, "s": s_exp, "N": int(toks.shape[0]), "F": int(lens.shape[0])}
    return Corpus(toks, lens, V, meta)


def load_serving(i: int, **kw) -> Grammar:
    tag = hashlib.sha1(json.dumps(["serving", i, kw, "v1"], sort_keys=True, default=str).encode()).hexdigest()[:12]
    path = cache_dir() / f"serving{i}_{tag}.npz"
    if path.exists():
        return Grammar.load(path)
    c = serving_corpus(i, **kw)
    g = sequitur(c.tokens, c.file_lens, c.num_words)
    g.meta = dict(c.meta)
    tmp = path.with_suffix(f".tmp{os.getpid()}.npz")
    g.save(tmp)
    os.replace(tmp, path)
    return g


def load_serving_set(n: int, tokens_range=(1_000_000, 32_000_000), workers: int | None = None) -> list:
    """Grammars of serving corpora 0..n-1, built in parallel threads (the
    generator's numpy work and the Sequitur builder release the GIL)."""
    from concurrent.futures import ThreadPoolExecutor
    workers = workers or min(16, os.cpu_count() or 1)
    with ThreadPoolExecutor(max_workers=workers) as ex:
        return list(ex.map(lambda i: load_serving(i, tokens_range=tokens_range), range(n)))


def cache_dir() -> Path:
    d = Path(os.environ.get("GT_CACHE_DIR", ROOT / ".gtcache"))
    d.mkdir(parents=True, exist_ok=True)
    return d


# corpora above this many tokens are compressed by sequitur_sharded
SHARD_ABOVE = 100_000_000


def load_config(name: str, scale: float = 1.0, keep_tokens: bool = False):
    """Corpus + Sequitur grammar for a named config, cached on disk.

    Returns ``(grammar, corpus_or_None)``.
    """
    tag = hashlib.sha1(json.dumps([name, CONFIGS[name], scale, "v1"], sort_keys=True).encode()).hexdigest()[:12]
    path = cache_dir() / f"{name}_{tag}.npz"
    if path.exists() and not keep_tokens:
        return Grammar.load(path), None
    corpus = make_corpus(name, scale=scale)
    if path.exists():
        g = Grammar.load(path)
    else:
        if corpus.tokens.shape[0] > SHARD_ABOVE:
            g = sequitur_sharded(corpus.tokens, corpus.file_lens, corpus.num_words,
                                 shards=min(16, os.cpu_count() or 1))
        else:
            g = sequitur(corpus.tokens, corpus.file_lens, corpus.num_words)
        g.meta = dict(corpus.meta)
        tmp = path.with_suffix(f".tmp{os.getpid()}.npz")
        g.save(tmp)
        os.replace(tmp, path)
    return g, (corpus if keep_tokens else None)


def prefix_files(g: Grammar, k: int) -> Grammar:
    """The same grammar restricted to its first ``k`` files (rules unchanged)."""
    return file_range(g, 0, max(1, min(k, g.num_files)))


def file_range(g: Grammar, a: int, b: int) -> Grammar:
    """The same grammar restricted to files ``a .. b-1`` (rules unchanged)."""
    a, b = max(0, a), min(b, g.num_files)
    r0, r1 = int(g.file_off[a]), int(g.file_off[b])
    root_len = int(g.rule_off[1])
    sym = np.concatenate([g.sym[r0:r1], g.sym[root_len:]]).astype(np.int32)
    rule_off = g.rule_off.copy()
    rule_off[1:] -= root_len - (r1 - r0)
    return Grammar(g.num_words, rule_off, sym, (g.file_off[a:b + 1] - r0).astype(np.int64), dict(g.meta))


def root_prefix(g: Grammar, n: int) -> Grammar:
    """A one-file grammar whose file is the first ``n`` root symbols of ``g``'s
    first file (rules unchanged): a bounded sample of a one-file corpus."""
    n = max(1, min(n, int(g.file_off[1])))
    root_len = int(g.rule_off[1])
    sym = np.concatenate([g.sym[:n], g.sym[root_len:]]).astype(np.int32)
    rule_off = g.rule_off.copy()
    rule_off[1:] -= root_len - n
    return Grammar(g.num_words, rule_off, sym, np.array([0, n], np.int64), dict(g.meta))
