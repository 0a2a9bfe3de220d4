// Sequitur grammar inference over an int32 token stream, producing the
// TADOC compressed form (Section II-A of G-TADOC, arXiv 2106.06889): a
// context-free grammar whose root rule holds every file, separated by unique
// splitter symbols, and whose other rules each stand for a repeated phrase.
//
// This is input preparation (the compressor), not part of the analytics: it
// only has to emit a grammar that expands back to the input and satisfies
// Sequitur's two invariants (Nevill-Manning & Witten, "Identifying
// hierarchical structure in sequences: a linear-time algorithm", JAIR 1997):
//   * digram uniqueness: no pair of adjacent symbols occurs twice without
//     overlapping anywhere in the grammar;
//   * rule utility: every rule other than the root is referenced at least
//     twice.
//
// Implementation notes (our own design):
//   * symbols live in index-based arrays (value, prev, next, kind) so the
//     working set is compact; each rule is a circular list through a guard;
//   * every reference node is also threaded on its rule's occurrence list,
//     so the single remaining use of a rule is found in O(1) when its use
//     count drops to one;
//   * digram checks and rule-utility repairs are deferred onto two explicit
//     work stacks instead of recursing, and each popped item is re-validated,
//     so no frame ever acts on a node another repair has already removed;
//   * the digram index is an open-addressing table whose entries are
//     re-validated on lookup.
//
// C interface (all sizes int64, all arrays caller-owned):
//   gtc_sequitur_build(tokens, n, num_words, num_files, file_len) -> handle
//   gtc_grammar_sizes(handle, &num_rules, &num_syms)
//   gtc_grammar_export(handle, rule_off, sym, file_off)
//   gtc_grammar_free(handle)
// Output encoding: rule 0 is the root; its body is the concatenation of the
// files with splitters removed and file_off[f] marks where file f starts.
// A body symbol s < num_words is a word; s >= num_words references rule
// s - num_words.

#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

namespace {

enum : uint8_t { K_DEAD = 0, K_TERM = 1, K_REF = 2, K_GUARD = 3 };

static inline uint64_t mix64(uint64_t x) {
  // splitmix64 finaliser
  x ^= x >> 30;
  x *= 0xbf58476d1ce4e5b9ULL;
  x ^= x >> 27;
  x *= 0x94d049bb133111ebULL;
  x ^= x >> 31;
  return x;
}

struct Sequitur {
  // node arrays; code >= 0 is a terminal, code < 0 references rule -(code+1);
  // for a guard node, code is the id of the rule it closes
  std::vector<int32_t> code, prv, nxt, occ_prev, occ_next;
  std::vector<uint8_t> kind;
  // rule arrays
  std::vector<int32_t> guard, uses, occ_head;
  std::vector<uint8_t> alive;
  // digram index: key -> node where the digram starts
  std::vector<uint64_t> tkey;
  std::vector<int32_t> tval;  // -1 empty, -2 tombstone
  uint64_t tmask = 0, tused = 0;
  std::vector<int32_t> checks, repairs;
  std::vector<int32_t> free_nodes;  // recycled node slots

  static uint64_t key_of(int32_t a, int32_t b) {
    return (uint64_t(uint32_t(a)) << 32) | uint64_t(uint32_t(b));
  }

  int32_t new_node(int32_t c, uint8_t k) {
    if (!free_nodes.empty()) {
      // A recycled slot may still be named by a queued check or an index
      // entry; both are re-validated before use, so reuse is harmless.
      int32_t id = free_nodes.back();
      free_nodes.pop_back();
      code[id] = c;
      prv[id] = nxt[id] = occ_prev[id] = occ_next[id] = -1;
      kind[id] = k;
      return id;
    }
    if (code.size() >= size_t(INT32_MAX)) throw std::bad_alloc();
    int32_t id = int32_t(code.size());
    code.push_back(c);
    prv.push_back(-1);
    nxt.push_back(-1);
    occ_prev.push_back(-1);
    occ_next.push_back(-1);
    kind.push_back(k);
    return id;
  }
  void link(int32_t a, int32_t b) {
    nxt[a] = b;
    prv[b] = a;
  }
  int32_t new_rule() {
    int32_t r = int32_t(guard.size());
    int32_t g = new_node(r, K_GUARD);
    link(g, g);
    guard.push_back(g);
    uses.push_back(0);
    occ_head.push_back(-1);
    alive.push_back(1);
    return r;
  }
  bool is_sym(int32_t a) const { return kind[a] == K_TERM || kind[a] == K_REF; }
  bool digram_at(int32_t a) const { return is_sym(a) && is_sym(nxt[a]); }

  // ---- occurrence lists ----
  void add_use(int32_t n) {
    int32_t r = -(code[n] + 1);
    uses[r]++;
    occ_prev[n] = -1;
    occ_next[n] = occ_head[r];
    if (occ_head[r] >= 0) occ_prev[occ_head[r]] = n;
    occ_head[r] = n;
  }
  void drop_use(int32_t n) {
    int32_t r = -(code[n] + 1);
    uses[r]--;
    if (occ_prev[n] >= 0) occ_next[occ_prev[n]] = occ_next[n];
    else occ_head[r] = occ_next[n];
    if (occ_next[n] >= 0) occ_prev[occ_next[n]] = occ_prev[n];
    if (uses[r] == 1) repairs.push_back(r);
  }

  // ---- digram table ----
  void table_init(uint64_t expect) {
    uint64_t cap = 1024;
    while (cap < expect * 2) cap <<= 1;
    tkey.assign(cap, 0);
    tval.assign(cap, -1);
    tmask = cap - 1;
    tused = 0;
  }
  bool entry_valid(uint64_t key, int32_t n) const {
    return n >= 0 && digram_at(n) && key_of(code[n], code[nxt[n]]) == key;
  }
  void rehash() {
    std::vector<uint64_t> ok;
    std::vector<int32_t> ov;
    ok.swap(tkey);
    ov.swap(tval);
    uint64_t live = 0;
    for (size_t i = 0; i < ov.size(); ++i)
      if (ov[i] >= 0) ++live;
    uint64_t cap = ok.size();
    while (cap < live * 4) cap <<= 1;
    tkey.assign(cap, 0);
    tval.assign(cap, -1);
    tmask = cap - 1;
    tused = 0;
    for (size_t i = 0; i < ov.size(); ++i) {
      if (ov[i] < 0 || !entry_valid(ok[i], ov[i])) continue;
      uint64_t h = mix64(ok[i]) & tmask;
      while (tval[h] != -1) h = (h + 1) & tmask;
      tkey[h] = ok[i];
      tval[h] = ov[i];
      ++tused;
    }
  }
  // returns the slot holding key, or -1
  int64_t table_find(uint64_t key) const {
    uint64_t h = mix64(key) & tmask;
    while (true) {
      int32_t v = tval[h];
      if (v == -1) return -1;
      if (v >= 0 && tkey[h] == key) return int64_t(h);
      h = (h + 1) & tmask;
    }
  }
  void table_put(uint64_t key, int32_t n) {
    int64_t s = table_find(key);
    if (s >= 0) {
      tval[s] = n;
      return;
    }
    if ((tused + 1) * 2 > tmask + 1) rehash();
    uint64_t h = mix64(key) & tmask;
    while (tval[h] >= 0) h = (h + 1) & tmask;
    if (tval[h] == -1) ++tused;
    tkey[h] = key;
    tval[h] = n;
  }
  // Forget the digram starting at a if the index points at this occurrence.
  // A digram skipped earlier because it overlapped this one may now be the
  // only occurrence, so its neighbours are queued for a fresh check.
  void forget(int32_t a) {
    if (!digram_at(a)) return;
    uint64_t key = key_of(code[a], code[nxt[a]]);
    int64_t s = table_find(key);
    if (s >= 0 && tval[s] == a) tval[s] = -2;
    if (is_sym(prv[a])) checks.push_back(prv[a]);
    if (is_sym(nxt[a])) checks.push_back(nxt[a]);
  }

  // ---- grammar edits ----
  void kill(int32_t n) {
    kind[n] = K_DEAD;
    free_nodes.push_back(n);
  }
  // Replace the digram starting at a by one reference to rule r.
  void substitute(int32_t a, int32_t r) {
    int32_t b = nxt[a], q = prv[a], c = nxt[b];
    forget(q);
    forget(a);
    forget(b);
    if (kind[a] == K_REF) drop_use(a);
    if (kind[b] == K_REF) drop_use(b);
    kill(a);
    kill(b);
    int32_t n = new_node(-(r + 1), K_REF);
    add_use(n);
    link(q, n);
    link(n, c);
    checks.push_back(q);
    checks.push_back(n);
  }
  // a and m start equal, non-overlapping digrams; m is the indexed one.
  void match(int32_t a, int32_t m) {
    int32_t m2 = nxt[m];
    if (kind[prv[m]] == K_GUARD && prv[m] == nxt[m2] && code[prv[m]] != 0) {
      substitute(a, code[prv[m]]);
      return;
    }
    int32_t r = new_rule();
    int32_t g = guard[r];
    int32_t n1 = new_node(code[m], kind[m]);
    int32_t n2 = new_node(code[m2], kind[m2]);
    link(g, n1);
    link(n1, n2);
    link(n2, g);
    if (kind[n1] == K_REF) add_use(n1);
    if (kind[n2] == K_REF) add_use(n2);
    substitute(m, r);
    substitute(a, r);
    table_put(key_of(code[n1], code[n2]), n1);
  }
  // Inline rule x at its single remaining use.
  void expand(int32_t x) {
    int32_t e = occ_head[x];
    int32_t q = prv[e], c = nxt[e];
    int32_t g = guard[x];
    int32_t f = nxt[g], l = prv[g];
    forget(q);
    forget(e);
    drop_use(e);
    kill(e);
    kill(g);
    alive[x] = 0;
    link(q, f);
    link(l, c);
    checks.push_back(q);
    checks.push_back(l);
  }
  void check(int32_t a) {
    if (!digram_at(a)) return;
    int32_t b = nxt[a];
    uint64_t key = key_of(code[a], code[b]);
    int64_t s = table_find(key);
    int32_t m = s >= 0 ? tval[s] : -1;
    if (m >= 0 && !entry_valid(key, m)) {
      tval[s] = -2;
      m = -1;
    }
    if (m < 0) {
      table_put(key, a);
      return;
    }
    if (m == a || nxt[m] == a || b == m) return;
    match(a, m);
  }
  void settle() {
    while (!repairs.empty() || !checks.empty()) {
      if (!repairs.empty()) {
        int32_t x = repairs.back();
        repairs.pop_back();
        if (x != 0 && alive[x] && uses[x] == 1) expand(x);
        continue;
      }
      int32_t a = checks.back();
      checks.pop_back();
      check(a);
    }
  }

  void run(const int32_t* tok, int64_t n, int32_t num_words, int32_t num_files, const int64_t* flen) {
    code.reserve(size_t(n) + size_t(n) / 2 + 16);
    prv.reserve(code.capacity());
    nxt.reserve(code.capacity());
    occ_prev.reserve(code.capacity());
    occ_next.reserve(code.capacity());
    kind.reserve(code.capacity());
    table_init(uint64_t(n) + 16);
    new_rule();  // root
    int32_t root_g = guard[0];
    int64_t pos = 0;
    for (int32_t f = 0; f < num_files; ++f) {
      for (int64_t i = 0; i < flen[f]; ++i, ++pos) {
        int32_t node = new_node(tok[pos], K_TERM);
        int32_t last = prv[root_g];
        link(last, node);
        link(node, root_g);
        checks.push_back(last);
        settle();
      }
      if (f + 1 < num_files) {  // unique splitter between files
        int32_t node = new_node(num_words + f, K_TERM);
        int32_t last = prv[root_g];
        link(last, node);
        link(node, root_g);
        checks.push_back(last);
        settle();
      }
    }
  }
};

struct Grammar {
  std::vector<int64_t> rule_off;
  std::vector<int32_t> sym;
  std::vector<int64_t> file_off;
};

Grammar* export_grammar(Sequitur& S, int32_t num_words, int32_t num_files) {
  Grammar* G = new Grammar();
  int32_t nr = int32_t(S.guard.size());
  std::vector<int32_t> newid(nr, -1);
  int32_t cnt = 0;
  for (int32_t r = 0; r < nr; ++r)
    if (S.alive[r]) newid[r] = cnt++;
  G->rule_off.reserve(cnt + 1);
  G->file_off.reserve(num_files + 1);
  for (int32_t r = 0; r < nr; ++r) {
    if (!S.alive[r]) continue;
    G->rule_off.push_back(int64_t(G->sym.size()));
    int32_t g = S.guard[r];
    if (r == 0) G->file_off.push_back(0);
    for (int32_t n = S.nxt[g]; n != g; n = S.nxt[n]) {
      int32_t c = S.code[n];
      if (S.kind[n] == K_REF) {
        G->sym.push_back(num_words + newid[-(c + 1)]);
      } else if (c >= num_words) {  // splitter: file boundary in the root
        G->file_off.push_back(int64_t(G->sym.size()) - G->rule_off[0]);
      } else {
        G->sym.push_back(c);
      }
    }
    if (r == 0) G->file_off.push_back(int64_t(G->sym.size()));
  }
  G->rule_off.push_back(int64_t(G->sym.size()));
  return G;
}

}  // namespace

extern "C" {

void* gtc_sequitur_build(const int32_t* tokens, int64_t n, int32_t num_words, int32_t num_files,
                         const int64_t* file_len) {
  if (!tokens && n > 0) return nullptr;
  if (num_files < 1 || num_words < 1) return nullptr;
  int64_t total = 0;
  for (int32_t f = 0; f < num_files; ++f) {
    if (file_len[f] < 0) return nullptr;
    total += file_len[f];
  }
  if (total != n) return nullptr;
  if (n + num_files > (int64_t(1) << 30)) return nullptr;  // node ids are int32
  for (int64_t i = 0; i < n; ++i)
    if (tokens[i] < 0 || tokens[i] >= num_words) return nullptr;
  try {
    Sequitur* S = new Sequitur();
    S->run(tokens, n, num_words, num_files, file_len);
    Grammar* G = export_grammar(*S, num_words, num_files);
    delete S;
    return G;
  } catch (const std::bad_alloc&) {
    return nullptr;
  }
}

void gtc_grammar_sizes(const void* h, int64_t* num_rules, int64_t* num_syms) {
  const Grammar* G = static_cast<const Grammar*>(h);
  *num_rules = int64_t(G->rule_off.size()) - 1;
  *num_syms = int64_t(G->sym.size());
}

void gtc_grammar_export(const void* h, int64_t* rule_off, int32_t* sym, int64_t* file_off) {
  const Grammar* G = static_cast<const Grammar*>(h);
  std::memcpy(rule_off, G->rule_off.data(), G->rule_off.size() * sizeof(int64_t));
  std::memcpy(sym, G->sym.data(), G->sym.size() * sizeof(int32_t));
  std::memcpy(file_off, G->file_off.data(), G->file_off.size() * sizeof(int64_t));
}

void gtc_grammar_free(void* h) { delete static_cast<Grammar*>(h); }

}  // extern "C"
