// Device helpers shared by the kernels: a search routine and the 3-word
// window helpers used by the global and per-file sequence paths.
#pragma once

#include <cstdint>

#include "gt_internal.cuh"

namespace gt {

// Lanes of the warp holding the same 8-bit digit as this lane (among `active`),
// from one ballot per digit bit.  Every lane of the warp must call it.
__device__ __forceinline__ unsigned warp_digit_peers(uint32_t d, unsigned active) {
  unsigned peers = active;
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    const bool bit = (d >> b) & 1u;
    const unsigned bal = __ballot_sync(0xffffffffu, bit);
    peers &= bit ? bal : ~bal;
  }
  return peers;
}

__device__ __forceinline__ int64_t upper_bound_dev(const int64_t* a, int64_t n, int64_t x) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (a[mid] <= x) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// ---- 3-word windows (shared by the top-down and bottom-up sequence paths) ----

struct Sym3 {
  int32_t first, second, second_last, last;  // -1 where the expansion is too short
};

__device__ __forceinline__ Sym3 sym_words(const DevGrammar& d, const int32_t* __restrict__ head,
                                          const int32_t* __restrict__ tail, int32_t x) {
  Sym3 r;
  if (x < d.V) {
    r.first = r.last = x;
    r.second = r.second_last = -1;
  } else {
    const int32_t c = x - d.V;
    r.first = head[2 * c];
    r.second = head[2 * c + 1];
    r.second_last = tail[2 * c];
    r.last = tail[2 * c + 1];
  }
  return r;
}

__device__ __forceinline__ uint64_t pack_compact(int32_t a, int32_t b, int32_t c, int kb) {
  return (uint64_t(uint32_t(a)) << (2 * kb)) | (uint64_t(uint32_t(b)) << kb) | uint64_t(uint32_t(c));
}

// End (exclusive) of the body sequence holding position j: the file's end in
// the root, the rule's end elsewhere.  Also returns the rule.
__device__ __forceinline__ int64_t seq_end(const DevGrammar& d, int64_t j, int32_t* rule, int32_t* file) {
  if (j < d.root_len) {
    const int64_t f = upper_bound_dev(d.file_off, int64_t(d.F) + 1, j) - 1;
    *rule = 0;
    *file = int32_t(f);
    return d.file_off[f + 1];
  }
  const int32_t r = d.sym_rule[j - d.first_rule_tile * kTile];
  *rule = r;
  *file = -1;
  return d.rule_off[r + 1];
}

// The (at most two) owned windows starting in body symbol j; returns how many.
__device__ __forceinline__ int windows_at(const DevGrammar& d, const int32_t* __restrict__ head,
                                          const int32_t* __restrict__ tail, int64_t j, int64_t end, int kb,
                                          uint64_t* k) {
  if (j + 1 >= end) return 0;
  const Sym3 a = sym_words(d, head, tail, d.sym[j]);
  const Sym3 b = sym_words(d, head, tail, d.sym[j + 1]);
  const int32_t n1 = b.first;
  int32_t n2 = b.second;
  if (n2 < 0) n2 = j + 2 < end ? sym_words(d, head, tail, d.sym[j + 2]).first : -1;
  // k[0], k[1] are always written (fixed indices keep them in registers)
  const bool w0 = a.second_last >= 0;  // child with >= 2 words
  const uint64_t x0 = w0 ? pack_compact(a.second_last, a.last, n1, kb) : 0;
  const uint64_t x1 = n2 >= 0 ? pack_compact(a.last, n1, n2, kb) : 0;
  k[0] = w0 ? x0 : x1;
  k[1] = x1;
  return int(w0) + int(n2 >= 0);
}

// Windows of the 4 symbols j0 .. j0+3: symbol i has n[i] of them, keys
// k[i][0..n[i]), owner rule r[i].
struct TileWin {
  uint64_t k[4][2];
  int32_t r[4];
  int n[4];
};

__device__ __forceinline__ int tile_windows(const DevGrammar& d, const int32_t* __restrict__ head,
                                            const int32_t* __restrict__ tail, int kb, int64_t j0, TileWin& t) {
  int c = 0;
  int64_t end = -1;  // end of the body sequence holding the previous symbol (rule or root file)
  int32_t rule = 0, f;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t j = j0 + i;
    t.n[i] = 0;
    t.r[i] = 0;
    if (j < d.G) {
      // the four symbols usually share one sequence: look it up again only
      // when the previous one ended (or at a root / rule boundary)
      if (j >= end || j == d.root_len) end = seq_end(d, j, &rule, &f);
      t.r[i] = rule;
      t.n[i] = windows_at(d, head, tail, j, end, kb, t.k[i]);
    }
    c += t.n[i];
  }
  return c;
}

// compact key (kb bits per word) -> w1 << 42 | w2 << 21 | w3; kb == 0 keeps it
__device__ __forceinline__ uint64_t to_output_key(uint64_t k, int kb) {
  if (kb == 0) return k;
  const uint64_t m = (uint64_t(1) << kb) - 1;
  return ((k >> (2 * kb)) << 42) | (((k >> kb) & m) << 21) | (k & m);
}

// ---- decoupled look-back over items taken in ticket order --------------
// Flag word per item: state in the top two bits (0 nothing published, 1 the
// item's own total, 2 the inclusive prefix through the item), value below.
// An item only waits on items with smaller tickets, i.e. ones already
// running, so every wait ends; each is bounded anyway.
constexpr uint64_t kFlagAgg = 1ull << 62, kFlagIncl = 2ull << 62, kFlagVal = (1ull << 62) - 1;
constexpr int kSpinLimit = 1 << 22;  // look-back polls before giving up (>= 0.25 s)

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// The item's own total, published as soon as it is known (one thread); item
// 0 publishes its inclusive prefix directly.
__device__ __forceinline__ void publish_aggregate(unsigned long long* flags, int64_t item, uint64_t agg) {
  atomicExch(&flags[item], (item == 0 ? kFlagIncl : kFlagAgg) | agg);
}

// By one warp: reads the flags of the 32 preceding items at once, adds their
// values up to the nearest one with a published prefix, and moves 32 items
// further back while there is none; then publishes the item's inclusive
// prefix.  Returns the exclusive prefix (to every lane); after kSpinLimit
// polls of an item that published nothing it sets ST_TIMEOUT in *status,
// still publishes (so that later items are not held up) and returns -1.
__device__ __forceinline__ int64_t warp_look_back(unsigned long long* flags, int64_t item, uint64_t agg,
                                                  unsigned* status, int spin_limit = kSpinLimit) {
  const int lane = threadIdx.x & 31;
  if (item == 0) return 0;
  uint64_t excl = 0;
  int64_t top = item - 1;  // the window is flags[top - 31 .. top], lane l reads top - l
  int spins = 0;
  bool ok = true;
  while (true) {
    const int64_t j = top - lane;
    const unsigned long long v = j >= 0 ? ld_acquire_u64(&flags[j]) : kFlagIncl;
    const uint64_t st = v & ~kFlagVal;
    if (__any_sync(0xffffffffu, st == 0)) {
      if (++spins > spin_limit) {
        ok = false;
        break;
      }
      __nanosleep(32);
      continue;
    }
    const unsigned incl = __ballot_sync(0xffffffffu, st == kFlagIncl);
    const int stop = incl ? __ffs(incl) - 1 : 31;  // nearest item with a prefix, else the whole window
    uint64_t part = lane <= stop ? (v & kFlagVal) : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    excl += part;
    if (incl) break;
    top -= 32;  // flags[0] always holds a prefix, so the walk ends
  }
  if (lane == 0) {
    if (!ok && status) atomicOr(status, ST_TIMEOUT);
    atomicExch(&flags[item], kFlagIncl | (excl + agg));
  }
  return ok ? int64_t(excl) : -1;
}

}  // namespace gt
