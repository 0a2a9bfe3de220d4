// Device helpers shared by the streaming kernels: bulk-copy staging through
// shared memory with mbarriers, bounded waits, and small search routines.
#pragma once

#include <cstdint>

#include "gt_internal.cuh"

namespace gt {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// 1-D bulk copy global -> shared (TMA engine, no tensor map).  Both addresses
// 16-byte aligned, size a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t global_timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for an mbarrier phase with a wall-clock limit.  Returns false (and
// raises ST_TIMEOUT in *status) if the limit passes first.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t* status,
                                                  uint64_t limit_ns = 2000000000ull) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_timer_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (global_timer_ns() - t0 > limit_ns) {
      atomicOr(status, ST_TIMEOUT);
      return false;
    }
  }
  return true;
}

// Index of the last element <= x in a[0..n) (a ascending, a[0] <= x).
template <class T>
__device__ __forceinline__ int last_le(const T* a, int n, T x) {
  int lo = 0, hi = n;  // answer in [lo, hi)
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (a[mid] <= x) lo = mid;
    else hi = mid;
  }
  return lo;
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

__device__ __forceinline__ uint32_t hash_u32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352dU;
  x ^= x >> 15;
  x *= 0x846ca68bU;
  x ^= x >> 16;
  return x;
}

__device__ __forceinline__ uint64_t hash_u64(uint64_t x) {
  x ^= x >> 33;
  x *= 0xff51afd7ed558ccdULL;
  x ^= x >> 33;
  x *= 0xc4ceb9fe1a85ec53ULL;
  x ^= x >> 33;
  return x;
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

}  // namespace gt
