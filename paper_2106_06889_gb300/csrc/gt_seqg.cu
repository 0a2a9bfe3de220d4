// Global 3-word sequence count (l = 3, Section IV-C/D) by sample-sort buckets
// (selected by the "seq_path" parameter; the default is the one-row-per-
// window radix sort of gt_seq.cu, which measured faster on the 500M-token
// corpus: the per-bucket sort below is bound by its instruction count).
//
// Every owned window (Eq. 1: the windows a rule's body crosses, built from
// the body, a two-symbol look-ahead and the children's head/tail buffers; see
// gt_seq.cu) is one row (compact key, weight of its rule).  The result is the
// sum of the weights per distinct key in ascending key order.  Instead of one
// global LSD radix sort over all rows (eight passes over ~12 bytes per row),
// the rows are put in key order by two bucket passes and reduced per bucket:
//
//   1. coarse bounds: the windows at 8192 evenly spaced body positions are
//      sorted in one CTA; up to 1023 equally spaced sample keys become the
//      bounds of the coarse buckets (sample sort, so a skewed - Zipf - key
//      distribution still gives buckets of similar size);
//   2. emit: every CTA of a persistent grid writes its tiles' windows as rows
//      in position order (row offsets per tile are structure, built once per
//      grammar) and counts them per coarse bucket; a scan gives each
//      (bucket, CTA) its output range;
//   3. scatter: each CTA re-reads its own rows, stages them in shared memory
//      in bucket order and writes them as runs;
//   4. fine split: one CTA per coarse bucket sorts a sample of its rows, cuts
//      the bucket into fine buckets of about kFineRows rows, counts and
//      scatters the rows into them (staged the same way);
//   5. reduce: a persistent kernel takes the fine buckets in key order; a CTA
//      sums the weights of equal keys in a shared-memory hash table (equal
//      keys of a warp merged first with __match_any_sync, so a hot 3-gram is
//      one update per warp), sorts the distinct keys in shared memory (sample
//      sort into 256 sub-buckets, finished by threads or warps) and writes
//      them at the position a decoupled look-back over the preceding fine
//      buckets gives.  A bucket
//      with more distinct keys than the table holds is sorted in place in
//      global memory by the same CTA instead (correct for any input; the
//      sample makes it rare).
//
// Only counts depend on the weights; the order of rows inside a bucket is
// whatever the atomics give, and the output is the same for every run.
#include <algorithm>
#include <cstddef>

#include "gt_device.cuh"

namespace gt {
namespace {

constexpr int kSgThreads = kTile / 4;  // 512 threads: one tile of symbols, 4 per thread
constexpr int kMaxCoarse = 1024;       // coarse buckets at most
constexpr int kMaxFine = 256;          // fine buckets per coarse bucket at most
constexpr int kFineRows = 1536;        // target rows per fine bucket
constexpr int kCoarseRows = 65536;     // target rows per coarse bucket (fewer than kMaxCoarse buckets)
constexpr int kSampPos = 8192;         // body positions sampled for the coarse bounds
constexpr int kSampKeys = 2 * kSampPos;
constexpr int kFineSamp = 4096;        // rows sampled per coarse bucket
constexpr int kFineTile = 4096;        // rows per step of the fine scatter
constexpr uint64_t kEmpty = ~0ull;     // above every compact key (they have at most 63 bits)

// number of entries of the ascending s[0, n) that are <= x
__device__ __forceinline__ int upper_bound_u64(const uint64_t* s, int n, uint64_t x) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (s[mid] <= x) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Ascending bitonic sort of a[0, n) in shared memory, n a power of two.
__device__ void bitonic_sort_shared(uint64_t* a, int n) {
  for (int k = 2; k <= n; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int p = i ^ j;
        if (p > i) {
          const uint64_t x = a[i], y = a[p];
          if ((x > y) == ((i & k) == 0)) {
            a[i] = y;
            a[p] = x;
          }
        }
      }
      __syncthreads();
    }
}

// Exclusive scan over the CTA (T threads, one value each); *total = sum.
template <int T>
__device__ __forceinline__ uint32_t block_scan_u32(uint32_t v, uint32_t* total) {
  __shared__ uint32_t warp_tot[T / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  uint32_t before = 0, all = 0;
#pragma unroll
  for (int w = 0; w < T / 32; ++w) {
    const uint32_t t = warp_tot[w];
    before += w < warp ? t : 0u;
    all += t;
  }
  __syncthreads();
  *total = all;
  return before + incl - v;
}

// Exclusive scan of h[0, n) into st[0, n) (n <= 2 * T); returns the total.
template <int T>
__device__ __forceinline__ uint32_t scan_counts(const uint32_t* h, uint32_t* st, int n) {
  const int i0 = 2 * threadIdx.x;
  const uint32_t a = i0 < n ? h[i0] : 0u, b = i0 + 1 < n ? h[i0 + 1] : 0u;
  uint32_t total;
  const uint32_t e = block_scan_u32<T>(a + b, &total);
  if (i0 < n) st[i0] = e;
  if (i0 + 1 < n) st[i0 + 1] = e + a;
  return total;
}

// Arguments of the passes over the grammar and over its rows.
struct SgArgs {
  DevGrammar d;
  const int32_t* head;
  const int32_t* tail;
  const uint64_t* wt;        // rule weights (Algorithm 1)
  const uint64_t* spl;       // coarse bounds, nspl of them
  const uint16_t* lut;       // [2^lut_bits + 1]: first bucket of each key prefix
  const int64_t* tile_off;   // [ntiles + 1]: first row of every tile of symbols
  int kb;                    // bits per word in a compact key
  int nspl;
  int lut_bits, lut_shift;   // prefix = key >> lut_shift has lut_bits bits
};

constexpr int kLutBitsMax = 12;

// Coarse bucket of a key: the number of bounds <= key, searched only among
// the bounds that share the key's prefix (usually none or one).
__device__ __forceinline__ int coarse_bucket(const uint64_t* spl, const uint16_t* lut, int lut_shift, uint64_t key) {
  const uint32_t p = uint32_t(key >> lut_shift);
  int lo = lut[p], hi = lut[p + 1];
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (spl[mid] <= key) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// ---- 1. coarse bounds -------------------------------------------------------

__global__ void __launch_bounds__(1024) sg_bounds_kernel(const __grid_constant__ SgArgs a, uint64_t* __restrict__ spl,
                                                         uint16_t* __restrict__ lut) {
  extern __shared__ __align__(16) uint64_t s_keys[];  // kSampKeys
  __shared__ uint64_t s_b[kMaxCoarse];
  __shared__ int s_valid;
  if (threadIdx.x == 0) s_valid = 0;
  __syncthreads();
  int mine = 0;
  for (int i = threadIdx.x; i < kSampPos; i += blockDim.x) {
    const int64_t j = (int64_t(2 * i + 1) * a.d.G) / (2 * kSampPos);
    int32_t r, f;
    const int64_t end = seq_end(a.d, j, &r, &f);
    uint64_t k[2];
    int n = windows_at(a.d, a.head, a.tail, j, end, a.kb, k);
    if (a.wt[r] == 0) n = 0;  // rules nothing references own no rows
    s_keys[2 * i] = n > 0 ? k[0] : kEmpty;
    s_keys[2 * i + 1] = n > 1 ? k[1] : kEmpty;
    mine += n;
  }
  atomicAdd(&s_valid, mine);
  __syncthreads();
  bitonic_sort_shared(s_keys, kSampKeys);
  const int nv = s_valid;
  for (int b = threadIdx.x; b < a.nspl; b += blockDim.x)
    s_b[b] = spl[b] = nv > 0 ? s_keys[int64_t(b + 1) * nv / (a.nspl + 1)] : kEmpty;
  __syncthreads();
  // prefix table: lut[p] = number of bounds below p << lut_shift, so the
  // bucket of a key with prefix p lies in [lut[p], lut[p + 1]]
  for (int p = threadIdx.x; p <= (1 << a.lut_bits); p += blockDim.x) {
    const uint64_t x = uint64_t(p) << a.lut_shift;
    int lo = 0, hi = a.nspl;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (s_b[mid] < x) lo = mid + 1;
      else hi = mid;
    }
    lut[p] = uint16_t(lo);
  }
}

// ---- 2. rows in position order, counted per (coarse bucket, CTA) -----------

// tiles [t0, t1) of CTA c of a grid of P
__device__ __forceinline__ void cta_tiles(int64_t ntiles, int64_t* t0, int64_t* t1) {
  *t0 = ntiles * blockIdx.x / gridDim.x;
  *t1 = ntiles * (blockIdx.x + 1) / gridDim.x;
}

// Windows of every tile (structure only: independent of the weights).
__global__ void __launch_bounds__(kSgThreads) sg_tile_count_kernel(DevGrammar d, const int32_t* __restrict__ head,
                                                                   const int32_t* __restrict__ tail, int kb,
                                                                   int64_t* __restrict__ tcnt) {
  TileWin t;
  uint32_t total;
  block_scan_u32<kSgThreads>(tile_windows(d, head, tail, kb, int64_t(blockIdx.x) * kTile + threadIdx.x * 4, t),
                             &total);
  if (threadIdx.x == 0) tcnt[blockIdx.x] = total;
}

// Every window of the CTA's tiles as a row (compact key, rule weight) at its
// position-order slot (tile_off + rank inside the tile); rows of rules of
// weight 0 are written with weight 0 and not counted.  cnt[b * P + c] = rows
// of bucket b from CTA c.
__global__ void __launch_bounds__(kSgThreads) sg_emit_kernel(const __grid_constant__ SgArgs a,
                                                             int64_t* __restrict__ cnt, uint64_t* __restrict__ okey,
                                                             uint32_t* __restrict__ oval) {
  __shared__ uint64_t s_spl[kMaxCoarse];
  __shared__ uint16_t s_lut[(1 << kLutBitsMax) + 1];
  __shared__ uint32_t s_hist[kMaxCoarse];
  const int nb = a.nspl + 1;
  for (int i = threadIdx.x; i < a.nspl; i += kSgThreads) s_spl[i] = a.spl[i];
  for (int i = threadIdx.x; i <= (1 << a.lut_bits); i += kSgThreads) s_lut[i] = a.lut[i];
  for (int i = threadIdx.x; i < nb; i += kSgThreads) s_hist[i] = 0;
  __syncthreads();
  int64_t t0, t1;
  cta_tiles(a.d.ntiles, &t0, &t1);
  for (int64_t tl = t0; tl < t1; ++tl) {
    TileWin t;
    uint32_t total;
    const uint32_t mine = tile_windows(a.d, a.head, a.tail, a.kb, tl * kTile + threadIdx.x * 4, t);
    // first row and weights requested before the scan's barriers
    const int64_t first = a.tile_off[tl];
    uint64_t wv[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) wv[i] = t.n[i] ? a.wt[t.r[i]] : 0;
    int64_t pos = first + block_scan_u32<kSgThreads>(mine, &total);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const uint64_t w64 = wv[i];
#pragma unroll
      for (int q = 0; q < 2; ++q)
        if (q < t.n[i]) {
          okey[pos] = t.k[i][q];
          oval[pos] = uint32_t(w64);  // weights are below 2^32 (fewer than 2^32 tokens)
          ++pos;
          if (w64 != 0) atomicAdd(&s_hist[coarse_bucket(s_spl, s_lut, a.lut_shift, t.k[i][q])], 1u);
        }
    }
  }
  __syncthreads();
  for (int b = threadIdx.x; b < nb; b += kSgThreads) cnt[int64_t(b) * gridDim.x + blockIdx.x] = s_hist[b];
}

// ---- 3. scatter into coarse buckets ---------------------------------------------

constexpr int kScTile = 4096;  // rows per step of the coarse scatter (8 per thread)

struct ScatterShared {
  uint64_t spl[kMaxCoarse];
  uint64_t base[kMaxCoarse];  // next output row of each bucket for this CTA
  uint32_t hist[kMaxCoarse];  // rows of the current step per bucket
  uint32_t start[kMaxCoarse]; // first staged row of each bucket
  uint16_t lut[(1 << kLutBitsMax) + 1];
  uint64_t key[kScTile];
  uint32_t val[kScTile];
  uint16_t bkt[kScTile];
};

// CTA c re-reads the rows it emitted (its tiles' contiguous row range) and
// writes each to its bucket's range: off[b * P + c] is the first row of
// bucket b's rows from CTA c (bucket-major exclusive scan of the counts), so
// every bucket is one contiguous range.  Rows are staged in shared memory in
// bucket order and written as runs.
__global__ void __launch_bounds__(kSgThreads) sg_scatter_kernel(const __grid_constant__ SgArgs a,
                                                                const int64_t* __restrict__ off,
                                                                const uint64_t* __restrict__ ikey,
                                                                const uint32_t* __restrict__ ival,
                                                                uint64_t* __restrict__ okey,
                                                                uint32_t* __restrict__ oval) {
  extern __shared__ __align__(16) unsigned char sg_smem[];
  ScatterShared& sh = *reinterpret_cast<ScatterShared*>(sg_smem);
  const int nb = a.nspl + 1;
  for (int i = threadIdx.x; i < a.nspl; i += kSgThreads) sh.spl[i] = a.spl[i];
  for (int i = threadIdx.x; i <= (1 << a.lut_bits); i += kSgThreads) sh.lut[i] = a.lut[i];
  for (int b = threadIdx.x; b < nb; b += kSgThreads) {
    sh.base[b] = uint64_t(off[int64_t(b) * gridDim.x + blockIdx.x]);
    sh.hist[b] = 0;
  }
  __syncthreads();
  int64_t t0, t1;
  cta_tiles(a.d.ntiles, &t0, &t1);
  const int64_t r0 = a.tile_off[t0], r1 = a.tile_off[t1];
  constexpr int kPer = kScTile / kSgThreads;
  for (int64_t s0 = r0; s0 < r1; s0 += kScTile) {
    uint64_t k[kPer];
    uint32_t w[kPer], rk[kPer];
    int bq[kPer];
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int64_t r = s0 + q * kSgThreads + threadIdx.x;
      w[q] = 0;
      if (r < r1) {
        k[q] = ikey[r];
        w[q] = ival[r];
      }
    }
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      bq[q] = -1;
      if (w[q]) {
        bq[q] = coarse_bucket(sh.spl, sh.lut, a.lut_shift, k[q]);
        rk[q] = atomicAdd(&sh.hist[bq[q]], 1u);
      }
    }
    __syncthreads();
    const uint32_t T = scan_counts<kSgThreads>(sh.hist, sh.start, nb);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kPer; ++q)
      if (bq[q] >= 0) {
        const uint32_t p = sh.start[bq[q]] + rk[q];
        sh.key[p] = k[q];
        sh.val[p] = w[q];
        sh.bkt[p] = uint16_t(bq[q]);
      }
    __syncthreads();
    for (uint32_t p = threadIdx.x; p < T; p += kSgThreads) {
      const int b = sh.bkt[p];
      const uint64_t gpos = sh.base[b] + (p - sh.start[b]);
      okey[gpos] = sh.key[p];
      oval[gpos] = sh.val[p];
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nb; b += kSgThreads) {
      sh.base[b] += sh.hist[b];
      sh.hist[b] = 0;
    }
    __syncthreads();
  }
}

// ---- 4. fine buckets -----------------------------------------------------------

__device__ __forceinline__ int fine_count(int64_t n) {
  return n <= 0 ? 0 : int(std::min<int64_t>(kMaxFine, (n + kFineRows - 1) / kFineRows));
}

// fbase[b] = first fine bucket of coarse bucket b (exclusive scan of their
// numbers), fbase[nb] = *ftot = all fine buckets.  One CTA of 1024 threads.
__global__ void __launch_bounds__(1024) sg_plan_kernel(const int64_t* __restrict__ off, int P, int nb,
                                                       int64_t* __restrict__ fbase, int64_t* __restrict__ ftot) {
  const int b = threadIdx.x;
  const uint32_t f = b < nb ? uint32_t(fine_count(off[int64_t(b + 1) * P] - off[int64_t(b) * P])) : 0u;
  uint32_t total;
  const uint32_t e = block_scan_u32<1024>(f, &total);
  if (b < nb) fbase[b] = e;
  if (b == 0) {
    fbase[nb] = total;
    *ftot = total;
  }
}

struct FineShared {
  uint64_t samp[kFineSamp];
  uint64_t fspl[kMaxFine];
  uint32_t hist[kMaxFine];
  uint32_t start[kMaxFine];
  uint32_t fstart[kMaxFine];
  uint32_t cum[kMaxFine];
  uint64_t key[kFineTile];
  uint32_t val[kFineTile];
  uint8_t fb[kFineTile];
};

// Counts one row of bucket x (x < 0: no row) in h and returns its rank among
// the rows of x counted so far.  A warp whose rows all fall in one bucket (a
// hot key) adds them with one atomic.
__device__ __forceinline__ uint32_t warp_count(uint32_t* h, int x) {
  const int lane = threadIdx.x & 31;
  const int x0 = __shfl_sync(0xffffffffu, x, 0);
  if (__all_sync(0xffffffffu, x == x0)) {
    uint32_t base = 0;
    if (lane == 0 && x0 >= 0) base = atomicAdd(&h[x0], 32u);
    return __shfl_sync(0xffffffffu, base, 0) + uint32_t(lane);
  }
  return x >= 0 ? atomicAdd(&h[x], 1u) : 0u;
}

// One CTA per coarse bucket b (rows [off[b*P], off[(b+1)*P]) of ikey/ival):
// bounds of its fine buckets from a sorted sample of its rows, rows counted
// per fine bucket, fine bucket descriptors written at fbase[b] (key order),
// rows scattered into ranges of okey/oval that mirror the coarse range.
__global__ void __launch_bounds__(kSgThreads) sg_fine_kernel(const int64_t* __restrict__ off, int P,
                                                             const int64_t* __restrict__ fbase,
                                                             const uint64_t* __restrict__ ikey,
                                                             const uint32_t* __restrict__ ival,
                                                             uint64_t* __restrict__ okey, uint32_t* __restrict__ oval,
                                                             uint8_t* __restrict__ fbkt,
                                                             int64_t* __restrict__ fd_start,
                                                             int64_t* __restrict__ fd_n) {
  extern __shared__ __align__(16) unsigned char sg_smem[];
  FineShared& sh = *reinterpret_cast<FineShared*>(sg_smem);
  const int b = blockIdx.x;
  const int64_t start = off[int64_t(b) * P];
  const int64_t n = off[int64_t(b + 1) * P] - start;
  if (n <= 0) return;
  const int f = fine_count(n), nsp = f - 1;
  const int64_t fb0 = fbase[b];
  if (nsp > 0) {
    const int s = int(std::min<int64_t>(n, kFineSamp));
    for (int i = threadIdx.x; i < kFineSamp; i += kSgThreads)
      sh.samp[i] = i < s ? ikey[start + int64_t(i) * n / s] : kEmpty;
    __syncthreads();
    bitonic_sort_shared(sh.samp, kFineSamp);
    for (int i = threadIdx.x; i < nsp; i += kSgThreads) sh.fspl[i] = sh.samp[int64_t(i + 1) * s / f];
  }
  for (int i = threadIdx.x; i < kMaxFine; i += kSgThreads) {
    sh.hist[i] = 0;
    sh.cum[i] = 0;
  }
  __syncthreads();
  // rows per fine bucket, kPer loads in flight per thread; each row's bucket
  // is kept (one byte) for the scatter
  constexpr int kPer = kFineTile / kSgThreads;
  for (int64_t t0 = 0; t0 < n; t0 += kFineTile) {
    uint64_t k[kPer];
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int64_t r = t0 + q * kSgThreads + threadIdx.x;
      k[q] = r < n ? ikey[start + r] : kEmpty;
    }
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int64_t r = t0 + q * kSgThreads + threadIdx.x;
      const int x = k[q] != kEmpty ? upper_bound_u64(sh.fspl, nsp, k[q]) : -1;
      if (x >= 0) fbkt[start + r] = uint8_t(x);
      warp_count(sh.hist, x);
    }
  }
  __syncthreads();
  scan_counts<kSgThreads>(sh.hist, sh.fstart, f);
  __syncthreads();
  for (int i = threadIdx.x; i < f; i += kSgThreads) {
    fd_start[fb0 + i] = start + sh.fstart[i];
    fd_n[fb0 + i] = sh.hist[i];
    sh.hist[i] = 0;
  }
  __syncthreads();
  for (int64_t t0 = 0; t0 < n; t0 += kFineTile) {
    uint64_t k[kPer];
    uint32_t v[kPer], rk[kPer];
    int x[kPer];
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int64_t r = t0 + q * kSgThreads + threadIdx.x;
      x[q] = -1;
      if (r < n) {
        k[q] = ikey[start + r];
        v[q] = ival[start + r];
        x[q] = fbkt[start + r];
      }
    }
#pragma unroll
    for (int q = 0; q < kPer; ++q) rk[q] = warp_count(sh.hist, x[q]);
    __syncthreads();
    const uint32_t T = scan_counts<kSgThreads>(sh.hist, sh.start, f);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kPer; ++q)
      if (x[q] >= 0) {
        const uint32_t p = sh.start[x[q]] + rk[q];
        sh.key[p] = k[q];
        sh.val[p] = v[q];
        sh.fb[p] = uint8_t(x[q]);
      }
    __syncthreads();
    for (uint32_t p = threadIdx.x; p < T; p += kSgThreads) {
      const int y = sh.fb[p];
      const int64_t g = start + sh.fstart[y] + sh.cum[y] + (p - sh.start[y]);
      okey[g] = sh.key[p];
      oval[g] = sh.val[p];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < f; i += kSgThreads) {
      sh.cum[i] += sh.hist[i];
      sh.hist[i] = 0;
    }
    __syncthreads();
  }
}

// ---- 5. reduce each fine bucket, in key order ----------------------------------

constexpr int kRdThreads = 512;
constexpr int kRdWarps = kRdThreads / 32;
constexpr int kRdSlots = 4096;         // shared-memory hash slots (power of two)
constexpr int kRdCapMax = 3072;        // distinct keys per bucket kept in shared memory (75% load)
constexpr int kSub = 256;              // sub-buckets of the shared-memory sample sort
constexpr int kThreadBin = 16;         // sub-buckets up to this size: insertion sort by one thread
constexpr int kWarpBin = 256;          // up to this size: bitonic network by one warp (8 keys per lane)
constexpr int kMaxBig = kSub;

struct ReduceShared {
  uint64_t tkey[kRdSlots];  // hash table, then the second sort buffer
  uint32_t tcnt[kRdSlots];
  uint64_t xkey[kRdSlots];  // distinct keys compacted, first sort buffer
  uint32_t xcnt[kRdSlots];
  union {
    uint16_t wcnt[kRdWarps][256];  // radix sort: per-warp digit counts, then their prefix over warps
    struct {
      uint64_t spl[kSub];          // sample sort: sampled keys, sorted in place into splitters
      uint32_t hist[kSub];         // keys per sub-bucket
      uint32_t start[kSub];        // first slot of each sub-bucket
      uint32_t cursor[kSub];       // next free slot
    } ss;
  };
  uint32_t big_start[kMaxBig];     // bins too large for one thread, finished afterwards
  uint32_t big_len[kMaxBig];
  uint32_t nbig, nmid;
  uint32_t dstart[256];          // first output slot of each digit
  uint32_t dtot[256];
  unsigned long long kmin, kmax;
  int64_t item, prefix;
  uint32_t heads, carry_w;
  int over, ok;
};

struct ReduceArgs {
  const uint64_t* key;  // rows grouped by fine bucket
  const uint32_t* val;
  uint64_t* skey;       // scratch rows (same indexing), for buckets sorted in global memory
  uint32_t* sval;
  const int64_t* fd_start;
  const int64_t* fd_n;
  const int64_t* ftot;
  unsigned long long* flags;   // look-back words, one per fine bucket, zeroed
  unsigned long long* ticket;  // next fine bucket to take, zeroed
  uint64_t* out_key;
  uint64_t* out_cnt;
  int64_t* out_len;
  int64_t cap_rows;            // room of out_key / out_cnt
  unsigned* status;
  int kb;
  int cap;                     // distinct keys handled in shared memory (<= kRdCapMax)
};


// The bucket's count, published as soon as it is known (one thread); bucket
// 0 publishes its inclusive prefix directly.
__device__ __forceinline__ void publish_count(const ReduceArgs& a, int64_t item, uint64_t agg) {
  publish_aggregate(a.flags, item, agg);
}

__device__ int64_t look_back(const ReduceArgs& a, int64_t item, uint64_t agg) {
  return warp_look_back(a.flags, item, agg, a.status);
}

constexpr int kProbeLimit = 128;  // a longer probe sequence sends the bucket to global memory

// Adds weight w to key in the shared table (linear probing).  A probe
// sequence longer than kProbeLimit marks the bucket as too large for the
// table (the table is then abandoned for the global-memory path).
__device__ __forceinline__ void table_add(ReduceShared& sh, uint64_t key, uint32_t w) {
  uint32_t h = uint32_t((key * 0x9E3779B97F4A7C15ull) >> 52);  // 12 bits: kRdSlots
  for (int probe = 0; probe < kProbeLimit; ++probe) {
    const unsigned long long prev = atomicCAS(reinterpret_cast<unsigned long long*>(&sh.tkey[h]), kEmpty, key);
    if (prev == kEmpty || prev == key) {
      atomicAdd(&sh.tcnt[h], w);
      return;
    }
    h = (h + 1) & (kRdSlots - 1);
  }
  sh.over = 1;
}

// Stable LSD sort of (k0, c0)[0, n) on bits [0, nbits), 8-bit digits, ping-
// pong with (k1, c1).  Warp w ranks the w-th slice, 32 rows per step, by one
// ballot per digit bit.  Returns which buffer holds the result (0: k0).
constexpr int kSortSteps = (kRdCapMax + kRdWarps * 32 - 1) / (kRdWarps * 32);  // 32-row steps per warp

__device__ int shared_radix_sort(ReduceShared& sh, uint64_t* k0, uint32_t* c0, uint64_t* k1, uint32_t* c1, int n,
                                 int nbits) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const int seg = ((n + kRdWarps - 1) / kRdWarps + 31) & ~31;  // n <= kRdCapMax: at most kSortSteps steps
  const int lo = min(n, warp * seg), hi = min(n, lo + seg);
  int cur = 0;
  for (int shift = 0; shift < nbits; shift += 8) {
    const uint64_t* sk = cur ? k1 : k0;
    const uint32_t* sc = cur ? c1 : c0;
    uint64_t* dk = cur ? k0 : k1;
    uint32_t* dc = cur ? c0 : c1;
    for (int i = threadIdx.x; i < kRdWarps * 256; i += kRdThreads) (&sh.wcnt[0][0])[i] = 0;
    __syncthreads();
    // rank of each row among the warp's earlier rows of its digit (kept for the scatter)
    uint16_t rk[kSortSteps];
    uint8_t dgs[kSortSteps];
#pragma unroll
    for (int st = 0; st < kSortSteps; ++st) {
      const int b = lo + st * 32;
      if (b >= hi) break;  // warp-uniform
      const int i = b + lane;
      const bool v = i < hi;
      const uint32_t dg = v ? uint32_t(sk[i] >> shift) & 255u : 0u;
      const unsigned peers = warp_digit_peers(dg, __ballot_sync(0xffffffffu, v));
      const uint16_t before = sh.wcnt[warp][dg];
      rk[st] = uint16_t(before + __popc(peers & lt));
      dgs[st] = uint8_t(dg);
      __syncwarp();
      if (v && lane == __ffs(peers) - 1) sh.wcnt[warp][dg] = uint16_t(before + __popc(peers));
      __syncwarp();
    }
    __syncthreads();
    uint32_t tot = 0;
    if (threadIdx.x < 256)
      for (int w = 0; w < kRdWarps; ++w) {
        const uint32_t c = sh.wcnt[w][threadIdx.x];
        sh.wcnt[w][threadIdx.x] = uint16_t(tot);
        tot += c;
      }
    uint32_t all;
    const uint32_t e = block_scan_u32<kRdThreads>(tot, &all);
    if (threadIdx.x < 256) sh.dstart[threadIdx.x] = e;
    __syncthreads();
#pragma unroll
    for (int st = 0; st < kSortSteps; ++st) {
      const int i = lo + st * 32 + lane;
      if (lo + st * 32 >= hi) break;
      if (i < hi) {
        const uint32_t p = sh.dstart[dgs[st]] + sh.wcnt[warp][dgs[st]] + rk[st];
        dk[p] = sk[i];
        dc[p] = sc[i];
      }
    }
    __syncthreads();
    cur ^= 1;
  }
  return cur;
}

// Bitonic sort of up to 32 * E (key, count) pairs by one warp, E per lane
// in registers (lane l holds positions E l .. E l + E - 1); missing positions
// are padded with kEmpty and sort last.
template <int E>
__device__ void warp_bitonic_sort(uint64_t* k, uint32_t* c, int n) {
  const int lane = threadIdx.x & 31;
  uint64_t rk[E];
  uint32_t rc[E];
#pragma unroll
  for (int i = 0; i < E; ++i) {
    const int e = lane * E + i;
    rk[i] = e < n ? k[e] : kEmpty;
    rc[i] = e < n ? c[e] : 0u;
  }
#pragma unroll
  for (int kk = 2; kk <= 32 * E; kk <<= 1) {
#pragma unroll
    for (int j = kk >> 1; j > 0; j >>= 1) {
      if (j >= E) {  // partner in lane ^ (j / E), same register
#pragma unroll
        for (int i = 0; i < E; ++i) {
          const int e = lane * E + i;
          const uint64_t ok = __shfl_xor_sync(0xffffffffu, rk[i], j / E);
          const uint32_t oc = __shfl_xor_sync(0xffffffffu, rc[i], j / E);
          const bool keep_min = ((e & j) == 0) == ((e & kk) == 0);
          if (keep_min ? ok < rk[i] : ok > rk[i]) {
            rk[i] = ok;
            rc[i] = oc;
          }
        }
      } else {  // partner in this lane's registers
#pragma unroll
        for (int i = 0; i < E; ++i) {
          const int p = i ^ j;
          if (p > i) {
            const int e = lane * E + i;
            const bool up = (e & kk) == 0;
            if ((rk[i] > rk[p]) == up) {
              const uint64_t tk = rk[i];
              rk[i] = rk[p];
              rk[p] = tk;
              const uint32_t tc = rc[i];
              rc[i] = rc[p];
              rc[p] = tc;
            }
          }
        }
      }
    }
  }
#pragma unroll
  for (int i = 0; i < E; ++i) {
    const int e = lane * E + i;
    if (e < n) {
      k[e] = rk[i];
      c[e] = rc[i];
    }
  }
}

// Ascending sort of the d distinct keys (xkey, xcnt)[0, d) into (tkey,
// tcnt)[0, d) (the table's storage, no longer needed).  Sample sort: kSub
// keys at evenly spaced positions of the hash-ordered array are sorted by a
// CTA bitonic network and their upper kSub - 1 become splitters; every key
// goes to its sub-bucket (about d / kSub keys each, whatever the key
// values), and each sub-bucket is finished where it lies: up to kThreadBin
// keys by one thread (insertion sort), up to 32 by one warp (one key per
// lane), up to kWarpBin by one warp (eight per lane), larger ones by the
// whole CTA (LSD radix, the (xkey, xcnt) range of the sub-bucket as scratch).
__device__ void sample_sort_shared(ReduceShared& sh, int d) {
  const int tid = threadIdx.x, warp = tid >> 5;
  if (d <= kWarpBin) {
    for (int i = tid; i < d; i += kRdThreads) {
      sh.tkey[i] = sh.xkey[i];
      sh.tcnt[i] = sh.xcnt[i];
    }
    __syncthreads();
    if (warp == 0) {
      if (d <= 32) warp_bitonic_sort<1>(sh.tkey, sh.tcnt, d);
      else warp_bitonic_sort<8>(sh.tkey, sh.tcnt, d);
    }
    __syncthreads();
    return;
  }
  if (tid < kSub) {
    sh.ss.spl[tid] = sh.xkey[int64_t(tid) * d / kSub];
    sh.ss.hist[tid] = 0;
  }
  if (tid == 0) {
    sh.nbig = 0;
    sh.nmid = 0;
  }
  __syncthreads();
  for (int kk = 2; kk <= kSub; kk <<= 1)  // bitonic network over the sample, kSub / 2 pairs per stage
    for (int j = kk >> 1; j > 0; j >>= 1) {
      if (tid < kSub / 2) {
        const int i = 2 * j * (tid / j) + (tid % j), p = i + j;
        const uint64_t x = sh.ss.spl[i], y = sh.ss.spl[p];
        if ((x > y) == ((i & kk) == 0)) {
          sh.ss.spl[i] = y;
          sh.ss.spl[p] = x;
        }
      }
      __syncthreads();
    }
  constexpr int kPer = (kRdCapMax + kRdThreads - 1) / kRdThreads;
  uint8_t bq[kPer];
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    const int i = tid + q * kRdThreads;
    if (i < d) {
      bq[q] = uint8_t(upper_bound_u64(sh.ss.spl + 1, kSub - 1, sh.xkey[i]));
      atomicAdd(&sh.ss.hist[bq[q]], 1u);
    }
  }
  __syncthreads();
  uint32_t total;
  const uint32_t e = block_scan_u32<kRdThreads>(tid < kSub ? sh.ss.hist[tid] : 0u, &total);
  if (tid < kSub) {
    sh.ss.start[tid] = e;
    sh.ss.cursor[tid] = e;
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    const int i = tid + q * kRdThreads;
    if (i < d) {
      const uint32_t p = atomicAdd(&sh.ss.cursor[bq[q]], 1u);
      sh.tkey[p] = sh.xkey[i];
      sh.tcnt[p] = sh.xcnt[i];
    }
  }
  __syncthreads();
  if (tid < kSub) {
    const uint32_t s = sh.ss.start[tid], n = sh.ss.hist[tid];
    if (n > uint32_t(kThreadBin)) {  // to a warp (or the CTA)
      const uint32_t b = n > 32u ? atomicAdd(&sh.nbig, 1u) : kSub - 1 - atomicAdd(&sh.nmid, 1u);
      sh.big_start[b] = s;
      sh.big_len[b] = n;
    } else {
      for (uint32_t i = s + 1; i < s + n; ++i) {
        const uint64_t k = sh.tkey[i];
        const uint32_t c = sh.tcnt[i];
        uint32_t j = i;
        while (j > s && sh.tkey[j - 1] > k) {
          sh.tkey[j] = sh.tkey[j - 1];
          sh.tcnt[j] = sh.tcnt[j - 1];
          --j;
        }
        sh.tkey[j] = k;
        sh.tcnt[j] = c;
      }
    }
  }
  __syncthreads();
  const int nbig = int(sh.nbig), nmid = int(sh.nmid);  // big from the front, mid from the back
  for (int b = warp; b < nmid; b += kRdWarps) {
    const int x = kSub - 1 - b;
    warp_bitonic_sort<1>(sh.tkey + sh.big_start[x], sh.tcnt + sh.big_start[x], int(sh.big_len[x]));
  }
  for (int b = warp; b < nbig; b += kRdWarps) {  // the smallest network that holds the sub-bucket
    const uint32_t n = sh.big_len[b];
    uint64_t* k = sh.tkey + sh.big_start[b];
    uint32_t* c = sh.tcnt + sh.big_start[b];
    if (n <= 64) warp_bitonic_sort<2>(k, c, int(n));
    else if (n <= 128) warp_bitonic_sort<4>(k, c, int(n));
    else if (n <= uint32_t(kWarpBin)) warp_bitonic_sort<8>(k, c, int(n));
  }
  __syncthreads();
  for (int b = 0; b < nbig; ++b) {  // CTA-uniform
    const uint32_t s = sh.big_start[b], n = sh.big_len[b];
    if (n <= uint32_t(kWarpBin)) continue;
    const int cur = shared_radix_sort(sh, sh.tkey + s, sh.tcnt + s, sh.xkey + s, sh.xcnt + s, int(n), 64);
    if (cur) {
      for (uint32_t i = tid; i < n; i += kRdThreads) {
        sh.tkey[s + i] = sh.xkey[s + i];
        sh.tcnt[s + i] = sh.xcnt[s + i];
      }
      __syncthreads();
    }
  }
}

// A bucket with more distinct keys than the shared table holds: its rows are
// sorted in global memory (stable LSD radix, 8-bit digits, between the
// bucket's rows and the same range of the scratch rows), then each run of
// equal keys becomes one output row.  Every thread of the CTA takes part.
__device__ void reduce_in_global(const ReduceArgs& a, ReduceShared& sh, int64_t item, int64_t start, int64_t n) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  uint64_t* k0 = const_cast<uint64_t*>(a.key) + start;
  uint32_t* c0 = const_cast<uint32_t*>(a.val) + start;
  uint64_t* k1 = a.skey + start;
  uint32_t* c1 = a.sval + start;
  if (threadIdx.x == 0) {
    sh.kmin = kEmpty;
    sh.kmax = 0;
  }
  __syncthreads();
  for (int64_t r = threadIdx.x; r < n; r += kRdThreads) {
    atomicMin(&sh.kmin, (unsigned long long)k0[r]);
    atomicMax(&sh.kmax, (unsigned long long)k0[r]);
  }
  __syncthreads();
  const int nbits = sh.kmin == sh.kmax ? 0 : 64 - __clzll((long long)(sh.kmin ^ sh.kmax));
  int cur = 0;
  for (int shift = 0; shift < nbits; shift += 8) {
    const uint64_t* sk = cur ? k1 : k0;
    const uint32_t* sc = cur ? c1 : c0;
    uint64_t* dk = cur ? k0 : k1;
    uint32_t* dc = cur ? c0 : c1;
    for (int i = threadIdx.x; i < 256; i += kRdThreads) sh.dtot[i] = 0;
    __syncthreads();
    for (int64_t r = threadIdx.x; r < n; r += kRdThreads) atomicAdd(&sh.dtot[uint32_t(sk[r] >> shift) & 255u], 1u);
    __syncthreads();
    uint32_t all;
    const uint32_t e = block_scan_u32<kRdThreads>(threadIdx.x < 256 ? sh.dtot[threadIdx.x] : 0u, &all);
    if (threadIdx.x < 256) sh.dstart[threadIdx.x] = e;
    __syncthreads();
    for (int64_t t0 = 0; t0 < n; t0 += kRdThreads) {  // rows in order, one per thread
      for (int i = threadIdx.x; i < kRdWarps * 256; i += kRdThreads) (&sh.wcnt[0][0])[i] = 0;
      __syncthreads();
      const int64_t r = t0 + threadIdx.x;
      const bool v = r < n;
      const uint32_t dg = v ? uint32_t(sk[r] >> shift) & 255u : 0u;
      const unsigned peers = warp_digit_peers(dg, __ballot_sync(0xffffffffu, v));
      if (v && lane == __ffs(peers) - 1) sh.wcnt[warp][dg] = uint16_t(__popc(peers));
      __syncthreads();
      if (threadIdx.x < 256) {
        uint32_t run = 0;
        for (int w = 0; w < kRdWarps; ++w) {
          const uint32_t c = sh.wcnt[w][threadIdx.x];
          sh.wcnt[w][threadIdx.x] = uint16_t(run);
          run += c;
        }
        sh.dtot[threadIdx.x] = run;
      }
      __syncthreads();
      if (v) {
        const uint64_t p = sh.dstart[dg] + sh.wcnt[warp][dg] + __popc(peers & lt);
        dk[p] = sk[r];
        dc[p] = sc[r];
      }
      __syncthreads();
      if (threadIdx.x < 256) sh.dstart[threadIdx.x] += sh.dtot[threadIdx.x];
      __syncthreads();
    }
    cur ^= 1;
  }
  const uint64_t* sk = cur ? k1 : k0;
  const uint32_t* sc = cur ? c1 : c0;
  // distinct keys = run heads
  if (threadIdx.x == 0) sh.heads = 0;
  __syncthreads();
  uint32_t h = 0;
  for (int64_t r = threadIdx.x; r < n; r += kRdThreads) h += (r == 0 || sk[r] != sk[r - 1]);
  atomicAdd(&sh.heads, h);
  __syncthreads();
  const uint32_t d = sh.heads;
  __syncthreads();
  if (threadIdx.x < 32) {
    if (threadIdx.x == 0) publish_count(a, item, d);
    const int64_t pre = look_back(a, item, d);
    if (threadIdx.x == 0) {
      sh.prefix = pre;
      if (pre >= 0 && pre + int64_t(d) > a.cap_rows) {
        atomicOr(a.status, ST_OVERFLOW);
        sh.prefix = -1;
      }
      sh.heads = 0;    // heads before the current tile
      sh.carry_w = 0;  // weights before the current tile
    }
  }
  __syncthreads();
  const int64_t prefix = sh.prefix;
  if (prefix >= 0) {
    // the count of a run is the running weight sum at its last row minus that
    // at the last row of the previous run: first store the running sums ...
    for (int64_t t0 = 0; t0 < n; t0 += kRdThreads) {
      const int64_t r = t0 + threadIdx.x;
      const bool v = r < n;
      const uint64_t k = v ? sk[r] : 0;
      const uint32_t w = v ? sc[r] : 0u;
      const uint32_t head = v && (r == 0 || k != sk[r - 1]);
      const bool last = v && (r == n - 1 || k != sk[r + 1]);
      uint32_t ht, wt;
      const uint32_t he = block_scan_u32<kRdThreads>(head, &ht);
      const uint32_t we = block_scan_u32<kRdThreads>(w, &wt);
      if (last) {
        const int64_t o = prefix + sh.heads + he + head - 1;
        a.out_key[o] = to_output_key(k, a.kb);
        a.out_cnt[o] = uint64_t(sh.carry_w + we + w);
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        sh.heads += ht;
        sh.carry_w += wt;
      }
      __syncthreads();
    }
    // ... then turn them into differences, keeping each step's last sum
    if (threadIdx.x == 0) sh.carry_w = 0;
    __syncthreads();
    for (int64_t t0 = 0; t0 < d; t0 += kRdThreads) {
      const int64_t i = t0 + threadIdx.x;
      const uint64_t cum = i < d ? a.out_cnt[prefix + i] : 0;
      const uint64_t before = i == t0 ? sh.carry_w : (i < d ? a.out_cnt[prefix + i - 1] : 0);
      __syncthreads();
      if (i < d) a.out_cnt[prefix + i] = cum - before;
      if (i == std::min<int64_t>(d, t0 + kRdThreads) - 1) sh.carry_w = uint32_t(cum);
      __syncthreads();
    }
  }
  if (threadIdx.x == 0 && item == *a.ftot - 1 && prefix >= 0) *a.out_len = prefix + d;
}

__global__ void __launch_bounds__(kRdThreads, 2) sg_reduce_kernel(const __grid_constant__ ReduceArgs a) {
  extern __shared__ __align__(16) unsigned char sg_smem[];
  ReduceShared& sh = *reinterpret_cast<ReduceShared*>(sg_smem);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t ftot = *a.ftot;
  while (true) {
    if (threadIdx.x == 0) sh.item = int64_t(atomicAdd(a.ticket, 1ull));
    for (int i = threadIdx.x; i < kRdSlots; i += kRdThreads) {
      sh.tkey[i] = kEmpty;
      sh.tcnt[i] = 0;
    }
    if (threadIdx.x == 0) {
      sh.over = 0;
      sh.kmin = kEmpty;
      sh.kmax = 0;
    }
    __syncthreads();
    const int64_t item = sh.item;
    if (item >= ftot) break;
    const int64_t start = a.fd_start[item], n = a.fd_n[item];
    // sum the weights of equal keys in the table; a warp whose rows all carry
    // one key (a hot 3-gram) adds them with one update
    for (int64_t r0 = 0; r0 < n; r0 += kRdThreads) {
      const int64_t r = r0 + threadIdx.x;
      const bool v = r < n;
      const uint64_t key = v ? a.key[start + r] : kEmpty;
      uint32_t w = v ? a.val[start + r] : 0u;
      const uint64_t k0 = __shfl_sync(0xffffffffu, key, 0);
      if (__all_sync(0xffffffffu, !v || key == k0)) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
        if (lane == 0 && k0 != kEmpty && !sh.over) table_add(sh, k0, w);
      } else if (v && !sh.over) {
        table_add(sh, key, w);
      }
    }
    __syncthreads();
    // distinct keys in slot order into the first sort buffer; their number
    // by a scan (no shared counter on the insert path)
    constexpr int kPer = kRdSlots / kRdThreads;
    uint32_t c = 0;
#pragma unroll
    for (int q = 0; q < kPer; ++q) c += sh.tkey[threadIdx.x * kPer + q] != kEmpty;
    uint32_t d;
    uint32_t o = block_scan_u32<kRdThreads>(c, &d);
    if (sh.over || d >= uint32_t(a.cap)) {  // too many distinct keys for the shared path
      reduce_in_global(a, sh, item, start, n);
      __syncthreads();
      continue;
    }
    if (threadIdx.x == 0) publish_count(a, item, d);
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int s = threadIdx.x * kPer + q;
      if (sh.tkey[s] != kEmpty) {
        sh.xkey[o] = sh.tkey[s];
        sh.xcnt[o] = sh.tcnt[s];
        ++o;
      }
    }
    __syncthreads();
    sample_sort_shared(sh, int(d));
    const uint64_t* sk = sh.tkey;
    const uint32_t* sc = sh.tcnt;
    if (warp == 0) {
      const int64_t pre = look_back(a, item, d);
      if (lane == 0) {
        sh.prefix = pre;
        if (pre >= 0 && pre + int64_t(d) > a.cap_rows) {
          atomicOr(a.status, ST_OVERFLOW);
          sh.prefix = -1;
        }
        if (item == ftot - 1 && sh.prefix >= 0) *a.out_len = sh.prefix + d;
      }
    }
    __syncthreads();
    const int64_t prefix = sh.prefix;
    if (prefix >= 0)
      for (int i = threadIdx.x; i < int(d); i += kRdThreads) {
        a.out_key[prefix + i] = to_output_key(sk[i], a.kb);
        a.out_cnt[prefix + i] = sc[i];
      }
    __syncthreads();
  }
}

}  // namespace

// Row offsets of every tile (the tile's first owned window in position
// order), built once per grammar; later calls on other streams wait for it.
const int64_t* seq_tile_offsets(gt_grammar* g, const int32_t* head, const int32_t* tail, int kb, cudaStream_t s) {
  std::lock_guard<std::mutex> lk(g->seq_mu);
  if (g->seq_tile_off) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    GT_CUDA(cudaStreamIsCapturing(s, &cap));
    if (cap == cudaStreamCaptureStatusNone) GT_CUDA(cudaStreamWaitEvent(s, g->seq_tile_ev, 0));
    return g->seq_tile_off;
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  GT_CUDA(cudaStreamIsCapturing(s, &cap));
  if (cap != cudaStreamCaptureStatusNone)  // they live as long as the grammar, not as a graph
    fail(GT_EINVAL, "run the global sequence count once outside stream capture before capturing it");
  const int64_t nt = g->d.ntiles;
  auto* off = static_cast<int64_t*>(grammar_alloc(g, size_t(nt + 1) * 8, s));
  Buf cnt(g->ctx, size_t(nt + 1) * 8, s), sc(g->ctx, scan_scratch_bytes(nt + 1), s);
  GT_CUDA(cudaMemsetAsync(cnt.as<int64_t>() + nt, 0, 8, s));
  sg_tile_count_kernel<<<unsigned(nt), kSgThreads, 0, s>>>(g->d, head, tail, kb, cnt.as<int64_t>());
  GT_LAUNCH_CHECK();
  exclusive_scan_i64(cnt.as<int64_t>(), off, nt + 1, sc.p, s);
  cudaEvent_t ev;
  GT_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  GT_CUDA(cudaEventRecord(ev, s));
  g->seq_tile_ev = ev;
  g->seq_tile_off = off;
  return off;
}

gt_result* run_sequence_count_global(gt_grammar* g, cudaStream_t s) {
  gt_ctx* ctx = g->ctx;
  const DevGrammar& d = g->d;
  if (d.V > (1 << 21)) fail(GT_EOVERFLOW, "3-word keys need num_words <= 2^21");
  if (d.N >= (uint64_t(1) << 32)) fail(GT_EOVERFLOW, "sequence count needs fewer than 2^32 tokens per grammar");
  int kb = 1;  // bits per word id
  while ((int64_t(1) << kb) <= std::max<int64_t>(d.V - 1, 1)) ++kb;
  ResultBuilder rb(ctx, s);
  const int64_t U = g->info.owned_windows;  // rows at most (rules of weight 0 own none)
  auto* okey = static_cast<uint64_t*>(rb.alloc(size_t(U) * 8));
  auto* ocnt = static_cast<uint64_t*>(rb.alloc(size_t(U) * 8));
  int64_t* len = rb.new_len_slot();
  rb.field_dyn("key", okey, len);
  rb.field_dyn("count", ocnt, len);
  if (U == 0 || d.G == 0) return rb.finish();

  Buf head(ctx, size_t(d.R) * 8, s), tail(ctx, size_t(d.R) * 8, s), wt(ctx, size_t(d.R) * 8, s);
  {
    Phase ph(ctx, "seq_headtail", s);
    run_head_tail(g, head.as<int32_t>(), tail.as<int32_t>(), s);
    run_rule_weights(g, wt.as<uint64_t>(), s);
  }
  const int nb = int(std::min<int64_t>(kMaxCoarse, std::max<int64_t>(1, (U + kCoarseRows - 1) / kCoarseRows)));
  const int P = int(std::min<int64_t>(d.ntiles, 2 * ctx->num_sms));
  const int64_t ncnt = int64_t(nb) * P + 1;
  const int64_t fmax = U / kFineRows + nb + 1;  // fine buckets at most
  const int lut_bits = std::min(kLutBitsMax, 3 * kb);
  Buf spl(ctx, size_t(nb) * 8, s), lut(ctx, size_t((1 << lut_bits) + 1) * 2, s);
  Buf cnt(ctx, size_t(ncnt) * 8, s), off(ctx, size_t(ncnt) * 8, s);
  Buf sc(ctx, scan_scratch_bytes(ncnt), s), fbase(ctx, size_t(nb + 1) * 8, s);
  // rows: emitted in position order into (ke, ve), scattered by coarse bucket
  // into (ka, va), by fine bucket back into (ke, ve); (ka, va) is then the
  // reduction's scratch
  Buf ke(ctx, size_t(U) * 8, s), ve(ctx, size_t(U) * 4, s), ka(ctx, size_t(U) * 8, s), va(ctx, size_t(U) * 4, s);
  // fine bucket descriptors, then the look-back words, the ticket and the
  // number of fine buckets, cleared with one memset
  Buf fd(ctx, size_t(fmax) * 16, s), lb(ctx, size_t(fmax + 2) * 8, s);
  auto* fd_start = fd.as<int64_t>();
  auto* fd_n = fd_start + fmax;
  auto* flags = lb.as<unsigned long long>();
  auto* ticket = flags + fmax;
  auto* ftot = reinterpret_cast<int64_t*>(flags + fmax + 1);
  GT_CUDA(cudaMemsetAsync(lb.p, 0, size_t(fmax + 2) * 8, s));
  SgArgs a{d, head.as<int32_t>(), tail.as<int32_t>(), wt.as<uint64_t>(), spl.as<uint64_t>(), lut.as<uint16_t>(),
           nullptr, kb, nb - 1, lut_bits, 3 * kb - lut_bits};
  {
    Phase ph(ctx, "seq_part", s);
    a.tile_off = seq_tile_offsets(g, head.as<int32_t>(), tail.as<int32_t>(), kb, s);
    if (nb > 1) {
      const int smem = kSampKeys * 8;
      GT_CUDA(cudaFuncSetAttribute(sg_bounds_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
      sg_bounds_kernel<<<1, 1024, smem, s>>>(a, spl.as<uint64_t>(), lut.as<uint16_t>());
      GT_LAUNCH_CHECK();
    } else {
      GT_CUDA(cudaMemsetAsync(lut.p, 0, size_t((1 << lut_bits) + 1) * 2, s));  // one bucket, no bounds
    }
    GT_CUDA(cudaMemsetAsync(cnt.as<int64_t>() + ncnt - 1, 0, 8, s));
    sg_emit_kernel<<<P, kSgThreads, 0, s>>>(a, cnt.as<int64_t>(), ke.as<uint64_t>(), ve.as<uint32_t>());
    GT_LAUNCH_CHECK();
    exclusive_scan_i64(cnt.as<int64_t>(), off.as<int64_t>(), ncnt, sc.p, s);
    sg_plan_kernel<<<1, 1024, 0, s>>>(off.as<int64_t>(), P, nb, fbase.as<int64_t>(), ftot);
    GT_LAUNCH_CHECK();
  }
  {
    Phase ph(ctx, "seq_scatter", s);
    const int smem = int(sizeof(ScatterShared));
    GT_CUDA(cudaFuncSetAttribute(sg_scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    sg_scatter_kernel<<<P, kSgThreads, smem, s>>>(a, off.as<int64_t>(), ke.as<uint64_t>(), ve.as<uint32_t>(),
                                                  ka.as<uint64_t>(), va.as<uint32_t>());
    GT_LAUNCH_CHECK();
  }
  {
    Phase ph(ctx, "seq_fine", s);
    const int smem = int(sizeof(FineShared));
    GT_CUDA(cudaFuncSetAttribute(sg_fine_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    Buf fb(ctx, size_t(U), s);  // fine bucket of every row
    sg_fine_kernel<<<nb, kSgThreads, smem, s>>>(off.as<int64_t>(), P, fbase.as<int64_t>(), ka.as<uint64_t>(),
                                                va.as<uint32_t>(), ke.as<uint64_t>(), ve.as<uint32_t>(),
                                                fb.as<uint8_t>(), fd_start, fd_n);
    GT_LAUNCH_CHECK();
  }
  {
    Phase ph(ctx, "seq_reduce", s);
    ReduceArgs ra{};
    ra.key = ke.as<uint64_t>();
    ra.val = ve.as<uint32_t>();
    ra.skey = ka.as<uint64_t>();
    ra.sval = va.as<uint32_t>();
    ra.fd_start = fd_start;
    ra.fd_n = fd_n;
    ra.ftot = ftot;
    ra.flags = flags;
    ra.ticket = ticket;
    ra.out_key = okey;
    ra.out_cnt = ocnt;
    ra.out_len = len;
    ra.cap_rows = U;
    ra.status = rb.status();
    ra.kb = kb;
    ra.cap = int(std::min<int64_t>(kRdCapMax, std::max<int64_t>(2, gparam(g, "seq_table_cap", kRdCapMax))));
    const int smem = int(sizeof(ReduceShared));
    GT_CUDA(cudaFuncSetAttribute(sg_reduce_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    sg_reduce_kernel<<<2 * ctx->num_sms, kRdThreads, smem, s>>>(ra);
    GT_LAUNCH_CHECK();
  }
  return rb.finish();
}

}  // namespace gt
