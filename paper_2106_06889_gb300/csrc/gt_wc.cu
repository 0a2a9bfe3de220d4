// Top-down rule weights, word count and head/tail buffers.
//
// Word count follows the top-down strategy of Algorithm 1: every rule gets
// its weight (how often it occurs in the full expansion), then every word
// occurrence in a rule body adds that weight to the word's count
// (reduceResultKernel).  The GB300 form:
//   * weights are pulled level by level over parent edges grouped by level
//     (no masks, no stop-flag relaunch loop);
//   * the reduction never uses global atomics, whose throughput on skewed
//     (Zipf) keys is ~20 G/s here, against ~700 G/s for atomics on a dense
//     histogram in shared memory.  It runs in three passes:
//       1. partition: every warp streams its own 512-symbol chunks with
//          16-byte vector loads (plus the rule id of every symbol past the
//          root), routes each word to its vocabulary bucket (2^14 words) and
//          writes its 14-bit index into a per-(CTA, bucket) region - 2 bytes
//          per root word, 8 bytes (index + weight) past the root;
//       2. histogram: CTA (bucket, slice) adds up one slice of a bucket's
//          regions in a dense shared-memory histogram;
//       3. reduce: each word's count is the sum of its bucket's slices.
#include <algorithm>
#include <memory>
#include <vector>

#include "gt_device.cuh"

namespace gt {
namespace {

constexpr int kBucketLog2 = 14;
constexpr int kBucket = 1 << kBucketLog2;
constexpr int kMaxBuckets = 128;  // num_words <= 2^21
constexpr int kHistThreads = 512;

// Where the partition pass writes.  Region (b, c) of CTA c for bucket b:
// plain  + (b * grid + c) * cap_p  (uint16 word index, weight 1: root tiles)
// wgt    + (b * grid + c) * cap_w  (uint64: weight << 32 | word index)
// A region that fills up spills to the overflow list (uint64: weight << 32 | word).
struct PartOut {
  uint16_t* plain;
  uint64_t* wgt;
  int64_t* cnt_p;  // [B * grid]
  int64_t* cnt_w;  // [B * grid]
  uint64_t* ovf;
  unsigned long long* ovf_n;
  int64_t cap_p, cap_w, ovf_cap;
  int nb;  // buckets in use
};

constexpr int kMaxWcJobs = 64;  // grammars per fused word-count launch

// CTA ranges of the jobs of one launch: job j owns CTAs [cta[j], cta[j+1]).
__device__ __forceinline__ int find_job(const int* cta, int n, int x) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (cta[mid] <= x) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// One grammar's slice of one level of the weight pass.
struct WtJob {
  const int32_t* lchild;
  const int32_t* lpar;
  const uint32_t* lmult;
  int64_t a, b;
  unsigned long long* wt;
};

template <int NJ>
struct WtBatch {
  WtJob job[NJ];
  int cta[NJ + 1];
  int n;
};

template <int NJ>
struct WtRoots {
  unsigned long long* wt[NJ];
  int n;
};

template <int NJ>
__global__ void wt_init_kernel(const __grid_constant__ WtRoots<NJ> r) {
  for (int j = threadIdx.x; j < r.n; j += blockDim.x) r.wt[j][0] = 1ull;
}

// Top-down weights for the children on one level: one thread per parent edge
// (edges of a level are grouped by child), mult * wt[parent] summed per child
// inside the warp, one atomic per child piece.  Parents sit on lower,
// finished levels, so every weight read is final.  A warp never spans two
// grammars: each has its own CTAs.
template <int NJ>
__global__ void wt_edges_kernel(const __grid_constant__ WtBatch<NJ> bt) {
  const int j = find_job(bt.cta, bt.n, blockIdx.x);
  const WtJob& jb = bt.job[j];
  const int cta = blockIdx.x - bt.cta[j], ncta = bt.cta[j + 1] - bt.cta[j];
  const int32_t* __restrict__ lchild = jb.lchild;
  const int32_t* __restrict__ lpar = jb.lpar;
  const uint32_t* __restrict__ lmult = jb.lmult;
  unsigned long long* __restrict__ wt = jb.wt;
  const int64_t b = jb.b;
  const int lane = threadIdx.x & 31;
  const int64_t stride = int64_t(ncta) * blockDim.x;
  for (int64_t i = jb.a + cta * int64_t(blockDim.x) + threadIdx.x; i - lane < b; i += stride) {
    const bool in = i < b;
    const int32_t c = in ? lchild[i] : -1;
    unsigned long long v = in ? (unsigned long long)lmult[i] * wt[lpar[i]] : 0ull;
    // suffix sums over equal children (children are sorted, so equal ones are adjacent)
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long u = __shfl_down_sync(0xffffffffu, v, o);
      const int32_t c2 = __shfl_down_sync(0xffffffffu, c, o);
      if (lane + o < 32 && c2 == c) v += u;
    }
    const int32_t cp = __shfl_up_sync(0xffffffffu, c, 1);
    if (in && (lane == 0 || cp != c)) atomicAdd(&wt[c], v);
  }
}

constexpr int kPartWarps = 32;
constexpr int kPartThreads = 32 * kPartWarps;
constexpr int kChunk = 512;  // symbols per warp work item: 4 int4 per lane

// One grammar's part of a (possibly multi-grammar) word-count launch.
struct WcJob {
  const int32_t* sym;
  const int32_t* sym_rule;
  const uint64_t* wt;
  uint32_t* partial;
  unsigned long long* counts;
  PartOut out;
  int64_t nchunks, first_rule_chunk;
  int32_t V;
  int grid1, K;  // partition CTAs; histogram CTAs per bucket
};

template <int NJ>
struct WcBatch {
  WcJob job[NJ];
  int part_cta[NJ + 1];  // partition CTAs of job j
  int hist_cta[NJ + 1];  // histogram CTAs (nb * K per job)
  int red_cta[NJ + 1];   // reduce CTAs
  int n;
};

struct PartShared {
  uint32_t cnt[kPartWarps][kMaxBuckets + 1];    // per-warp counts of the chunk (rows padded)
  uint32_t base[kPartWarps][kMaxBuckets + 1];   // per-warp start in the CTA region (or overflow)
  uint32_t start[kPartWarps][kMaxBuckets + 1];  // per-warp start of bucket b in the staging row
  uint32_t stage[kPartWarps][kChunk];           // chunk entries (bucket << 16 | index) in bucket order
  uint32_t cur_p[kMaxBuckets];                  // CTA region reservations, plain entries
  uint32_t cur_w[kMaxBuckets];                  // CTA region reservations, weighted entries
  uint32_t fail_p[kMaxBuckets];                 // first reservation that did not fit (entries
  uint32_t fail_w[kMaxBuckets];                 //   below it are all written)
};

// Reserve room for c entries of bucket b in the CTA's region; returns the
// start, or 0x80000000 | overflow position if the region is full.
__device__ __forceinline__ uint32_t reserve(PartShared& sh, const PartOut& out, bool past_root, int b, uint32_t c,
                                            uint32_t* status) {
  uint32_t* cur = past_root ? &sh.cur_w[b] : &sh.cur_p[b];
  const int64_t cap = past_root ? out.cap_w : out.cap_p;
  const uint32_t at = atomicAdd(cur, c);
  if (int64_t(at) + c <= cap) return at;
  atomicMin(past_root ? &sh.fail_w[b] : &sh.fail_p[b], at);
  const unsigned long long o = atomicAdd(out.ovf_n, (unsigned long long)c);
  if (o + c > (unsigned long long)out.ovf_cap) atomicOr(status, ST_TABLE_FULL);
  return 0x80000000u | uint32_t(o);  // overflow positions stay below 2^31
}

// Pass 1.  Every warp works alone on 512-symbol chunks (chunk index strided
// over all warps of the grid): it loads them with 16-byte vector loads, ranks
// each word inside (warp, bucket) and reserves room for each bucket in its
// CTA's region with one shared-memory atomic.  Root chunks are then staged in
// bucket order in shared memory and written bucket run by bucket run, so
// consecutive lanes store consecutive addresses.  No CTA-wide barrier is
// needed after set-up.
template <int NJ>
__global__ void __launch_bounds__(kPartThreads, 1)
    wc_partition_kernel(const __grid_constant__ WcBatch<NJ> bt, uint32_t* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  PartShared& sh = *reinterpret_cast<PartShared*>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int jid = find_job(bt.part_cta, bt.n, blockIdx.x);
  const WcJob& jb = bt.job[jid];
  const PartOut& out = jb.out;
  const uint64_t* __restrict__ wt = jb.wt;
  const int32_t V = jb.V;
  const int cta = blockIdx.x - bt.part_cta[jid], grid = jb.grid1;
  const int nb = out.nb;
  for (int i = tid; i < kPartWarps * (kMaxBuckets + 1); i += kPartThreads) (&sh.cnt[0][0])[i] = 0;
  for (int b = tid; b < kMaxBuckets; b += kPartThreads) {
    sh.cur_p[b] = 0;
    sh.cur_w[b] = 0;
    sh.fail_p[b] = 0xffffffffu;
    sh.fail_w[b] = 0xffffffffu;
  }
  __syncthreads();
  const int64_t nchunks = jb.nchunks;
  const int64_t first_rule_chunk = jb.first_rule_chunk;
  const int64_t gw = int64_t(grid) * kPartWarps;
  uint32_t* cnt = sh.cnt[warp];
  uint32_t* base = sh.base[warp];
  uint32_t* start = sh.start[warp];
  uint32_t* stage = sh.stage[warp];
  const int64_t reg0 = cta;
  for (int64_t ch = int64_t(cta) * kPartWarps + warp; ch < nchunks; ch += gw) {
    const bool past_root = ch >= first_rule_chunk;
    const int4* src = reinterpret_cast<const int4*>(jb.sym + ch * kChunk);
    int4 v[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] = src[j * 32 + lane];
    uint32_t rank[16];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int32_t w4[4] = {v[j].x, v[j].y, v[j].z, v[j].w};
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (uint32_t(w4[q]) < uint32_t(V)) rank[j * 4 + q] = atomicAdd(&cnt[w4[q] >> kBucketLog2], 1u);
    }
    __syncwarp();
    if (!past_root) {
      // bucket starts inside the staging row (exclusive scan over buckets) and region room
      uint32_t run = 0;
      for (int b0 = 0; b0 < nb; b0 += 32) {
        const int b = b0 + lane;
        const uint32_t c = b < nb ? cnt[b] : 0u;
        uint32_t incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += u;
        }
        if (b < nb) {
          start[b] = run + incl - c;
          cnt[b] = 0;
          if (c) base[b] = reserve(sh, out, false, b, c, status);
        }
        run += __shfl_sync(0xffffffffu, incl, 31);
      }
      __syncwarp();
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int32_t w4[4] = {v[j].x, v[j].y, v[j].z, v[j].w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int32_t w = w4[q];
          if (uint32_t(w) >= uint32_t(V)) continue;
          const int b = w >> kBucketLog2;
          stage[start[b] + rank[j * 4 + q]] = (uint32_t(b) << 16) | (uint32_t(w) & (kBucket - 1));
        }
      }
      __syncwarp();
      for (uint32_t i = lane; i < run; i += 32) {
        const uint32_t e = stage[i];
        const int b = int(e >> 16);
        const uint32_t bs = base[b];
        const uint32_t k = i - start[b];
        if (bs & 0x80000000u) {
          const int64_t pos = int64_t(bs & 0x7fffffffu) + k;
          if (pos < out.ovf_cap) out.ovf[pos] = (uint64_t(1) << 32) | ((uint32_t(b) << kBucketLog2) | (e & 0xffffu));
        } else {
          out.plain[(reg0 + int64_t(b) * grid) * out.cap_p + bs + k] = uint16_t(e);
        }
      }
    } else {
      int4 r[4];
      const int4* rsrc = reinterpret_cast<const int4*>(jb.sym_rule + (ch - first_rule_chunk) * kChunk);
#pragma unroll
      for (int j = 0; j < 4; ++j) r[j] = rsrc[j * 32 + lane];
      for (int b = lane; b < nb; b += 32) {
        const uint32_t c = cnt[b];
        if (c) {
          cnt[b] = 0;
          base[b] = reserve(sh, out, true, b, c, status);
        }
      }
      __syncwarp();
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int32_t w4[4] = {v[j].x, v[j].y, v[j].z, v[j].w};
        const int32_t r4[4] = {r[j].x, r[j].y, r[j].z, r[j].w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int32_t w = w4[q];
          if (uint32_t(w) >= uint32_t(V)) continue;
          const int b = w >> kBucketLog2;
          const uint32_t bs = base[b];
          const uint32_t weight = uint32_t(wt[r4[q]]);
          if (bs & 0x80000000u) {
            const int64_t pos = int64_t(bs & 0x7fffffffu) + rank[j * 4 + q];
            if (pos < out.ovf_cap) out.ovf[pos] = (uint64_t(weight) << 32) | uint32_t(w);
          } else {
            out.wgt[(reg0 + int64_t(b) * grid) * out.cap_w + bs + rank[j * 4 + q]] =
                (uint64_t(weight) << 32) | (uint32_t(w) & (kBucket - 1));
          }
        }
      }
    }
    __syncwarp();
  }
  __syncthreads();
  for (int b = tid; b < nb; b += kPartThreads) {
    out.cnt_p[int64_t(b) * grid + cta] = min(min(int64_t(sh.cur_p[b]), out.cap_p), int64_t(sh.fail_p[b]));
    out.cnt_w[int64_t(b) * grid + cta] = min(min(int64_t(sh.cur_w[b]), out.cap_w), int64_t(sh.fail_w[b]));
  }
}

// Pass 2.  CTA (b, k) adds the regions of partition CTAs [c0, c1) for bucket b
// - and the overflow entries of bucket b in slice k - into a dense histogram
// of the bucket's 2^14 words, then stores it as partial k of bucket b.
template <bool kAggregate, int NJ>
__global__ void __launch_bounds__(kHistThreads) wc_hist_kernel(const __grid_constant__ WcBatch<NJ> bt) {
  __shared__ uint32_t hist[kBucket];
  const int jid = find_job(bt.hist_cta, bt.n, blockIdx.x);
  const WcJob& jb = bt.job[jid];
  const PartOut& out = jb.out;
  const int grid1 = jb.grid1, K = jb.K;
  const int local = blockIdx.x - bt.hist_cta[jid];
  const int b = local / K, k = local % K;
  const int lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < kBucket; i += kHistThreads) hist[i] = 0;
  __syncthreads();
  const int c0 = int(int64_t(grid1) * k / K), c1 = int(int64_t(grid1) * (k + 1) / K);
  for (int c = c0; c < c1; ++c) {
    const int64_t region = int64_t(b) * grid1 + c;
    const int64_t n = min(out.cnt_p[region], out.cap_p);
    const uint16_t* p = out.plain + region * out.cap_p;
    // 8 entries per thread per step (cap_p is a multiple of 8, so loads stay aligned)
    for (int64_t i = int64_t(threadIdx.x) * 8; i - int64_t(lane) * 8 < n; i += int64_t(kHistThreads) * 8) {
      uint4 v = make_uint4(0, 0, 0, 0);
      if (i < n) v = *reinterpret_cast<const uint4*>(p + i);
      const uint32_t wd[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const bool ok = i + q < n;
        const uint32_t e = (wd[q >> 1] >> ((q & 1) * 16)) & 0xffffu;
        if (kAggregate) {
          const unsigned act = __ballot_sync(0xffffffffu, ok);
          if (ok) {
            const unsigned peers = __match_any_sync(act, e);
            if (lane == __ffs(peers) - 1) atomicAdd(&hist[e], uint32_t(__popc(peers)));
          }
        } else if (ok) {
          atomicAdd(&hist[e], 1u);
        }
      }
    }
    const int64_t m = min(out.cnt_w[region], out.cap_w);
    const uint64_t* pw = out.wgt + region * out.cap_w;
    for (int64_t i = threadIdx.x; i < m; i += kHistThreads) {
      const uint64_t e = pw[i];
      atomicAdd(&hist[uint32_t(e) & (kBucket - 1)], uint32_t(e >> 32));
    }
  }
  const int64_t no = int64_t(min(*out.ovf_n, (unsigned long long)out.ovf_cap));
  for (int64_t i = int64_t(k) * kHistThreads + threadIdx.x; i < no; i += int64_t(K) * kHistThreads) {
    const uint64_t e = out.ovf[i];
    const uint32_t w = uint32_t(e);
    if (int(w >> kBucketLog2) == b) atomicAdd(&hist[w & (kBucket - 1)], uint32_t(e >> 32));
  }
  __syncthreads();
  uint32_t* dst = jb.partial + int64_t(local) * kBucket;
  for (int i = threadIdx.x; i < kBucket; i += kHistThreads) dst[i] = hist[i];
}

// Pass 3: counts[w] = sum of the K partials of w's bucket.
constexpr int kReduceThreads = 256;

template <int NJ>
__global__ void __launch_bounds__(kReduceThreads) wc_reduce_kernel(const __grid_constant__ WcBatch<NJ> bt) {
  const int jid = find_job(bt.red_cta, bt.n, blockIdx.x);
  const WcJob& jb = bt.job[jid];
  const int K = jb.K;
  const int64_t w = int64_t(blockIdx.x - bt.red_cta[jid]) * kReduceThreads + threadIdx.x;
  if (w >= jb.V) return;
  const int64_t bk = w >> kBucketLog2, l = w & (kBucket - 1);
  const uint32_t* __restrict__ partial = jb.partial;
  unsigned long long s = 0;
  for (int k = 0; k < K; ++k) s += partial[(bk * K + k) * kBucket + l];
  jb.counts[w] = s;
}

// Head/tail buffers (Section IV-C), bottom-up: a rule's first two words come
// from its first body symbols, taking a child's head when the symbol is a
// rule (children are on deeper levels, finished earlier).
__global__ void head_tail_level_kernel(const int32_t* __restrict__ order, int64_t a, int64_t b, DevGrammar d,
                                       int32_t* __restrict__ head, int32_t* __restrict__ tail) {
  for (int64_t k = a + blockIdx.x * int64_t(blockDim.x) + threadIdx.x; k < b; k += int64_t(gridDim.x) * blockDim.x) {
    const int32_t r = order[k];
    const int64_t lo = d.rule_off[r], hi = d.rule_off[r + 1];
    int32_t h[2] = {-1, -1};
    int n = 0;
    for (int64_t i = lo; i < hi && n < 2; ++i) {
      const int32_t s = d.sym[i];
      if (s < d.V) {
        h[n++] = s;
      } else {
        const int32_t c = s - d.V;
        const int32_t c0 = head[2 * c], c1 = head[2 * c + 1];
        h[n++] = c0;
        if (n < 2 && c1 >= 0) h[n++] = c1;
      }
    }
    int32_t t[2] = {-1, -1};  // t[1] = last word, t[0] = the one before
    int m = 0;
    for (int64_t i = hi - 1; i >= lo && m < 2; --i) {
      const int32_t s = d.sym[i];
      if (s < d.V) {
        t[1 - m++] = s;
      } else {
        const int32_t c = s - d.V;
        const int32_t c0 = tail[2 * c], c1 = tail[2 * c + 1];
        t[1 - m++] = c1;
        if (m < 2 && c0 >= 0) t[1 - m++] = c0;
      }
    }
    head[2 * r] = h[0];
    head[2 * r + 1] = h[1];
    tail[2 * r] = t[0];
    tail[2 * r + 1] = t[1];
  }
}

}  // namespace

namespace {

// Weights of n grammars (n <= kMaxWcJobs): one launch per DAG level covers
// every grammar that has that level.
template <int NJ>
void weights_batch(gt_grammar* const* gs, uint64_t* const* wts, int n, cudaStream_t s) {
  gt_ctx* ctx = gs[0]->ctx;
  Phase ph(ctx, "weights", s);
  const int threads = 256;
  const int cap = ctx->num_sms * 16;
  WtRoots<NJ> roots{};
  roots.n = n;
  int depth = 0;
  for (int j = 0; j < n; ++j) {
    GT_CUDA(cudaMemsetAsync(wts[j], 0, size_t(gs[j]->d.R) * 8, s));
    roots.wt[j] = reinterpret_cast<unsigned long long*>(wts[j]);
    depth = std::max(depth, int(gs[j]->d.depth));
  }
  wt_init_kernel<NJ><<<1, 64, 0, s>>>(roots);
  GT_LAUNCH_CHECK();
  for (int lv = 1; lv < depth; ++lv) {
    WtBatch<NJ> bt{};
    int ctas = 0;
    for (int j = 0; j < n; ++j) {
      const gt_grammar* g = gs[j];
      if (lv >= g->d.depth) continue;
      const int64_t a = g->ledge_off[lv], b = g->ledge_off[lv + 1];
      if (b <= a) continue;
      WtJob& jb = bt.job[bt.n];
      jb = {g->d.ledge_child, g->d.ledge_par, g->d.ledge_mult, a, b, roots.wt[j]};
      bt.cta[bt.n++] = ctas;
      ctas += grid_for(b - a, threads, cap);
    }
    if (bt.n == 0) continue;
    bt.cta[bt.n] = ctas;
    wt_edges_kernel<NJ><<<ctas, threads, 0, s>>>(bt);
    GT_LAUNCH_CHECK();
  }
}

// Scratch of one grammar's word count.
struct WcScratch {
  Buf plain, wgt, cnt, ovf, partial;
};

template <int NJ>
void word_count_batch(gt_grammar* const* gs, const uint64_t* const* wts, uint64_t* const* counts, int n,
                      cudaStream_t s, uint32_t* status) {
  gt_ctx* ctx = gs[0]->ctx;
  if (!status) status = ctx->d_status;
  WcBatch<NJ> bt{};
  std::unique_ptr<WcScratch[]> scr(new WcScratch[size_t(n)]);
  int part = 0, hist = 0, red = 0;
  bool aggregate = false;
  for (int j = 0; j < n; ++j) {
    gt_grammar* g = gs[j];
    const DevGrammar& d = g->d;
    if (d.N >= (uint64_t(1) << 32)) fail(GT_EOVERFLOW, "word count needs fewer than 2^32 tokens per grammar");
    if (d.V > kMaxBuckets * kBucket) fail(GT_EOVERFLOW, "word count supports num_words <= 2^21");
    if (d.ntiles * kTile >= (int64_t(1) << 31)) fail(GT_EOVERFLOW, "word count supports fewer than 2^31 symbols");
    if (d.ntiles == 0) {
      GT_CUDA(cudaMemsetAsync(counts[j], 0, size_t(d.V) * 8, s));
      continue;
    }
    const int nb = int((d.V + kBucket - 1) / kBucket);
    const int64_t nchunks = d.ntiles * kTile / kChunk;
    const int grid1 = int(std::min<int64_t>((nchunks + kPartWarps - 1) / kPartWarps, ctx->num_sms));
    const int64_t my_syms = (nchunks + grid1 - 1) / grid1 * kChunk;
    const int64_t nr_chunks = nchunks - d.first_rule_tile * (kTile / kChunk);
    const int64_t my_nr = nr_chunks > 0 ? ((nr_chunks + grid1 - 1) / grid1 + kPartWarps) * kChunk : 0;
    WcJob& jb = bt.job[bt.n];
    PartOut& po = jb.out;
    po.nb = nb;
    // a region holds 4x a CTA's even share of symbols per bucket, plus slack;
    // whatever does not fit goes to the overflow list
    po.cap_p = (4 * my_syms / nb + 4096 + 7) / 8 * 8;
    po.cap_w = my_nr > 0 ? (4 * my_nr / nb + 1024 + 1) / 2 * 2 : 2;
    po.ovf_cap = d.ntiles * kTile;
    // hist CTAs per bucket (partial histograms reduced afterwards)
    const int64_t k_param = gparam(g, "wc_slices", 0);
    const int K = k_param > 0 ? int(std::min<int64_t>(k_param, 64)) : std::max(1, (3 * ctx->num_sms + nb - 1) / nb);
    WcScratch& sc = scr[j];
    sc.plain = Buf(ctx, size_t(nb) * grid1 * po.cap_p * 2, s);
    sc.wgt = Buf(ctx, size_t(nb) * grid1 * po.cap_w * 8, s);
    sc.cnt = Buf(ctx, size_t(nb) * grid1 * 16 + 16, s);
    sc.ovf = Buf(ctx, size_t(po.ovf_cap) * 8, s);
    sc.partial = Buf(ctx, size_t(nb) * K * kBucket * 4, s);
    po.plain = sc.plain.as<uint16_t>();
    po.wgt = sc.wgt.as<uint64_t>();
    po.cnt_p = sc.cnt.as<int64_t>();
    po.cnt_w = po.cnt_p + int64_t(nb) * grid1;
    po.ovf_n = reinterpret_cast<unsigned long long*>(po.cnt_w + int64_t(nb) * grid1);
    po.ovf = sc.ovf.as<uint64_t>();
    GT_CUDA(cudaMemsetAsync(sc.cnt.p, 0, size_t(nb) * grid1 * 16 + 16, s));
    jb.sym = d.sym;
    jb.sym_rule = d.sym_rule;
    jb.wt = wts[j];
    jb.partial = sc.partial.as<uint32_t>();
    jb.counts = reinterpret_cast<unsigned long long*>(counts[j]);
    jb.nchunks = nchunks;
    jb.first_rule_chunk = d.first_rule_tile * (kTile / kChunk);
    jb.V = d.V;
    jb.grid1 = grid1;
    jb.K = K;
    bt.part_cta[bt.n] = part;
    bt.hist_cta[bt.n] = hist;
    bt.red_cta[bt.n] = red;
    part += grid1;
    hist += nb * K;
    red += int((int64_t(d.V) + kReduceThreads - 1) / kReduceThreads);
    aggregate = aggregate || gparam(g, "wc_aggregate", 0) != 0;
    ++bt.n;
  }
  if (bt.n == 0) return;
  bt.part_cta[bt.n] = part;
  bt.hist_cta[bt.n] = hist;
  bt.red_cta[bt.n] = red;
  {
    Phase ph(ctx, "wc_partition", s);
    const size_t smem = sizeof(PartShared);
    GT_CUDA(cudaFuncSetAttribute(wc_partition_kernel<NJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    wc_partition_kernel<NJ><<<part, kPartThreads, smem, s>>>(bt, status);
    GT_LAUNCH_CHECK();
  }
  {
    Phase ph2(ctx, "wc_hist", s);
    if (aggregate)
      wc_hist_kernel<true, NJ><<<hist, kHistThreads, 0, s>>>(bt);
    else
      wc_hist_kernel<false, NJ><<<hist, kHistThreads, 0, s>>>(bt);
    GT_LAUNCH_CHECK();
    wc_reduce_kernel<NJ><<<red, kReduceThreads, 0, s>>>(bt);
    GT_LAUNCH_CHECK();
  }
}

}  // namespace

void run_rule_weights(gt_grammar* g, uint64_t* d_wt, cudaStream_t s) { weights_batch<1>(&g, &d_wt, 1, s); }

void run_word_count(gt_grammar* g, const uint64_t* d_wt, uint64_t* d_counts, cudaStream_t s, uint32_t* status) {
  word_count_batch<1>(&g, &d_wt, &d_counts, 1, s, status);
}

void run_word_count_multi(gt_grammar* const* gs, uint64_t* const* counts, int n, cudaStream_t s,
                          uint32_t* status) {
  if (n <= 0) return;
  if (n > kMaxWcJobs) fail(GT_EINVAL, "at most 64 grammars per fused word count");
  std::vector<Buf> wt;
  std::vector<uint64_t*> wp;
  for (int j = 0; j < n; ++j) {
    wt.emplace_back(gs[j]->ctx, size_t(gs[j]->d.R) * 8, s);
    wp.push_back(wt.back().as<uint64_t>());
  }
  if (n == 1) {
    weights_batch<1>(gs, wp.data(), 1, s);
    word_count_batch<1>(gs, wp.data(), counts, 1, s, status);
  } else {
    weights_batch<kMaxWcJobs>(gs, wp.data(), n, s);
    word_count_batch<kMaxWcJobs>(gs, wp.data(), counts, n, s, status);
  }
}

void run_head_tail(gt_grammar* g, int32_t* d_head, int32_t* d_tail, cudaStream_t s) {
  const DevGrammar& d = g->d;
  const int threads = 256;
  const int cap = g->ctx->num_sms * 8;
  for (int lv = d.depth - 1; lv >= 0; --lv) {
    const int64_t a = g->lvl_off[lv], b = g->lvl_off[lv + 1];
    if (b > a) {
      head_tail_level_kernel<<<grid_for(b - a, threads, cap), threads, 0, s>>>(d.lvl_order, a, b, d, d_head, d_tail);
      GT_LAUNCH_CHECK();
    }
  }
}

}  // namespace gt
