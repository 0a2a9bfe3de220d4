// Grammar load: the initialisation phase of Section IV-A, run once per grammar.
//
// From the raw bodies it builds, on the device:
//   * the deduplicated child list of every rule with multiplicities - the
//     (subRuleId, subRuleFreq) pairs Algorithm 1 iterates;
//   * the parent list of every rule (genRuleParentsKernel of Algorithm 2);
//   * the root's child list per file, for per-file analytics (the root's own
//     child list is their sum over files, so the root's references are sorted
//     once, by (file, child));
//   * DAG levels by a frontier (Kahn) traversal: level(c) > level(p) for every
//     edge p -> c, so processing levels in increasing order is a valid
//     top-down schedule and in decreasing order a valid bottom-up one.  This
//     replaces the paper's readiness masks and stop-flag relaunch loop
//     (Algorithms 1 and 2) with a schedule computed once;
//   * W_r (words in the body), S_r (references in the body) and L_r (words in
//     the expansion), and the owned-window total of Eq. 1.
#include <algorithm>

#include "gt_internal.cuh"

namespace gt {
namespace {

__device__ __forceinline__ int64_t upper_bound_i64(const int64_t* a, int64_t n, int64_t x) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (a[mid] <= x) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ int64_t lower_bound_u32key(const uint64_t* keys, int64_t n, uint32_t hi_part) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (uint32_t(keys[mid] >> 32) < hi_part) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

__global__ void validate_kernel(const int32_t* __restrict__ sym, int64_t G, int32_t V, int32_t R,
                                uint32_t* status, unsigned long long* nref, unsigned long long* nref_root,
                                int64_t root_len) {
  unsigned long long c = 0, cr = 0;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < G; i += int64_t(gridDim.x) * blockDim.x) {
    int32_t s = sym[i];
    if (s < 0 || s >= V + R || s == V) atomicOr(status, ST_INVALID);
    if (s >= V) {
      ++c;
      if (i < root_len) ++cr;
    }
  }
  for (int o = 16; o; o >>= 1) {
    c += __shfl_xor_sync(0xffffffffu, c, o);
    cr += __shfl_xor_sync(0xffffffffu, cr, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (c) atomicAdd(nref, c);
    if (cr) atomicAdd(nref_root, cr);
  }
}

// For every rule reference in a rule body: key (parent << 32 | child), the
// parent read from sym_rule; for every reference in the root: (file << 32 |
// child).  A block takes tiles of kEkTile symbols (kEkItems per thread,
// coalesced) and claims the tile's output slots with one atomic per key array,
// so the shared counters see G / kEkTile atomics in all.
constexpr int kEkThreads = 256;
constexpr int kEkItems = 16;
constexpr int64_t kEkTile = int64_t(kEkThreads) * kEkItems;

__global__ void __launch_bounds__(kEkThreads) edge_keys_kernel(
    const int32_t* __restrict__ sym, int64_t G, int32_t V, const int32_t* __restrict__ sym_rule, int64_t sr_base,
    const int64_t* __restrict__ file_off, int32_t F, int64_t root_len, uint64_t* __restrict__ gkeys,
    unsigned long long* gcount, uint64_t* __restrict__ rkeys, unsigned long long* rcount) {
  constexpr int kWarps = kEkThreads / 32;
  __shared__ unsigned s_cnt[2][kWarps];
  __shared__ unsigned long long s_base[2];
  __shared__ int32_t s_file[2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  for (int64_t t0 = blockIdx.x * kEkTile; t0 < G; t0 += int64_t(gridDim.x) * kEkTile) {
    int32_t sv[kEkItems];
    unsigned ref_bits = 0, root_bits = 0, wc = 0, wr = 0;
#pragma unroll
    for (int k = 0; k < kEkItems; ++k) {
      const int64_t i = t0 + k * kEkThreads + threadIdx.x;
      sv[k] = i < G ? sym[i] : 0;
      const bool rr = i < G && sv[k] >= V && i < root_len;
      const bool ref = i < G && sv[k] >= V && i >= root_len;
      ref_bits |= unsigned(ref) << k;
      root_bits |= unsigned(rr) << k;
      wc += __popc(__ballot_sync(0xffffffffu, ref));
      wr += __popc(__ballot_sync(0xffffffffu, rr));
    }
    if (lane == 0) {
      s_cnt[0][warp] = wc;
      s_cnt[1][warp] = wr;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
      unsigned tot = 0;
      for (int w = 0; w < kWarps; ++w) tot += s_cnt[threadIdx.x][w];
      s_base[threadIdx.x] = tot ? atomicAdd(threadIdx.x ? rcount : gcount, (unsigned long long)tot) : 0ull;
      // the files holding the tile's first and last root symbols
      if (t0 < root_len) {
        const int64_t last = t0 + kEkTile - 1 < root_len ? t0 + kEkTile - 1 : root_len - 1;
        s_file[threadIdx.x] = int32_t(upper_bound_i64(file_off, int64_t(F) + 1, threadIdx.x ? last : t0) - 1);
      }
    }
    __syncthreads();
    unsigned long long gb = s_base[0], rb = s_base[1];
    const int32_t f_lo = s_file[0], f_hi = s_file[1];
    for (int w = 0; w < warp; ++w) {
      gb += s_cnt[0][w];
      rb += s_cnt[1][w];
    }
#pragma unroll
    for (int k = 0; k < kEkItems; ++k) {
      const int64_t i = t0 + k * kEkThreads + threadIdx.x;
      const bool ref = (ref_bits >> k) & 1u, rr = (root_bits >> k) & 1u;
      const unsigned m = __ballot_sync(0xffffffffu, ref), mr = __ballot_sync(0xffffffffu, rr);
      const uint32_t child = uint32_t(sv[k] - V);
      if (ref) gkeys[gb + __popc(m & lt)] = (uint64_t(uint32_t(sym_rule[i - sr_base])) << 32) | child;
      if (rr) {
        const int64_t f =
            f_lo == f_hi ? f_lo : f_lo + upper_bound_i64(file_off + f_lo, int64_t(f_hi - f_lo) + 2, i) - 1;
        rkeys[rb + __popc(mr & lt)] = (uint64_t(f) << 32) | child;
      }
      gb += __popc(m);
      rb += __popc(mr);
    }
    __syncthreads();  // s_cnt and s_base are rewritten by the next tile
  }
}

__global__ void run_flags_kernel(const uint64_t* __restrict__ k, int64_t n, int64_t* __restrict__ flag) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    flag[i] = (i == 0 || k[i] != k[i - 1]) ? 1 : 0;
}

__global__ void run_compact_kernel(const uint64_t* __restrict__ k, int64_t n, const int64_t* __restrict__ flag,
                                   const int64_t* __restrict__ pos, uint64_t* __restrict__ uk,
                                   int64_t* __restrict__ ustart) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    if (flag[i]) {
      uk[pos[i]] = k[i];
      ustart[pos[i]] = i;
    }
}

// Split unique (hi << 32 | lo) keys into lo and the run length (multiplicity).
__global__ void run_split_kernel(const uint64_t* __restrict__ uk, const int64_t* __restrict__ ustart, int64_t nu,
                                 int64_t n, int32_t* __restrict__ lo_out, uint32_t* __restrict__ mult) {
  for (int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; j < nu; j += int64_t(gridDim.x) * blockDim.x) {
    lo_out[j] = int32_t(uint32_t(uk[j]));
    const int64_t next = j + 1 < nu ? ustart[j + 1] : n;
    mult[j] = uint32_t(next - ustart[j]);
  }
}

// off[h] = first index whose high 32 bits are >= h, for h in [0, nh].
__global__ void csr_offsets_kernel(const uint64_t* __restrict__ keys, int64_t n, int64_t nh, int64_t* __restrict__ off) {
  for (int64_t h = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; h <= nh; h += int64_t(gridDim.x) * blockDim.x)
    off[h] = h == nh ? n : lower_bound_u32key(keys, n, uint32_t(h));
}

// Root multiplicity of every child: the sum over files of its per-file
// multiplicity.  The (child << 32 | file) keys are sorted by child, so a warp
// adds up each run it holds (segmented shuffle scan) and issues one atomic per
// run piece.
__global__ void root_mult_kernel(const uint64_t* __restrict__ tks, const uint32_t* __restrict__ fm, int64_t n,
                                 unsigned* __restrict__ rm) {
  const int lane = threadIdx.x & 31;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i - lane < n; i += stride) {
    const bool in = i < n;
    const uint32_t c = in ? uint32_t(tks[i] >> 32) : 0xffffffffu;
    unsigned v = in ? fm[i] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned tv = __shfl_up_sync(0xffffffffu, v, o);
      const uint32_t tc = __shfl_up_sync(0xffffffffu, c, o);
      if (lane >= o && tc == c) v += tv;
    }
    const uint32_t nc = __shfl_down_sync(0xffffffffu, c, 1);
    if (in && (lane == 31 || nc != c)) atomicAdd(&rm[c], v);
  }
}

__global__ void nonzero_flags_kernel(const unsigned* __restrict__ rm, int32_t R, int64_t* __restrict__ flag) {
  for (int64_t c = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; c < R; c += int64_t(gridDim.x) * blockDim.x)
    flag[c] = rm[c] != 0u ? 1 : 0;
}

__global__ void root_compact_kernel(const unsigned* __restrict__ rm, int32_t R, const int64_t* __restrict__ flag,
                                    const int64_t* __restrict__ pos, int32_t* __restrict__ lo,
                                    uint32_t* __restrict__ mult) {
  for (int64_t c = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; c < R; c += int64_t(gridDim.x) * blockDim.x)
    if (flag[c]) {
      lo[pos[c]] = int32_t(c);
      mult[pos[c]] = rm[c];
    }
}

// Keys (0 << 32 | child) of the root's distinct children.
__global__ void prefix_keys_kernel(const int32_t* __restrict__ lo, int64_t n, uint64_t* __restrict__ uk) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    uk[i] = uint64_t(uint32_t(lo[i]));
}

__global__ void transpose_keys_kernel(const uint64_t* __restrict__ uk, int64_t n, uint64_t* __restrict__ tk) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const uint64_t k = uk[i];
    tk[i] = (k << 32) | (k >> 32);
  }
}

__global__ void indegree_kernel(const int64_t* __restrict__ pedge_off, int32_t R, int32_t* __restrict__ rem,
                                int32_t* __restrict__ level, int32_t* __restrict__ order,
                                unsigned long long* __restrict__ tail) {
  for (int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < R; r += int64_t(gridDim.x) * blockDim.x) {
    const int32_t d = int32_t(pedge_off[r + 1] - pedge_off[r]);
    rem[r] = d;
    level[r] = -1;
    if (d == 0) {
      level[r] = 0;
      order[atomicAdd(tail, 1ull)] = int32_t(r);
    }
  }
}

// Number of children of each frontier rule (to spread the frontier's edges
// evenly over threads).
__global__ void frontier_count_kernel(const int32_t* __restrict__ order, int64_t a, int64_t n,
                                      const int64_t* __restrict__ cedge_off, int64_t* __restrict__ cnt) {
  for (int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
    const int32_t r = order[a + k];
    cnt[k] = cedge_off[r + 1] - cedge_off[r];
  }
}

// One thread per edge leaving the frontier.  A child whose last parent is done
// joins the next level.
__global__ void frontier_edges_kernel(const int32_t* __restrict__ order, int64_t a, int64_t n,
                                      const int64_t* __restrict__ foff, int64_t total,
                                      const int64_t* __restrict__ cedge_off, const int32_t* __restrict__ cedge_child,
                                      int32_t* __restrict__ rem, int32_t* __restrict__ level, int32_t next_level,
                                      int32_t* __restrict__ out_order, unsigned long long* __restrict__ tail) {
  const int lane = threadIdx.x & 31;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  // warp-uniform trips (stride is a multiple of 32): one append per warp
  for (int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; j - lane < total; j += stride) {
    bool done = false;
    int32_t c = 0;
    if (j < total) {
      const int64_t k = upper_bound_i64(foff, n, j) - 1;
      const int32_t r = order[a + k];
      c = cedge_child[cedge_off[r] + (j - foff[k])];
      done = atomicSub(&rem[c], 1) == 1;
    }
    const unsigned m = __ballot_sync(0xffffffffu, done);
    if (!m) continue;
    unsigned long long base = 0;
    if (lane == __ffs(m) - 1) base = atomicAdd(tail, (unsigned long long)__popc(m));
    base = __shfl_sync(0xffffffffu, base, __ffs(m) - 1);
    if (done) {
      level[c] = next_level;
      out_order[base + __popc(m & ((1u << lane) - 1u))] = c;
    }
  }
}

// One warp per frontier rule (levels after the first, whose frontiers hold
// many rules with few children each): no per-level count and scan.
__global__ void frontier_warp_kernel(const int32_t* __restrict__ order, int64_t a, int64_t n,
                                     const int64_t* __restrict__ cedge_off, const int32_t* __restrict__ cedge_child,
                                     int32_t* __restrict__ rem, int32_t* __restrict__ level, int32_t next_level,
                                     int32_t* __restrict__ out_order, unsigned long long* __restrict__ tail) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t k = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5; k < n; k += nwarps) {
    const int32_t r = order[a + k];
    const int64_t e1 = cedge_off[r + 1];
    for (int64_t e0 = cedge_off[r]; e0 < e1; e0 += 32) {
      const int64_t e = e0 + lane;
      bool done = false;
      int32_t c = 0;
      if (e < e1) {
        c = cedge_child[e];
        done = atomicSub(&rem[c], 1) == 1;
      }
      const unsigned m = __ballot_sync(0xffffffffu, done);
      if (!m) continue;
      unsigned long long base = 0;
      if (lane == __ffs(m) - 1) base = atomicAdd(tail, (unsigned long long)__popc(m));
      base = __shfl_sync(0xffffffffu, base, __ffs(m) - 1);
      if (done) {
        level[c] = next_level;
        out_order[base + __popc(m & ((1u << lane) - 1u))] = c;
      }
    }
  }
}

// keys[e] = level(child of parent edge e) << 32 | e, to group parent edges by
// the level of their child.
__global__ void ledge_keys_kernel(const int32_t* __restrict__ pchild, const int32_t* __restrict__ level, int64_t E,
                                  uint64_t* __restrict__ keys) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < E; e += int64_t(gridDim.x) * blockDim.x)
    keys[e] = (uint64_t(uint32_t(level[pchild[e]])) << 32) | uint64_t(e);
}

__global__ void ledge_gather_kernel(const uint64_t* __restrict__ keys, int64_t E, const int32_t* __restrict__ pchild,
                                    const int32_t* __restrict__ ppar, const uint32_t* __restrict__ pmult,
                                    int32_t* __restrict__ lchild, int32_t* __restrict__ lpar,
                                    uint32_t* __restrict__ lmult) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < E; i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t e = int64_t(uint32_t(keys[i]));
    lchild[i] = pchild[e];
    lpar[i] = ppar[e];
    lmult[i] = pmult[e];
  }
}

__global__ void high32_kernel(const uint64_t* __restrict__ keys, int64_t n, int32_t* __restrict__ out) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    out[i] = int32_t(uint32_t(keys[i] >> 32));
}

__global__ void level_keys_kernel(const int32_t* __restrict__ level, int32_t R, uint64_t* __restrict__ keys) {
  for (int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < R; r += int64_t(gridDim.x) * blockDim.x)
    keys[r] = (uint64_t(uint32_t(level[r])) << 32) | uint64_t(r);
}

__global__ void low32_kernel(const uint64_t* __restrict__ keys, int64_t n, int32_t* __restrict__ out) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    out[i] = int32_t(uint32_t(keys[i]));
}

// W_r and S_r for non-root rules (bodies are short: one thread each).
__global__ void body_counts_kernel(const int32_t* __restrict__ sym, const int64_t* __restrict__ rule_off, int32_t R,
                                   int32_t V, int32_t* __restrict__ W, int32_t* __restrict__ S) {
  for (int64_t r = 1 + blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < R; r += int64_t(gridDim.x) * blockDim.x) {
    int32_t w = 0, s = 0;
    for (int64_t i = rule_off[r]; i < rule_off[r + 1]; ++i) (sym[i] < V ? w : s) += 1;
    W[r] = w;
    S[r] = s;
  }
}

__device__ __forceinline__ uint64_t owned_part(uint64_t L) { return L >= 2 ? L - 2 : 0; }

// Expansion lengths for one level of non-root rules (children are on deeper,
// already finished levels).  A group of 4 lanes per rule (most rules have a
// few children).  Also adds each rule's owned 3-word windows (the exact count
// behind Eq. 1's bound) to *owned, one atomic per block.
constexpr int kExpGroup = 4;

__global__ void exp_len_kernel(const int32_t* __restrict__ order, int64_t a, int64_t b,
                               const int64_t* __restrict__ cedge_off, const int32_t* __restrict__ cedge_child,
                               const uint32_t* __restrict__ cedge_mult, const int32_t* __restrict__ W,
                               uint64_t* __restrict__ L, unsigned long long* __restrict__ owned) {
  __shared__ unsigned long long block_owned;
  if (threadIdx.x == 0) block_owned = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int grp = lane / kExpGroup, sub = lane % kExpGroup;
  constexpr int kGroups = 32 / kExpGroup;
  const int64_t warps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  const int64_t w0 = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
  unsigned long long own = 0;
  // a warp takes kGroups consecutive rules per trip: warp-uniform trips
  for (int64_t kb = a + w0 * kGroups; kb < b; kb += warps * kGroups) {
    const int64_t k = kb + grp;
    const bool in = k < b;
    const int32_t r = in ? order[k] : 0;
    uint64_t sum = 0, inner = 0;
    if (in && r != 0)
      for (int64_t e = cedge_off[r] + sub; e < cedge_off[r + 1]; e += kExpGroup) {
        const uint64_t lc = L[cedge_child[e]];
        sum += cedge_mult[e] * lc;
        inner += cedge_mult[e] * owned_part(lc);
      }
#pragma unroll
    for (int o = kExpGroup / 2; o; o >>= 1) {
      sum += __shfl_xor_sync(0xffffffffu, sum, o, kExpGroup);
      inner += __shfl_xor_sync(0xffffffffu, inner, o, kExpGroup);
    }
    if (in && r != 0 && sub == 0) {
      const uint64_t lr = uint64_t(W[r]) + sum;
      L[r] = lr;
      own += owned_part(lr) - inner;
    }
  }
  if (own) atomicAdd(&block_owned, own);
  __syncthreads();
  if (threadIdx.x == 0 && block_owned) atomicAdd(owned, block_owned);
}

// Root, per file: references S_f, sum of mult * L_c and of mult * (L_c - 2)+
// over the file's distinct children.  Block (f, y) reduces one slice of file
// f's edges, so a large file is spread over many blocks.
__global__ void root_file_sums_kernel(const int64_t* __restrict__ redge_off, const int32_t* __restrict__ redge_child,
                                      const uint32_t* __restrict__ redge_mult, int32_t F,
                                      const uint64_t* __restrict__ L, unsigned long long* __restrict__ sums) {
  __shared__ unsigned long long acc[3];
  for (int32_t f = blockIdx.x; f < F; f += gridDim.x) {
    if (threadIdx.x < 3) acc[threadIdx.x] = 0;
    __syncthreads();
    const int64_t lo = redge_off[f], n = redge_off[f + 1] - lo;
    const int64_t a = lo + n * blockIdx.y / gridDim.y, b = lo + n * (blockIdx.y + 1) / gridDim.y;
    unsigned long long s = 0, sl = 0, so = 0;
    for (int64_t e = a + threadIdx.x; e < b; e += blockDim.x) {
      const uint64_t m = redge_mult[e], lc = L[redge_child[e]];
      s += m;
      sl += m * lc;
      so += m * owned_part(lc);
    }
    for (int o = 16; o; o >>= 1) {
      s += __shfl_xor_sync(0xffffffffu, s, o);
      sl += __shfl_xor_sync(0xffffffffu, sl, o);
      so += __shfl_xor_sync(0xffffffffu, so, o);
    }
    if ((threadIdx.x & 31) == 0 && (s | sl | so)) {
      atomicAdd(&acc[0], s);
      atomicAdd(&acc[1], sl);
      atomicAdd(&acc[2], so);
    }
    __syncthreads();
    if (threadIdx.x < 3 && acc[threadIdx.x]) atomicAdd(&sums[3 * f + threadIdx.x], acc[threadIdx.x]);
    __syncthreads();
  }
}

// Root, per file: words W_f = symbols - S_f, length N_f = W_f + sum mult*L_c,
// and the root's owned windows (per file, since windows stop at file ends).
__global__ void root_file_final_kernel(const int64_t* __restrict__ file_off, int32_t F,
                                       const unsigned long long* __restrict__ sums, uint64_t* __restrict__ file_len,
                                       unsigned long long* __restrict__ tot) {
  for (int32_t f = blockIdx.x * blockDim.x + threadIdx.x; f < F; f += gridDim.x * blockDim.x) {
    const uint64_t S = sums[3 * f], sl = sums[3 * f + 1], so = sums[3 * f + 2];
    const uint64_t W = uint64_t(file_off[f + 1] - file_off[f]) - S;
    const uint64_t lf = W + sl;
    file_len[f] = lf;
    atomicAdd(&tot[0], (unsigned long long)W);
    atomicAdd(&tot[1], (unsigned long long)S);
    atomicAdd(&tot[2], (unsigned long long)lf);
    atomicAdd(&tot[3], (unsigned long long)(owned_part(lf) - so));
  }
}

__global__ void max_u64_kernel(const uint64_t* __restrict__ x, int64_t n, unsigned long long* __restrict__ out) {
  unsigned long long m = 0;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    m = max(m, (unsigned long long)x[i]);
  for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

// Rule of every symbol from the tile holding the end of the root onwards.
// Rule of every symbol from tile t_first on (root symbols read 0).  Block per
// tile of kTile symbols: the tile's rules lie between tile_rule[t] and
// tile_rule[t + 1] (at most kTile + 1 of them: non-root bodies are non-empty),
// so their offsets fit in shared memory and each symbol searches there.
__global__ void __launch_bounds__(256) sym_rule_kernel(const int64_t* __restrict__ rule_off,
                                                       const int32_t* __restrict__ tile_rule, int64_t G,
                                                       int64_t root_len, int64_t t_first, int64_t ntiles,
                                                       int32_t* __restrict__ out) {
  __shared__ int64_t so[kTile + 3];
  for (int64_t t = t_first + blockIdx.x; t < ntiles; t += gridDim.x) {
    const int32_t r0 = tile_rule[t], r1 = tile_rule[t + 1];
    const int nr = r1 - r0 + 2;  // rule_off[r0 .. r1 + 1]
    __syncthreads();
    for (int k = threadIdx.x; k < nr; k += blockDim.x) so[k] = rule_off[r0 + k];
    __syncthreads();
    for (int j = threadIdx.x; j < kTile; j += blockDim.x) {
      const int64_t pos = t * kTile + j;
      int32_t r = 0;
      if (pos >= root_len && pos < G) {
        int lo = 0, hi = nr - 1;  // so[lo] <= pos < so[hi]
        while (hi - lo > 1) {
          const int mid = (lo + hi) >> 1;
          if (so[mid] <= pos) lo = mid;
          else hi = mid;
        }
        r = r0 + lo;
      }
      out[(t - t_first) * kTile + j] = r;
    }
  }
}

// Sizes for the bottom-up per-file path: over every distinct (file, child)
// root pair, the child's expansion length and its number of 3-word windows.
__global__ void bu_sizes_kernel(const int32_t* __restrict__ redge_child, int64_t ER, const uint64_t* __restrict__ L,
                                unsigned long long* __restrict__ out) {
  unsigned long long a = 0, b = 0;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < ER; e += int64_t(gridDim.x) * blockDim.x) {
    const uint64_t l = L[redge_child[e]];
    a += l;
    b += l >= 2 ? l - 2 : 0;
  }
  for (int o = 16; o; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&out[0], a);
    atomicAdd(&out[1], b);
  }
}

__global__ void tile_rule_kernel(const int64_t* __restrict__ rule_off, int32_t R, int64_t G, int64_t ntiles,
                                 int32_t* __restrict__ tile_rule) {
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t <= ntiles; t += int64_t(gridDim.x) * blockDim.x) {
    const int64_t pos = t < ntiles ? t * kTile : (G > 0 ? G - 1 : 0);
    tile_rule[t] = int32_t(upper_bound_i64(rule_off, int64_t(R) + 1, pos) - 1);
  }
}

template <class T>
T* dalloc(gt_grammar* g, size_t n, cudaStream_t s) {
  return static_cast<T*>(grammar_alloc(g, n * sizeof(T) + 16, s));
}

int bits_for(int64_t x) {
  int b = 0;
  while (b < 63 && (int64_t(1) << b) <= x) ++b;
  return b;
}

// Sort keys (hi << 32 | lo) with lo < 2^lo_bits and hi < 2^hi_bits on the bits
// that can be nonzero only.  The result lands in out (in is clobbered).
void sort_hi_lo(uint64_t* in, uint64_t* out, void* vin, void* vout, int vb, int64_t n, int lo_bits, int hi_bits,
                void* scratch, cudaStream_t s) {
  radix_sort_u64_split(in, out, vin, vout, vb, n, 0, std::min(lo_bits, 32), 32, 32 + hi_bits, scratch, s);
}

// Sort keys, deduplicate runs, split into (lo, multiplicity) and build CSR
// offsets over the high half.  Returns the number of distinct keys.
// With prefix > 0 the outputs start with `prefix` given entries of high half 0
// (lo pre_lo, multiplicity pre_mult, lo ascending) and keys must all have a
// nonzero high half.
int64_t dedup_csr(gt_grammar* g, uint64_t* keys, int64_t n, int hi_bits, int lo_bits, int64_t nh, int64_t** off_out,
                  int32_t** lo_out, uint32_t** mult_out, uint64_t** ukeys_keep, cudaStream_t s, int64_t prefix = 0,
                  const int32_t* pre_lo = nullptr, const uint32_t* pre_mult = nullptr) {
  gt_ctx* ctx = g->ctx;
  const int threads = 256;
  const int cap = ctx->num_sms * 16;
  Buf sorted(ctx, size_t(n) * 8, s);
  Buf rscratch(ctx, radix_scratch_bytes(n, false, 0), s);
  sort_hi_lo(keys, sorted.as<uint64_t>(), nullptr, nullptr, 0, n, lo_bits, hi_bits, rscratch.p, s);
  Buf flag(ctx, size_t(n) * 8, s), pos(ctx, size_t(n) * 8, s);
  Buf sscratch(ctx, scan_scratch_bytes(n), s);
  int64_t nu = 0;
  if (n > 0) {
    run_flags_kernel<<<grid_for(n, threads, cap), threads, 0, s>>>(sorted.as<uint64_t>(), n, flag.as<int64_t>());
    GT_LAUNCH_CHECK();
    exclusive_scan_i64(flag.as<int64_t>(), pos.as<int64_t>(), n, sscratch.p, s);
    int64_t last_pos = 0, last_flag = 0;
    GT_CUDA(cudaMemcpyAsync(&last_pos, pos.as<int64_t>() + n - 1, 8, cudaMemcpyDeviceToHost, s));
    GT_CUDA(cudaMemcpyAsync(&last_flag, flag.as<int64_t>() + n - 1, 8, cudaMemcpyDeviceToHost, s));
    GT_CUDA(cudaStreamSynchronize(s));
    nu = last_pos + last_flag;
  }
  uint64_t* uk = dalloc<uint64_t>(g, size_t(prefix + nu), s);
  Buf ustart(ctx, size_t(nu) * 8, s);
  int32_t* lo = dalloc<int32_t>(g, size_t(prefix + nu), s);
  uint32_t* mult = dalloc<uint32_t>(g, size_t(prefix + nu), s);
  int64_t* off = dalloc<int64_t>(g, size_t(nh) + 1, s);
  if (prefix > 0) {
    prefix_keys_kernel<<<grid_for(prefix, threads, cap), threads, 0, s>>>(pre_lo, prefix, uk);
    GT_LAUNCH_CHECK();
    GT_CUDA(cudaMemcpyAsync(lo, pre_lo, size_t(prefix) * 4, cudaMemcpyDeviceToDevice, s));
    GT_CUDA(cudaMemcpyAsync(mult, pre_mult, size_t(prefix) * 4, cudaMemcpyDeviceToDevice, s));
  }
  if (n > 0) {
    run_compact_kernel<<<grid_for(n, threads, cap), threads, 0, s>>>(
        sorted.as<uint64_t>(), n, flag.as<int64_t>(), pos.as<int64_t>(), uk + prefix, ustart.as<int64_t>());
    GT_LAUNCH_CHECK();
    run_split_kernel<<<grid_for(nu, threads, cap), threads, 0, s>>>(uk + prefix, ustart.as<int64_t>(), nu, n,
                                                                    lo + prefix, mult + prefix);
    GT_LAUNCH_CHECK();
  }
  csr_offsets_kernel<<<grid_for(nh + 1, threads, cap), threads, 0, s>>>(uk, prefix + nu, nh, off);
  GT_LAUNCH_CHECK();
  *off_out = off;
  *lo_out = lo;
  *mult_out = mult;
  if (ukeys_keep) *ukeys_keep = uk;
  return prefix + nu;
}

}  // namespace

void csr_offsets_hi(const uint64_t* keys, int64_t n, int64_t nh, int64_t* off, cudaStream_t s) {
  csr_offsets_kernel<<<grid_for(nh + 1, 256, 4096), 256, 0, s>>>(keys, n, nh, off);
  GT_LAUNCH_CHECK();
}

void load_build_dag(gt_grammar* g, cudaStream_t s) {
  gt_ctx* ctx = g->ctx;
  DevGrammar& d = g->d;
  const int threads = 256;
  const int cap = ctx->num_sms * 16;
  const int32_t V = d.V, R = d.R, F = d.F;
  const int64_t G = d.G;

  // ---- validate symbols and count references ----
  Buf counters(ctx, 16 * 8, s);
  unsigned long long* ctr = counters.as<unsigned long long>();
  GT_CUDA(cudaMemsetAsync(ctr, 0, 16 * 8, s));
  GT_CUDA(cudaMemsetAsync(ctx->d_status, 0, 4, s));
  if (G > 0) {
    validate_kernel<<<grid_for(G, threads, cap), threads, 0, s>>>(d.sym, G, V, R, ctx->d_status, ctr + 0, ctr + 1,
                                                                  d.root_len);
    GT_LAUNCH_CHECK();
  }
  unsigned long long h[2] = {0, 0};
  uint32_t st = 0;
  GT_CUDA(cudaMemcpyAsync(h, ctr, 16, cudaMemcpyDeviceToHost, s));
  GT_CUDA(cudaMemcpyAsync(&st, ctx->d_status, 4, cudaMemcpyDeviceToHost, s));
  GT_CUDA(cudaStreamSynchronize(s));
  if (st & ST_INVALID) fail(GT_EINVAL, "grammar symbol out of range or referencing the root");
  const int64_t nref = int64_t(h[0]), nref_root = int64_t(h[1]);

  // ---- tiles and the rule of every body symbol ----
  {
    d.ntiles = (G + kTile - 1) / kTile;
    int32_t* tr = dalloc<int32_t>(g, size_t(d.ntiles) + 1, s);
    tile_rule_kernel<<<grid_for(d.ntiles + 1, threads, cap), threads, 0, s>>>(d.rule_off, R, G, d.ntiles, tr);
    GT_LAUNCH_CHECK();
    d.tile_rule = tr;
    d.first_rule_tile = d.root_len / kTile;
    const int64_t nt = d.ntiles - d.first_rule_tile;
    int32_t* sr = dalloc<int32_t>(g, size_t(nt > 0 ? nt * kTile : 1), s);
    if (nt > 0) {
      sym_rule_kernel<<<unsigned(std::min<int64_t>(nt, int64_t(ctx->num_sms) * 8)), 256, 0, s>>>(
          d.rule_off, tr, G, d.root_len, d.first_rule_tile, d.ntiles, sr);
      GT_LAUNCH_CHECK();
    }
    d.sym_rule = sr;
  }

  // ---- edge keys ----
  Buf gkeys(ctx, size_t(nref - nref_root) * 8, s), rkeys(ctx, size_t(nref_root) * 8, s);
  GT_CUDA(cudaMemsetAsync(ctr, 0, 16, s));
  if (G > 0) {
    edge_keys_kernel<<<grid_for((G + kEkItems - 1) / kEkItems, kEkThreads, cap), kEkThreads, 0, s>>>(
        d.sym, G, V, d.sym_rule, d.first_rule_tile * kTile, d.file_off, F, d.root_len, gkeys.as<uint64_t>(), ctr + 0,
        rkeys.as<uint64_t>(), ctr + 1);
    GT_LAUNCH_CHECK();
  }
  const int rbits = bits_for(R);
  uint64_t* ukeys = nullptr;
  int32_t* pedge_child = nullptr;
  int64_t* cedge_off;
  int32_t* cedge_child;
  uint32_t* cedge_mult;
  int64_t* redge_off;
  int32_t* redge_child;
  uint32_t* redge_mult;
  uint64_t* rukeys = nullptr;
  d.ER = dedup_csr(g, rkeys.as<uint64_t>(), nref_root, bits_for(F), rbits, F, &redge_off, &redge_child,
                   &redge_mult, &rukeys, s);
  d.redge_off = redge_off;
  d.redge_child = redge_child;
  d.redge_mult = redge_mult;
  // the same root edges child-major (for each child, the files referencing
  // it), and from them the root's distinct children with their multiplicities
  Buf root_lo(ctx, size_t(R) * 4, s), root_mult(ctx, size_t(R) * 4, s);
  int64_t e_root = 0;
  {
    const int64_t ER = d.ER;
    Buf tk(ctx, size_t(ER) * 8, s), tks(ctx, size_t(ER) * 8, s), mv(ctx, size_t(ER) * 4, s);
    Buf rs(ctx, radix_scratch_bytes(ER, true, 4), s);
    uint32_t* fm = dalloc<uint32_t>(g, size_t(ER), s);
    int32_t* ff = dalloc<int32_t>(g, size_t(ER), s);
    int64_t* fo = dalloc<int64_t>(g, size_t(R) + 1, s);
    if (ER > 0) {
      transpose_keys_kernel<<<grid_for(ER, threads, cap), threads, 0, s>>>(rukeys, ER, tk.as<uint64_t>());
      GT_LAUNCH_CHECK();
      GT_CUDA(cudaMemcpyAsync(mv.p, redge_mult, size_t(ER) * 4, cudaMemcpyDeviceToDevice, s));
      // rukeys ascend by (file, child): a stable sort on the child alone keeps
      // the files of each child ascending
      radix_sort_u64(tk.as<uint64_t>(), tks.as<uint64_t>(), mv.p, fm, 4, ER, 32, 32 + rbits, rs.p, s);
      low32_kernel<<<grid_for(ER, threads, cap), threads, 0, s>>>(tks.as<uint64_t>(), ER, ff);
      GT_LAUNCH_CHECK();
      Buf rm(ctx, size_t(R) * 4, s), flag(ctx, size_t(R) * 8, s), pos(ctx, size_t(R) * 8, s);
      Buf sscratch(ctx, scan_scratch_bytes(R), s);
      GT_CUDA(cudaMemsetAsync(rm.p, 0, size_t(R) * 4, s));
      root_mult_kernel<<<grid_for(ER, threads, cap), threads, 0, s>>>(tks.as<uint64_t>(), fm, ER, rm.as<unsigned>());
      GT_LAUNCH_CHECK();
      nonzero_flags_kernel<<<grid_for(R, threads, cap), threads, 0, s>>>(rm.as<unsigned>(), R, flag.as<int64_t>());
      GT_LAUNCH_CHECK();
      exclusive_scan_i64(flag.as<int64_t>(), pos.as<int64_t>(), R, sscratch.p, s);
      root_compact_kernel<<<grid_for(R, threads, cap), threads, 0, s>>>(
          rm.as<unsigned>(), R, flag.as<int64_t>(), pos.as<int64_t>(), root_lo.as<int32_t>(), root_mult.as<uint32_t>());
      GT_LAUNCH_CHECK();
      int64_t last[2];
      GT_CUDA(cudaMemcpyAsync(&last[0], pos.as<int64_t>() + R - 1, 8, cudaMemcpyDeviceToHost, s));
      GT_CUDA(cudaMemcpyAsync(&last[1], flag.as<int64_t>() + R - 1, 8, cudaMemcpyDeviceToHost, s));
      GT_CUDA(cudaStreamSynchronize(s));
      e_root = last[0] + last[1];
    }
    csr_offsets_kernel<<<grid_for(int64_t(R) + 1, threads, cap), threads, 0, s>>>(tks.as<uint64_t>(), ER, R, fo);
    GT_LAUNCH_CHECK();
    d.rfile_off = fo;
    d.rfile_f = ff;
    d.rfile_m = fm;
  }
  // all distinct edges (parent << 32 | child): the root's first, then the
  // deduplicated references of the rule bodies
  d.E = dedup_csr(g, gkeys.as<uint64_t>(), nref - nref_root, rbits, rbits, R, &cedge_off, &cedge_child, &cedge_mult,
                  &ukeys, s, e_root, root_lo.as<int32_t>(), root_mult.as<uint32_t>());
  d.cedge_off = cedge_off;
  d.cedge_child = cedge_child;
  d.cedge_mult = cedge_mult;

  // ---- parent lists: transpose the distinct edges, keep multiplicities ----
  {
    const int64_t E = d.E;
    Buf tk(ctx, size_t(E) * 8, s), tks(ctx, size_t(E) * 8, s), mv(ctx, size_t(E) * 4, s);
    Buf rs(ctx, radix_scratch_bytes(E, true, 4), s);
    uint32_t* pm = dalloc<uint32_t>(g, size_t(E), s);
    int32_t* pp = dalloc<int32_t>(g, size_t(E), s);
    int32_t* pc = dalloc<int32_t>(g, size_t(E), s);
    int64_t* po = dalloc<int64_t>(g, size_t(R) + 1, s);
    if (E > 0) {
      transpose_keys_kernel<<<grid_for(E, threads, cap), threads, 0, s>>>(ukeys, E, tk.as<uint64_t>());
      GT_LAUNCH_CHECK();
      GT_CUDA(cudaMemcpyAsync(mv.p, cedge_mult, size_t(E) * 4, cudaMemcpyDeviceToDevice, s));
      // ukeys ascend by (parent, child): sort stably on the child alone
      radix_sort_u64(tk.as<uint64_t>(), tks.as<uint64_t>(), mv.p, pm, 4, E, 32, 32 + rbits, rs.p, s);
      low32_kernel<<<grid_for(E, threads, cap), threads, 0, s>>>(tks.as<uint64_t>(), E, pp);
      GT_LAUNCH_CHECK();
      high32_kernel<<<grid_for(E, threads, cap), threads, 0, s>>>(tks.as<uint64_t>(), E, pc);
      GT_LAUNCH_CHECK();
    }
    csr_offsets_kernel<<<grid_for(int64_t(R) + 1, threads, cap), threads, 0, s>>>(tks.as<uint64_t>(), E, R, po);
    GT_LAUNCH_CHECK();
    d.pedge_off = po;
    d.pedge_par = pp;
    d.pedge_mult = pm;
    pedge_child = pc;
  }

  // ---- levels (Kahn frontiers) ----
  {
    int32_t* level = dalloc<int32_t>(g, size_t(R), s);
    int32_t* order = dalloc<int32_t>(g, size_t(R), s);
    Buf rem(ctx, size_t(R) * 4, s), korder(ctx, size_t(R) * 4, s);
    unsigned long long* tail = ctr + 2;
    GT_CUDA(cudaMemsetAsync(tail, 0, 8, s));
    indegree_kernel<<<grid_for(R, threads, cap), threads, 0, s>>>(d.pedge_off, R, rem.as<int32_t>(), level,
                                                                  korder.as<int32_t>(), tail);
    GT_LAUNCH_CHECK();
    int64_t a = 0, b = 0;
    unsigned long long t = 0;
    GT_CUDA(cudaMemcpyAsync(&t, tail, 8, cudaMemcpyDeviceToHost, s));
    GT_CUDA(cudaStreamSynchronize(s));
    b = int64_t(t);
    int32_t lv = 0;
    Buf fcnt(ctx, size_t(R) * 8, s), foff(ctx, size_t(R) * 8, s), fsc(ctx, scan_scratch_bytes(R), s);
    while (b > a) {
      const int64_t n = b - a;
      if (lv == 0) {
        // the root's level: few rules with very many children, spread edge-wise
        frontier_count_kernel<<<grid_for(n, threads, cap), threads, 0, s>>>(korder.as<int32_t>(), a, n, d.cedge_off,
                                                                            fcnt.as<int64_t>());
        GT_LAUNCH_CHECK();
        exclusive_scan_i64(fcnt.as<int64_t>(), foff.as<int64_t>(), n, fsc.p, s);
        int64_t lastc[2];
        GT_CUDA(cudaMemcpyAsync(&lastc[0], foff.as<int64_t>() + n - 1, 8, cudaMemcpyDeviceToHost, s));
        GT_CUDA(cudaMemcpyAsync(&lastc[1], fcnt.as<int64_t>() + n - 1, 8, cudaMemcpyDeviceToHost, s));
        GT_CUDA(cudaStreamSynchronize(s));
        const int64_t total = lastc[0] + lastc[1];
        if (total > 0) {
          frontier_edges_kernel<<<grid_for(total, threads, cap), threads, 0, s>>>(
              korder.as<int32_t>(), a, n, foff.as<int64_t>(), total, d.cedge_off, d.cedge_child, rem.as<int32_t>(),
              level, lv + 1, korder.as<int32_t>(), tail);
          GT_LAUNCH_CHECK();
        }
      } else {
        frontier_warp_kernel<<<grid_for(n * 32, threads, cap), threads, 0, s>>>(
            korder.as<int32_t>(), a, n, d.cedge_off, d.cedge_child, rem.as<int32_t>(), level, lv + 1,
            korder.as<int32_t>(), tail);
        GT_LAUNCH_CHECK();
      }
      GT_CUDA(cudaMemcpyAsync(&t, tail, 8, cudaMemcpyDeviceToHost, s));
      GT_CUDA(cudaStreamSynchronize(s));
      a = b;
      b = int64_t(t);
      ++lv;
    }
    if (b != R) fail(GT_EINVAL, "the rule graph has a cycle");
    d.depth = lv;
    // deterministic order inside each level: sort by (level, rule)
    Buf lk(ctx, size_t(R) * 8, s), lks(ctx, size_t(R) * 8, s);
    Buf rs(ctx, radix_scratch_bytes(R, false, 0), s);
    level_keys_kernel<<<grid_for(R, threads, cap), threads, 0, s>>>(level, R, lk.as<uint64_t>());
    GT_LAUNCH_CHECK();
    // keys are made in rule order: a stable sort on the level alone suffices
    radix_sort_u64(lk.as<uint64_t>(), lks.as<uint64_t>(), nullptr, nullptr, 0, R, 32, 32 + bits_for(lv), rs.p, s);
    low32_kernel<<<grid_for(R, threads, cap), threads, 0, s>>>(lks.as<uint64_t>(), R, order);
    GT_LAUNCH_CHECK();
    Buf loff(ctx, size_t(lv + 1) * 8, s);
    csr_offsets_kernel<<<grid_for(lv + 1, threads, cap), threads, 0, s>>>(lks.as<uint64_t>(), R, lv,
                                                                           loff.as<int64_t>());
    GT_LAUNCH_CHECK();
    g->lvl_off.assign(size_t(lv) + 1, 0);
    GT_CUDA(cudaMemcpyAsync(g->lvl_off.data(), loff.p, size_t(lv + 1) * 8, cudaMemcpyDeviceToHost, s));
    d.level = level;
    d.lvl_order = order;
    // parent edges grouped by the level of their child (for the weight pass)
    const int64_t E = d.E;
    int32_t* lc = dalloc<int32_t>(g, size_t(E), s);
    int32_t* lp = dalloc<int32_t>(g, size_t(E), s);
    uint32_t* lm = dalloc<uint32_t>(g, size_t(E), s);
    Buf ek(ctx, size_t(E) * 8, s), eks(ctx, size_t(E) * 8, s), ers(ctx, radix_scratch_bytes(E, false, 0), s);
    Buf eoff(ctx, size_t(lv + 1) * 8, s);
    if (E > 0) {
      ledge_keys_kernel<<<grid_for(E, threads, cap), threads, 0, s>>>(pedge_child, level, E, ek.as<uint64_t>());
      GT_LAUNCH_CHECK();
      radix_sort_u64(ek.as<uint64_t>(), eks.as<uint64_t>(), nullptr, nullptr, 0, E, 32, 32 + bits_for(lv), ers.p,
                     s);
      ledge_gather_kernel<<<grid_for(E, threads, cap), threads, 0, s>>>(eks.as<uint64_t>(), E, pedge_child,
                                                                        d.pedge_par, d.pedge_mult, lc, lp, lm);
      GT_LAUNCH_CHECK();
    }
    csr_offsets_kernel<<<grid_for(lv + 1, threads, cap), threads, 0, s>>>(eks.as<uint64_t>(), E, lv,
                                                                           eoff.as<int64_t>());
    GT_LAUNCH_CHECK();
    g->ledge_off.assign(size_t(lv) + 1, 0);
    GT_CUDA(cudaMemcpyAsync(g->ledge_off.data(), eoff.p, size_t(lv + 1) * 8, cudaMemcpyDeviceToHost, s));
    d.ledge_child = lc;
    d.ledge_par = lp;
    d.ledge_mult = lm;
  }

  // ---- per-rule counts and expansion lengths ----
  {
    int32_t* W = dalloc<int32_t>(g, size_t(R), s);
    int32_t* S = dalloc<int32_t>(g, size_t(R), s);
    uint64_t* L = dalloc<uint64_t>(g, size_t(R), s);
    uint64_t* flen = dalloc<uint64_t>(g, size_t(F), s);
    Buf fsums(ctx, size_t(F) * 3 * 8, s);
    unsigned long long* owned = ctr + 6;
    unsigned long long* tot = ctr + 8;  // W_root, S_root, N, root owned windows
    GT_CUDA(cudaMemsetAsync(ctr + 6, 0, 6 * 8, s));
    GT_CUDA(cudaMemsetAsync(fsums.p, 0, size_t(F) * 3 * 8, s));
    GT_CUDA(cudaMemsetAsync(W, 0, 4, s));
    GT_CUDA(cudaMemsetAsync(S, 0, 4, s));
    GT_CUDA(cudaMemsetAsync(L, 0, 8, s));
    if (R > 1) {
      body_counts_kernel<<<grid_for(R, threads, cap), threads, 0, s>>>(d.sym, d.rule_off, R, V, W, S);
      GT_LAUNCH_CHECK();
    }
    for (int32_t lv = d.depth - 1; lv >= 0; --lv) {
      const int64_t a = g->lvl_off[lv], b = g->lvl_off[lv + 1];
      if (b > a) {
        exp_len_kernel<<<grid_for((b - a) * kExpGroup + 32, threads, cap), threads, 0, s>>>(
            d.lvl_order, a, b, d.cedge_off, d.cedge_child, d.cedge_mult, W, L, owned);
        GT_LAUNCH_CHECK();
      }
    }
    root_file_sums_kernel<<<dim3(std::min(F, cap), 32), threads, 0, s>>>(d.redge_off, d.redge_child, d.redge_mult, F,
                                                                         L, fsums.as<unsigned long long>());
    GT_LAUNCH_CHECK();
    root_file_final_kernel<<<grid_for(F, threads, cap), threads, 0, s>>>(d.file_off, F,
                                                                         fsums.as<unsigned long long>(), flen, tot);
    GT_LAUNCH_CHECK();
    unsigned long long hv[6];
    GT_CUDA(cudaMemcpyAsync(hv, ctr + 6, 48, cudaMemcpyDeviceToHost, s));
    GT_CUDA(cudaStreamSynchronize(s));
    // root entries: W and S of the whole root, L = N
    const int32_t wr = int32_t(std::min<unsigned long long>(hv[2], 0x7fffffffull));
    const int32_t sr = int32_t(std::min<unsigned long long>(hv[3], 0x7fffffffull));
    const uint64_t n = hv[4];
    GT_CUDA(cudaMemcpyAsync(W, &wr, 4, cudaMemcpyHostToDevice, s));
    GT_CUDA(cudaMemcpyAsync(S, &sr, 4, cudaMemcpyHostToDevice, s));
    GT_CUDA(cudaMemcpyAsync(L, &n, 8, cudaMemcpyHostToDevice, s));
    d.nwords = W;
    d.nrefs = S;
    d.exp_len = L;
    d.file_len = flen;
    d.N = n;
    g->info.num_tokens = int64_t(n);
    g->info.root_words = int64_t(hv[2]);
    g->info.owned_windows = int64_t(hv[0] + hv[5]);
    GT_CUDA(cudaStreamSynchronize(s));
  }

  // ---- sizes of the bottom-up per-file rows, longest file ----
  {
    GT_CUDA(cudaMemsetAsync(ctr + 12, 0, 24, s));
    if (d.ER > 0) {
      bu_sizes_kernel<<<grid_for(d.ER, threads, cap), threads, 0, s>>>(d.redge_child, d.ER, d.exp_len, ctr + 12);
      GT_LAUNCH_CHECK();
    }
    if (F > 0) {
      max_u64_kernel<<<grid_for(F, threads, cap), threads, 0, s>>>(d.file_len, F, ctr + 14);
      GT_LAUNCH_CHECK();
    }
    unsigned long long hb[3];
    GT_CUDA(cudaMemcpyAsync(hb, ctr + 12, 24, cudaMemcpyDeviceToHost, s));
    GT_CUDA(cudaStreamSynchronize(s));
    g->bu_words = int64_t(hb[0]);
    g->bu_windows = int64_t(hb[1]);
    g->max_file_len = int64_t(hb[2]);
  }

  GT_CUDA(cudaStreamSynchronize(s));
  g->info.num_edges = d.E;
  g->info.num_root_edges = d.ER;
  g->info.depth = d.depth;
}

}  // namespace gt
