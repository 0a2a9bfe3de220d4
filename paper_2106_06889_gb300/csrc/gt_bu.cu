// Bottom-up per-file analytics (Section IV-A's bottom-up traversal, the
// strategy the paper selects when there are many files, Section V-C).
//
// The paper's bottom-up pass merges every rule's local table into its parents
// and finally merges the tables of the root's children ("level-2 nodes") into
// per-file results.  Here the per-file result is built the same way - root
// words of the file plus, for every distinct (file, root child) pair, the
// child's expansion weighted by how often the file references it - but a
// child's "table" is produced on the fly by walking its derivation depth
// first (an explicit stack bounded by the DAG depth), so no per-rule table has
// to be materialised.  The (file, key, weight) rows are then radix-sorted and
// summed, which yields the canonical order directly.  There is no limit on
// the number of files.
#include <algorithm>

#include "gt_device.cuh"

namespace gt {

int file_strategy(const gt_grammar* g) {
  const int64_t p = gparam(g, "file_strategy", 0);
  if (p == 1 || p == 2) return int(p);
  return g->d.F <= 64 ? 1 : 2;
}

namespace {

constexpr int kMaxStack = 64;

int bits_for(int64_t x) {
  int b = 1;
  while ((int64_t(1) << b) <= x) ++b;
  return b;
}

// Visit the words of expand(c) in order.
template <class Emit>
__device__ __forceinline__ void walk_rule(const DevGrammar& d, int32_t c, Emit&& emit) {
  int64_t spos[kMaxStack], send[kMaxStack];
  int sp = 0;
  int64_t pos = d.rule_off[c], end = d.rule_off[c + 1];
  while (true) {
    if (pos == end) {
      if (sp == 0) return;
      --sp;
      pos = spos[sp];
      end = send[sp];
      continue;
    }
    const int32_t s = d.sym[pos++];
    if (s < d.V) {
      emit(s);
    } else {
      spos[sp] = pos;
      send[sp] = end;
      ++sp;
      const int32_t ch = s - d.V;
      pos = d.rule_off[ch];
      end = d.rule_off[ch + 1];
    }
  }
}

__device__ __forceinline__ int32_t file_of_redge(const DevGrammar& d, int64_t e) {
  return int32_t(upper_bound_dev(d.redge_off, int64_t(d.F) + 1, e) - 1);
}

__global__ void redge_len_kernel(const DevGrammar d, bool windows, int64_t* __restrict__ cnt) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < d.ER; e += int64_t(gridDim.x) * blockDim.x) {
    const uint64_t l = d.exp_len[d.redge_child[e]];
    cnt[e] = windows ? (l >= 2 ? int64_t(l - 2) : 0) : int64_t(l);
  }
}

// ---- word rows: key = file << kbw | word ----

__global__ void root_word_rows_kernel(const DevGrammar d, int kbw, uint64_t pad, uint64_t* __restrict__ key,
                                      uint32_t* __restrict__ val) {
  for (int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; j < d.root_len; j += int64_t(gridDim.x) * blockDim.x) {
    const int32_t s = d.sym[j];
    if (s < d.V) {
      const int64_t f = upper_bound_dev(d.file_off, int64_t(d.F) + 1, j) - 1;
      key[j] = (uint64_t(f) << kbw) | uint64_t(uint32_t(s));
      val[j] = 1u;
    } else {
      key[j] = pad;
      val[j] = 0u;
    }
  }
}

__global__ void child_word_rows_kernel(const DevGrammar d, int kbw, const int64_t* __restrict__ pos,
                                       uint64_t* __restrict__ key, uint32_t* __restrict__ val) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < d.ER; e += int64_t(gridDim.x) * blockDim.x) {
    const uint64_t f = uint64_t(file_of_redge(d, e)) << kbw;
    const uint32_t m = d.redge_mult[e];
    int64_t o = pos[e];
    walk_rule(d, d.redge_child[e], [&](int32_t w) {
      key[o] = f | uint64_t(uint32_t(w));
      val[o] = m;
      ++o;
    });
  }
}

// ---- window rows: key = compact 3-word key, file separately ----

__global__ void root_window_rows_kernel(const DevGrammar d, const int32_t* __restrict__ head,
                                        const int32_t* __restrict__ tail, int kb, uint64_t pad,
                                        uint64_t* __restrict__ key, uint64_t* __restrict__ file,
                                        uint32_t* __restrict__ val) {
  for (int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; j < d.root_len; j += int64_t(gridDim.x) * blockDim.x) {
    int32_t r, f;
    const int64_t end = seq_end(d, j, &r, &f);
    uint64_t k[2];
    const int n = windows_at(d, head, tail, j, end, kb, k);
    for (int i = 0; i < 2; ++i) {
      key[2 * j + i] = i < n ? k[i] : pad;
      file[2 * j + i] = uint64_t(uint32_t(f));
      val[2 * j + i] = i < n ? 1u : 0u;
    }
  }
}

__global__ void child_window_rows_kernel(const DevGrammar d, int kb, const int64_t* __restrict__ pos,
                                         uint64_t* __restrict__ key, uint64_t* __restrict__ file,
                                         uint32_t* __restrict__ val) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < d.ER; e += int64_t(gridDim.x) * blockDim.x) {
    const uint64_t f = uint64_t(file_of_redge(d, e));
    const uint32_t m = d.redge_mult[e];
    int64_t o = pos[e];
    int32_t a = -1, b = -1;
    walk_rule(d, d.redge_child[e], [&](int32_t w) {
      if (a >= 0) {
        key[o] = pack_compact(a, b, w, kb);
        file[o] = f;
        val[o] = m;
        ++o;
      }
      a = b;
      b = w;
    });
  }
}

__global__ void reduce_flags_kernel(const uint64_t* __restrict__ key, const uint32_t* __restrict__ val, int64_t n,
                                    uint64_t pad, int64_t* __restrict__ flag, int64_t* __restrict__ v64) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const bool real = key[i] != pad;
    flag[i] = real && (i == 0 || key[i] != key[i - 1]);
    v64[i] = real ? int64_t(val[i]) : 0;
  }
}

// One row per distinct (file, word): word, file, summed count.
__global__ void reduce_write_kernel(const uint64_t* __restrict__ key, int64_t n, const int64_t* __restrict__ flag,
                                    const int64_t* __restrict__ pos, int kbw, int32_t* __restrict__ word,
                                    int32_t* __restrict__ file, int64_t* __restrict__ start) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    if (flag[i]) {
      const int64_t u = pos[i];
      word[u] = int32_t(key[i] & ((uint64_t(1) << kbw) - 1));
      file[u] = int32_t(key[i] >> kbw);
      start[u] = i;
    }
}

__global__ void reduce_sum_kernel(const int64_t* __restrict__ start, const int64_t* __restrict__ nr_dev,
                                  const int64_t* __restrict__ wsum, const int64_t* __restrict__ v64, int64_t n,
                                  uint64_t* __restrict__ cnt) {
  const int64_t nr = *nr_dev;
  for (int64_t u = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; u < nr; u += int64_t(gridDim.x) * blockDim.x) {
    const int64_t a = start[u], b = u + 1 < nr ? start[u + 1] : n;
    const int64_t end_sum = b < n ? wsum[b] : wsum[n - 1] + v64[n - 1];
    cnt[u] = uint64_t(end_sum - wsum[a]);
  }
}

__global__ void total_kernel(const int64_t* __restrict__ ex, const int64_t* __restrict__ flag, int64_t n,
                             int64_t* __restrict__ out) {
  *out = n > 0 ? ex[n - 1] + flag[n - 1] : 0;
}

// off[f] = first row whose file is >= f (rows sorted by file), f in [0, F].
__global__ void file_offsets_kernel(const int32_t* __restrict__ file, const int64_t* __restrict__ n_dev, int32_t F,
                                    int64_t* __restrict__ off) {
  const int64_t n = *n_dev;
  for (int32_t f = blockIdx.x * blockDim.x + threadIdx.x; f <= F; f += gridDim.x * blockDim.x) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (file[mid] < f) lo = mid + 1;
      else hi = mid;
    }
    off[f] = lo;
  }
}

// Inverted index from (file, word) rows: stable sort by word carrying the
// file, so the files come out ascending inside each word; offsets per word.
__global__ void word_keys_kernel(const int32_t* __restrict__ word, const int32_t* __restrict__ file,
                                 const int64_t* __restrict__ n_dev, int64_t bound, int32_t V, uint64_t* __restrict__ k,
                                 uint32_t* __restrict__ f) {
  const int64_t n = *n_dev;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < bound; i += int64_t(gridDim.x) * blockDim.x) {
    k[i] = i < n ? uint64_t(uint32_t(word[i])) : uint64_t(uint32_t(V));
    f[i] = i < n ? uint32_t(file[i]) : 0u;
  }
}

__global__ void widen_i32_kernel(const int32_t* __restrict__ a, const int64_t* __restrict__ n_dev,
                                 uint64_t* __restrict__ out) {
  const int64_t n = *n_dev;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    out[i] = uint64_t(uint32_t(a[i]));
}

__global__ void word_offsets_kernel(const uint64_t* __restrict__ sk, const int64_t* __restrict__ n_dev, int32_t V,
                                    int64_t* __restrict__ off) {
  const int64_t n = *n_dev;
  for (int64_t w = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; w <= V; w += int64_t(gridDim.x) * blockDim.x) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (int64_t(sk[mid]) < w) lo = mid + 1;
      else hi = mid;
    }
    off[w] = lo;
  }
}

// ---- small files: expanded and sorted in shared memory, one CTA per file ----
//
// When every file has at most kLocalMax tokens, a CTA expands one file into
// shared memory (root symbols of the file, each rule reference walked), sorts
// its words with an LSD radix sort in shared memory (8-bit digits, ranks by
// ballot multisplit, stable), and run-length encodes them into the file's
// (word, count) rows, written to a slot of the file's length.  A second pass
// packs the slots.  No global sort is involved.

constexpr int kLocalThreads = 256;
constexpr int kLocalWarps = kLocalThreads / 32;
constexpr int64_t kLocalMax = 8192;

// Exclusive prefix over the CTA (kLocalThreads threads); *total gets the sum.
__device__ __forceinline__ int local_scan(int v, int* total, int* warp_tot) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  int before = 0, all = 0;
#pragma unroll
  for (int w = 0; w < kLocalWarps; ++w) {
    const int t = warp_tot[w];
    before += w < warp ? t : 0;
    all += t;
  }
  __syncthreads();
  *total = all;
  return before + incl - v;
}

__device__ __forceinline__ unsigned local_peers(uint32_t dg, unsigned active) {
  unsigned peers = active;
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    const bool bit = (dg >> b) & 1u;
    const unsigned bal = __ballot_sync(0xffffffffu, bit);
    peers &= bit ? bal : ~bal;
  }
  return peers;
}

// Stable LSD radix sort of keys[0, n) over bits [0, key_bits) in shared
// memory, 8-bit digits, ping-ponging between a and b; returns the buffer that
// holds the result.  Warp w ranks its contiguous slice 32 keys at a time.
template <typename K>
__device__ K* local_sort(K* a, K* b, int n, int key_bits, uint32_t (*wcnt)[256], uint32_t* dstart, uint32_t* dtot) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned lt = (1u << lane) - 1u;
  K* src = a;
  K* dst = b;
  const int per = (n + kLocalWarps * 32 - 1) / (kLocalWarps * 32) * 32;  // warp slice, a multiple of 32
  const int lo = min(n, warp * per), hi = min(n, lo + per);
  for (int shift = 0; shift < key_bits; shift += 8) {
    const uint32_t mask = key_bits - shift >= 8 ? 0xffu : ((1u << (key_bits - shift)) - 1u);
    for (int q = lane; q < 256; q += 32) wcnt[warp][q] = 0;
    __syncwarp();
    for (int i = lo + lane; i < hi; i += 32) atomicAdd(&wcnt[warp][uint32_t(src[i] >> shift) & mask], 1u);
    __syncthreads();
    {  // thread = digit: exclusive over warps, then over digits
      const int dg = tid;
      uint32_t run = 0;
#pragma unroll
      for (int w = 0; w < kLocalWarps; ++w) {
        const uint32_t c = wcnt[w][dg];
        wcnt[w][dg] = run;
        run += c;
      }
      uint32_t incl = run;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
      }
      if (lane == 31) dtot[warp] = incl;
      __syncthreads();
      uint32_t pre = 0;
#pragma unroll
      for (int w = 0; w < kLocalWarps; ++w) pre += w < warp ? dtot[w] : 0u;
      dstart[dg] = pre + incl - run;
    }
    __syncthreads();
    for (int i0 = lo; i0 < hi; i0 += 32) {
      const int i = i0 + lane;
      const bool valid = i < hi;
      const K key = valid ? src[i] : K(0);
      const uint32_t dg = uint32_t(key >> shift) & mask;
      const unsigned peers = local_peers(dg, __ballot_sync(0xffffffffu, valid));
      const uint32_t before = wcnt[warp][dg];
      const uint32_t r = __popc(peers & lt);
      if (valid) dst[dstart[dg] + before + r] = key;
      __syncwarp();
      if (valid && r == 0) wcnt[warp][dg] = before + __popc(peers);
      __syncwarp();
    }
    __syncthreads();
    K* t = src;
    src = dst;
    dst = t;
  }
  return src;
}

// Expand file f into words[0, n) (its root symbols, each reference walked);
// returns n.
__device__ __forceinline__ int local_expand(const DevGrammar& d, int32_t f, uint32_t* words, int* warp_tot) {
  const int tid = threadIdx.x;
  const int64_t r0 = d.file_off[f], r1 = d.file_off[f + 1];
  int base = 0;
  for (int64_t j0 = r0; j0 < r1; j0 += kLocalThreads) {
    const int64_t j = j0 + tid;
    const int32_t sy = j < r1 ? d.sym[j] : 0;
    const int len = j < r1 ? (sy < d.V ? 1 : int(d.exp_len[sy - d.V])) : 0;
    int chunk;
    int o = base + local_scan(len, &chunk, warp_tot);
    if (j < r1) {
      if (sy < d.V) {
        words[o] = uint32_t(sy);
      } else {
        walk_rule(d, sy - d.V, [&](int32_t w) { words[o++] = uint32_t(w); });
      }
    }
    base += chunk;
  }
  __syncthreads();
  return base;
}

// Run-length encoding of sorted keys[0, n): head positions go to heads[];
// returns the number of distinct keys.
template <typename K>
__device__ __forceinline__ int local_heads(const K* keys, int n, uint32_t* heads, int* warp_tot) {
  const int tid = threadIdx.x;
  int rows = 0;
  for (int i0 = 0; i0 < n; i0 += kLocalThreads) {
    const int i = i0 + tid;
    const int head = (i < n && (i == 0 || keys[i] != keys[i - 1])) ? 1 : 0;
    int chunk;
    const int at = rows + local_scan(head, &chunk, warp_tot);
    if (head) heads[at] = uint32_t(i);
    rows += chunk;
  }
  __syncthreads();
  return rows;
}

__global__ void __launch_bounds__(kLocalThreads) local_word_rows_kernel(const DevGrammar d, int cap, int kbw,
                                                                        const int64_t* __restrict__ slot_off,
                                                                        int32_t* __restrict__ slot_word,
                                                                        uint32_t* __restrict__ slot_cnt,
                                                                        int64_t* __restrict__ nrows) {
  extern __shared__ __align__(16) uint32_t lsm[];
  uint32_t* bufa = lsm;
  uint32_t* bufb = lsm + cap;
  __shared__ uint32_t wcnt[kLocalWarps][256];
  __shared__ uint32_t dstart[256];
  __shared__ uint32_t dtot[kLocalWarps];
  __shared__ int warp_tot[kLocalWarps];
  const int tid = threadIdx.x;
  for (int32_t f = blockIdx.x; f < d.F; f += gridDim.x) {
    const int n = local_expand(d, f, bufa, warp_tot);
    uint32_t* src = local_sort(bufa, bufb, n, kbw, wcnt, dstart, dtot);
    uint32_t* dst = src == bufa ? bufb : bufa;
    const int rows = local_heads(src, n, dst, warp_tot);
    const int64_t so = slot_off[f];
    for (int k = tid; k < rows; k += kLocalThreads) {
      const uint32_t a = dst[k], b = k + 1 < rows ? dst[k + 1] : uint32_t(n);
      slot_word[so + k] = int32_t(src[a]);
      slot_cnt[so + k] = b - a;
    }
    if (tid == 0) nrows[f] = rows;
    __syncthreads();
  }
}

// Per-file 3-word windows of small files: the file expanded in shared memory,
// its window keys built and sorted there, one (key, count) row per distinct
// window.  The words alias the second key buffer until the keys are built.
__global__ void __launch_bounds__(kLocalThreads) local_window_rows_kernel(const DevGrammar d, int cap, int kb,
                                                                          int key_bits,
                                                                          const int64_t* __restrict__ slot_off,
                                                                          uint64_t* __restrict__ slot_key,
                                                                          uint32_t* __restrict__ slot_cnt,
                                                                          int64_t* __restrict__ nrows) {
  extern __shared__ __align__(16) uint32_t lsm[];
  uint64_t* ka = reinterpret_cast<uint64_t*>(lsm);
  uint64_t* kz = ka + cap;
  uint32_t* words = reinterpret_cast<uint32_t*>(kz);
  __shared__ uint32_t wcnt[kLocalWarps][256];
  __shared__ uint32_t dstart[256];
  __shared__ uint32_t dtot[kLocalWarps];
  __shared__ int warp_tot[kLocalWarps];
  const int tid = threadIdx.x;
  for (int32_t f = blockIdx.x; f < d.F; f += gridDim.x) {
    const int n = local_expand(d, f, words, warp_tot);
    const int nk = n >= 3 ? n - 2 : 0;
    for (int i = tid; i < nk; i += kLocalThreads)
      ka[i] = pack_compact(int32_t(words[i]), int32_t(words[i + 1]), int32_t(words[i + 2]), kb);
    __syncthreads();
    uint64_t* src = local_sort(ka, kz, nk, key_bits, wcnt, dstart, dtot);
    uint32_t* heads = reinterpret_cast<uint32_t*>(src == ka ? kz : ka);
    const int rows = local_heads(src, nk, heads, warp_tot);
    const int64_t so = slot_off[f];
    for (int k = tid; k < rows; k += kLocalThreads) {
      const uint32_t a = heads[k], b = k + 1 < rows ? heads[k + 1] : uint32_t(nk);
      slot_key[so + k] = src[a];
      slot_cnt[so + k] = b - a;
    }
    if (tid == 0) nrows[f] = rows;
    __syncthreads();
  }
}

// Pack window slots into (key, file, count) rows.
__global__ void local_pack_windows_kernel(int32_t F, const int64_t* __restrict__ slot_off,
                                          const int64_t* __restrict__ row_off, const uint64_t* __restrict__ slot_key,
                                          const uint32_t* __restrict__ slot_cnt, uint64_t* __restrict__ key,
                                          int32_t* __restrict__ file, uint64_t* __restrict__ cnt) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t f = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5; f < F; f += nwarps) {
    const int64_t so = slot_off[f], ro = row_off[f], n = row_off[f + 1] - ro;
    for (int64_t k = lane; k < n; k += 32) {
      key[ro + k] = slot_key[so + k];
      file[ro + k] = int32_t(f);
      cnt[ro + k] = slot_cnt[so + k];
    }
  }
}

// Token offsets of the files (slots) from their lengths.
__global__ void file_len_i64_kernel(const uint64_t* __restrict__ len, int32_t F, int64_t* __restrict__ out) {
  for (int32_t f = blockIdx.x * blockDim.x + threadIdx.x; f <= F; f += gridDim.x * blockDim.x)
    out[f] = f < F ? int64_t(len[f]) : 0;
}

// Pack the slots: warp per file.
__global__ void local_pack_kernel(int32_t F, const int64_t* __restrict__ slot_off, const int64_t* __restrict__ row_off,
                                  const int32_t* __restrict__ slot_word, const uint32_t* __restrict__ slot_cnt,
                                  int32_t* __restrict__ word, int32_t* __restrict__ file, uint64_t* __restrict__ cnt) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t f = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5; f < F; f += nwarps) {
    const int64_t so = slot_off[f], ro = row_off[f], n = row_off[f + 1] - ro;
    for (int64_t k = lane; k < n; k += 32) {
      word[ro + k] = slot_word[so + k];
      file[ro + k] = int32_t(f);
      cnt[ro + k] = slot_cnt[so + k];
    }
  }
}

// (file, word, count) rows of every file, sorted by (file, word).
struct WordRows {
  Buf word, file, cnt, total;
  int64_t bound = 0;
};

void bu_local_word_rows(gt_grammar* g, int kbw, cudaStream_t s, WordRows& out) {
  gt_ctx* ctx = g->ctx;
  const DevGrammar& d = g->d;
  const int64_t N = int64_t(d.N);
  const int cap = int(std::max<int64_t>(256, (g->max_file_len + 255) / 256 * 256));
  Phase ph(ctx, "bu_local", s);
  Buf soff(ctx, size_t(d.F + 1) * 8, s), flen(ctx, size_t(d.F + 1) * 8, s), sc(ctx, scan_scratch_bytes(d.F + 1), s);
  Buf sw(ctx, size_t(N) * 4, s), scn(ctx, size_t(N) * 4, s), nr(ctx, size_t(d.F + 1) * 8, s);
  Buf roff(ctx, size_t(d.F + 1) * 8, s);
  out.bound = N;
  out.word = Buf(ctx, size_t(N) * 4, s);
  out.file = Buf(ctx, size_t(N) * 4, s);
  out.cnt = Buf(ctx, size_t(N) * 8, s);
  out.total = Buf(ctx, 8, s);
  file_len_i64_kernel<<<grid_for(int64_t(d.F) + 1, 256, ctx->num_sms * 8), 256, 0, s>>>(d.file_len, d.F,
                                                                                     flen.as<int64_t>());
  GT_LAUNCH_CHECK();
  exclusive_scan_i64(flen.as<int64_t>(), soff.as<int64_t>(), d.F + 1, sc.p, s);
  const size_t smem = size_t(cap) * 8;
  GT_CUDA(cudaFuncSetAttribute(local_word_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
  GT_CUDA(cudaMemsetAsync(nr.as<int64_t>() + d.F, 0, 8, s));
  local_word_rows_kernel<<<unsigned(std::min<int64_t>(d.F, 65535)), kLocalThreads, smem, s>>>(
      d, cap, kbw, soff.as<int64_t>(), sw.as<int32_t>(), scn.as<uint32_t>(), nr.as<int64_t>());
  GT_LAUNCH_CHECK();
  exclusive_scan_i64(nr.as<int64_t>(), roff.as<int64_t>(), d.F + 1, sc.p, s);
  GT_CUDA(cudaMemcpyAsync(out.total.p, roff.as<int64_t>() + d.F, 8, cudaMemcpyDeviceToDevice, s));
  local_pack_kernel<<<grid_for(int64_t(d.F) * 32, 256, ctx->num_sms * 16), 256, 0, s>>>(
      d.F, soff.as<int64_t>(), roff.as<int64_t>(), sw.as<int32_t>(), scn.as<uint32_t>(), out.word.as<int32_t>(),
      out.file.as<int32_t>(), out.cnt.as<uint64_t>());
  GT_LAUNCH_CHECK();
}

void bu_word_rows(gt_grammar* g, cudaStream_t s, WordRows& out) {
  gt_ctx* ctx = g->ctx;
  const DevGrammar& d = g->d;
  const int threads = 256, cap = ctx->num_sms * 16;
  if (d.depth > kMaxStack) fail(GT_EOVERFLOW, "bottom-up expansion supports DAG depth <= 64");
  if (d.N >= (uint64_t(1) << 32)) fail(GT_EOVERFLOW, "per-file analytics need fewer than 2^32 tokens per grammar");
  const int kbw = bits_for(d.V);
  const int fb = bits_for(d.F);
  if (g->max_file_len <= kLocalMax && gparam(g, "bu_local", 1)) {
    bu_local_word_rows(g, kbw, s, out);
    return;
  }
  if (kbw + fb > 63) fail(GT_EOVERFLOW, "too many files x words for 64-bit (file, word) keys");
  const uint64_t pad = uint64_t(uint32_t(d.F)) << kbw;
  const int64_t n = d.root_len + g->bu_words;
  Phase ph(ctx, "bu_rows", s);
  Buf k0(ctx, size_t(n) * 8, s), v0(ctx, size_t(n) * 4, s), k1(ctx, size_t(n) * 8, s), v1(ctx, size_t(n) * 4, s);
  Buf ecnt(ctx, size_t(d.ER) * 8, s), epos(ctx, size_t(d.ER) * 8, s), sc(ctx, scan_scratch_bytes(d.ER), s);
  if (d.root_len > 0) {
    root_word_rows_kernel<<<grid_for(d.root_len, threads, cap), threads, 0, s>>>(d, kbw, pad, k0.as<uint64_t>(),
                                                                                  v0.as<uint32_t>());
    GT_LAUNCH_CHECK();
  }
  if (d.ER > 0) {
    redge_len_kernel<<<grid_for(d.ER, threads, cap), threads, 0, s>>>(d, false, ecnt.as<int64_t>());
    GT_LAUNCH_CHECK();
    exclusive_scan_i64(ecnt.as<int64_t>(), epos.as<int64_t>(), d.ER, sc.p, s);
    child_word_rows_kernel<<<grid_for(d.ER, 128, cap), 128, 0, s>>>(d, kbw, epos.as<int64_t>(),
                                                                     k0.as<uint64_t>() + d.root_len,
                                                                     v0.as<uint32_t>() + d.root_len);
    GT_LAUNCH_CHECK();
  }
  out.bound = n;
  out.word = Buf(ctx, size_t(n) * 4, s);
  out.file = Buf(ctx, size_t(n) * 4, s);
  out.cnt = Buf(ctx, size_t(n) * 8, s);
  out.total = Buf(ctx, 8, s);
  if (n == 0) {
    GT_CUDA(cudaMemsetAsync(out.total.p, 0, 8, s));
    return;
  }
  Buf rs(ctx, radix_scratch_bytes(n, true, 4), s);
  radix_sort_u64(k0.as<uint64_t>(), k1.as<uint64_t>(), v0.p, v1.p, 4, n, 0, kbw + fb, rs.p, s);
  Buf flag(ctx, size_t(n) * 8, s), pos(ctx, size_t(n) * 8, s), v64(ctx, size_t(n) * 8, s), wsum(ctx, size_t(n) * 8, s);
  Buf sc2(ctx, scan_scratch_bytes(n), s), start(ctx, size_t(n) * 8, s);
  reduce_flags_kernel<<<grid_for(n, threads, cap), threads, 0, s>>>(k1.as<uint64_t>(), v1.as<uint32_t>(), n, pad,
                                                                     flag.as<int64_t>(), v64.as<int64_t>());
  GT_LAUNCH_CHECK();
  exclusive_scan_i64(flag.as<int64_t>(), pos.as<int64_t>(), n, sc2.p, s);
  exclusive_scan_i64(v64.as<int64_t>(), wsum.as<int64_t>(), n, sc2.p, s);
  total_kernel<<<1, 1, 0, s>>>(pos.as<int64_t>(), flag.as<int64_t>(), n, out.total.as<int64_t>());
  GT_LAUNCH_CHECK();
  reduce_write_kernel<<<grid_for(n, threads, cap), threads, 0, s>>>(k1.as<uint64_t>(), n, flag.as<int64_t>(),
                                                                     pos.as<int64_t>(), kbw, out.word.as<int32_t>(),
                                                                     out.file.as<int32_t>(), start.as<int64_t>());
  GT_LAUNCH_CHECK();
  reduce_sum_kernel<<<grid_for(n, threads, cap), threads, 0, s>>>(start.as<int64_t>(), out.total.as<int64_t>(),
                                                                   wsum.as<int64_t>(), v64.as<int64_t>(), n,
                                                                   out.cnt.as<uint64_t>());
  GT_LAUNCH_CHECK();
}

gt_result* bu_inverted_index(gt_grammar* g, WordRows& wr, cudaStream_t s) {
  gt_ctx* ctx = g->ctx;
  const DevGrammar& d = g->d;
  const int threads = 256, cap = ctx->num_sms * 16;
  ResultBuilder rb(ctx, s);
  const int64_t n = wr.bound;
  auto* off = static_cast<int64_t*>(rb.alloc(size_t(d.V + 1) * 8));
  auto* files = static_cast<int32_t*>(rb.alloc(size_t(n) * 4));
  int64_t* len = rb.new_len_slot();
  GT_CUDA(cudaMemcpyAsync(len, wr.total.p, 8, cudaMemcpyDeviceToDevice, s));
  Buf k0(ctx, size_t(n) * 8, s), k1(ctx, size_t(n) * 8, s), f0(ctx, size_t(n) * 4, s);
  if (n > 0) {
    Buf rs(ctx, radix_scratch_bytes(n, true, 4), s);
    word_keys_kernel<<<grid_for(n, threads, cap), threads, 0, s>>>(wr.word.as<int32_t>(), wr.file.as<int32_t>(),
                                                                    wr.total.as<int64_t>(), n, d.V, k0.as<uint64_t>(),
                                                                    f0.as<uint32_t>());
    GT_LAUNCH_CHECK();
    radix_sort_u64(k0.as<uint64_t>(), k1.as<uint64_t>(), f0.p, files, 4, n, 0, bits_for(d.V), rs.p, s);
  }
  word_offsets_kernel<<<grid_for(int64_t(d.V) + 1, threads, cap), threads, 0, s>>>(k1.as<uint64_t>(),
                                                                                    wr.total.as<int64_t>(), d.V, off);
  GT_LAUNCH_CHECK();
  rb.field("offsets", off, int64_t(d.V) + 1);
  rb.field_dyn("file", files, len);
  return rb.finish();
}

}  // namespace

// Term vectors from the rows (offsets from the file column), and the
// inverted index; one set of rows serves every query.
void run_file_batch_bu(gt_grammar* g, const int* tv_topk, int n_tv, gt_result** tv_out, gt_result** ii_out,
                       cudaStream_t s) {
  WordRows wr;
  bu_word_rows(g, s, wr);
  const DevGrammar& d = g->d;
  if (n_tv > 0) {
    Buf toff(g->ctx, size_t(d.F + 1) * 8, s);
    file_offsets_kernel<<<grid_for(int64_t(d.F) + 1, 256, 4096), 256, 0, s>>>(wr.file.as<int32_t>(),
                                                                              wr.total.as<int64_t>(), d.F,
                                                                              toff.as<int64_t>());
    GT_LAUNCH_CHECK();
    for (int i = 0; i < n_tv; ++i)
      tv_out[i] = tv_from_arrays(g->ctx, wr.word.as<int32_t>(), wr.cnt.as<uint64_t>(), toff.as<int64_t>(),
                                 wr.total.as<int64_t>(), wr.bound, d.F, tv_topk[i], s, d.V);
  }
  if (ii_out) *ii_out = bu_inverted_index(g, wr, s);
}

gt_result* run_ranked_words_bu(gt_grammar* g, cudaStream_t s) {
  WordRows wr;
  bu_word_rows(g, s, wr);
  const int64_t n = wr.bound;
  gt_ctx* ctx = g->ctx;
  Buf rkey(ctx, size_t(n) * 8, s);
  if (n > 0) {
    widen_i32_kernel<<<grid_for(n, 256, ctx->num_sms * 16), 256, 0, s>>>(wr.word.as<int32_t>(), wr.total.as<int64_t>(),
                                                                          rkey.as<uint64_t>());
    GT_LAUNCH_CHECK();
  }
  return ranked_from_rows(ctx, rkey, wr.file, wr.cnt, wr.total.as<int64_t>(), n, 0, false, uint64_t(g->d.V),
                          uint64_t(g->max_file_len), s);
}

// Per-file window rows of small files, built per file in shared memory.
void bu_local_window_rows(gt_grammar* g, int kb, uint64_t key_pad, cudaStream_t s, Windows& out) {
  gt_ctx* ctx = g->ctx;
  const DevGrammar& d = g->d;
  const int64_t N = int64_t(d.N);
  const int cap = int(std::max<int64_t>(256, (g->max_file_len + 255) / 256 * 256));
  Phase ph(ctx, "bu_local", s);
  Buf soff(ctx, size_t(d.F + 1) * 8, s), flen(ctx, size_t(d.F + 1) * 8, s), sc(ctx, scan_scratch_bytes(d.F + 1), s);
  Buf sk(ctx, size_t(N) * 8, s), scn(ctx, size_t(N) * 4, s), nr(ctx, size_t(d.F + 1) * 8, s);
  Buf roff(ctx, size_t(d.F + 1) * 8, s);
  out.n = N;
  out.reduced = true;
  out.keys = Buf(ctx, size_t(N) * 8, s);
  out.rfile = Buf(ctx, size_t(N) * 4, s);
  out.rcnt = Buf(ctx, size_t(N) * 8, s);
  out.total = Buf(ctx, 8, s);
  file_len_i64_kernel<<<grid_for(int64_t(d.F) + 1, 256, ctx->num_sms * 8), 256, 0, s>>>(d.file_len, d.F,
                                                                                     flen.as<int64_t>());
  GT_LAUNCH_CHECK();
  exclusive_scan_i64(flen.as<int64_t>(), soff.as<int64_t>(), d.F + 1, sc.p, s);
  const size_t smem = size_t(cap) * 16;
  GT_CUDA(cudaFuncSetAttribute(local_window_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
  GT_CUDA(cudaMemsetAsync(nr.as<int64_t>() + d.F, 0, 8, s));
  local_window_rows_kernel<<<unsigned(std::min<int64_t>(d.F, 65535)), kLocalThreads, smem, s>>>(
      d, cap, kb, 3 * kb, soff.as<int64_t>(), sk.as<uint64_t>(), scn.as<uint32_t>(), nr.as<int64_t>());
  GT_LAUNCH_CHECK();
  exclusive_scan_i64(nr.as<int64_t>(), roff.as<int64_t>(), d.F + 1, sc.p, s);
  GT_CUDA(cudaMemcpyAsync(out.total.p, roff.as<int64_t>() + d.F, 8, cudaMemcpyDeviceToDevice, s));
  local_pack_windows_kernel<<<grid_for(int64_t(d.F) * 32, 256, ctx->num_sms * 16), 256, 0, s>>>(
      d.F, soff.as<int64_t>(), roff.as<int64_t>(), sk.as<uint64_t>(), scn.as<uint32_t>(), out.keys.as<uint64_t>(),
      out.rfile.as<int32_t>(), out.rcnt.as<uint64_t>());
  GT_LAUNCH_CHECK();
}

// Per-file window rows: windows owned by the root in each file, plus every
// window inside each (file, root child) expansion, weighted by multiplicity.
void bu_window_rows(gt_grammar* g, Buf& head, Buf& tail, int kb, uint64_t key_pad, cudaStream_t s, Windows& out) {
  gt_ctx* ctx = g->ctx;
  const DevGrammar& d = g->d;
  const int threads = 256, cap = ctx->num_sms * 16;
  if (d.depth > kMaxStack) fail(GT_EOVERFLOW, "bottom-up expansion supports DAG depth <= 64");
  if (g->max_file_len <= kLocalMax && gparam(g, "bu_local", 1)) {
    bu_local_window_rows(g, kb, key_pad, s, out);
    return;
  }
  const int64_t n = 2 * d.root_len + g->bu_windows;
  Phase ph(ctx, "bu_rows", s);
  Buf k0(ctx, size_t(n) * 8, s), f0(ctx, size_t(n) * 8, s), v0(ctx, size_t(n) * 4, s);
  Buf ecnt(ctx, size_t(d.ER) * 8, s), epos(ctx, size_t(d.ER) * 8, s), sc(ctx, scan_scratch_bytes(d.ER), s);
  if (d.root_len > 0) {
    root_window_rows_kernel<<<grid_for(d.root_len, threads, cap), threads, 0, s>>>(
        d, head.as<int32_t>(), tail.as<int32_t>(), kb, key_pad, k0.as<uint64_t>(), f0.as<uint64_t>(),
        v0.as<uint32_t>());
    GT_LAUNCH_CHECK();
  }
  if (d.ER > 0) {
    redge_len_kernel<<<grid_for(d.ER, threads, cap), threads, 0, s>>>(d, true, ecnt.as<int64_t>());
    GT_LAUNCH_CHECK();
    exclusive_scan_i64(ecnt.as<int64_t>(), epos.as<int64_t>(), d.ER, sc.p, s);
    child_window_rows_kernel<<<grid_for(d.ER, 128, cap), 128, 0, s>>>(
        d, kb, epos.as<int64_t>(), k0.as<uint64_t>() + 2 * d.root_len, f0.as<uint64_t>() + 2 * d.root_len,
        v0.as<uint32_t>() + 2 * d.root_len);
    GT_LAUNCH_CHECK();
  }
  sort_by_file_key(ctx, k0, f0, v0, n, 3 * kb + 1, bits_for(d.F), s, out);
}

}  // namespace gt
