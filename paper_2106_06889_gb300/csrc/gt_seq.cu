// Sequence count (l = 3) and the ranked inverted index (Section IV-C/D).
//
// Every 3-word window of a file lies inside the expansion of exactly one
// lowest rule occurrence: the rule whose body it crosses (it touches two or
// more body symbols).  That rule "owns" the window, and the window occurs as
// many times as the rule does (its top-down weight).  So instead of the
// paper's two traversal phases with retry-on-unready relaunches, the engine
//   1. builds the head/tail buffers bottom-up (first and last two words of
//      every rule's expansion);
//   2. enumerates, for every body position j, the windows that start in
//      symbol j and leave it: a word starts one window, a child rule with two
//      or more words starts two (at its last two words).  Their words come from
//      the symbol, the next two body symbols (look-ahead that stops at the end
//      of the rule, or of the file in the root) and children's head/tail
//      buffers - the boundary fix-up between rule pieces;
//   3. weights each window by its rule's weight (global counts) or by the
//      rule's per-file weights (per-file counts);
//   4. canonicalises: radix sort by key, then a segmented sum per key.
// For rule r this yields W_r + 2 S_r - 2 windows when all children expand to
// two or more words - Eq. 1's bound with l = 3, which is then exact.
#include <algorithm>

#include "gt_device.cuh"

namespace gt {
namespace {

// Global counts, compacted: every owned window gets one row, in body
// position order.  One CTA per tile of kTile symbols (4 per thread); each
// tile's first row comes from the per-grammar tile offsets (the windows of
// every tile counted and scanned once, seq_tile_offsets), and the emit pass
// ranks the windows inside the tile.
constexpr int kWinThreads = kTile / 4;

// Exclusive prefix of v over the CTA (kWinThreads threads); *total gets the sum.
__device__ __forceinline__ int cta_excl_scan(int v, int* total) {
  __shared__ int warp_tot[kWinThreads / 32];
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
  for (int w = 0; w < kWinThreads / 32; ++w) {
    const int t = warp_tot[w];
    before += w < warp ? t : 0;
    all += t;
  }
  __syncthreads();
  *total = all;
  return before + incl - v;
}

// Rows of rules nothing references (weight 0) get the pad key.  Rows past
// `bound` are not written; the status word records it.
__global__ void __launch_bounds__(kWinThreads) win_emit_kernel(DevGrammar d, const int32_t* __restrict__ head,
                                                               const int32_t* __restrict__ tail,
                                                               const uint64_t* __restrict__ wt, int kb,
                                                               uint64_t key_pad, const int64_t* __restrict__ tile_off,
                                                               int64_t bound, uint64_t* __restrict__ keys,
                                                               uint32_t* __restrict__ vals,
                                                               unsigned* __restrict__ status) {
  TileWin t;
  const int c = tile_windows(d, head, tail, kb, int64_t(blockIdx.x) * kTile + threadIdx.x * 4, t);
  // the tile's first row and the owners' weights are requested before the
  // scan's barriers, so they arrive while the CTA ranks its windows
  const int64_t first = tile_off[blockIdx.x];
  uint32_t wv[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) wv[i] = t.n[i] ? uint32_t(wt[t.r[i]]) : 0u;
  int total;
  int64_t pos = first + cta_excl_scan(c, &total);
  bool over = false;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const uint32_t w = wv[i];
#pragma unroll
    for (int q = 0; q < 2; ++q)
      if (q < t.n[i]) {
        if (pos < bound) {
          keys[pos] = w ? t.k[i][q] : key_pad;
          vals[pos] = w;
        } else {
          over = true;
        }
        ++pos;
      }
  }
  if (over) atomicOr(status, ST_OVERFLOW);
}

// Per-file counts, pass 1: entries produced at each position (windows x files).
__global__ void win_count_file_kernel(DevGrammar d, const int32_t* __restrict__ head,
                                      const int32_t* __restrict__ tail, const unsigned long long* __restrict__ mask,
                                      int kb, int64_t* __restrict__ cnt) {
  for (int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; j < d.G; j += int64_t(gridDim.x) * blockDim.x) {
    int32_t r, f;
    const int64_t end = seq_end(d, j, &r, &f);
    uint64_t k[2];
    const int n = windows_at(d, head, tail, j, end, kb, k);
    cnt[j] = r == 0 ? n : n * __popcll(mask[r]);
  }
}

// Pass 2: write (file << 32 | slot) and the key of every entry.
__global__ void win_emit_file_kernel(DevGrammar d, const int32_t* __restrict__ head, const int32_t* __restrict__ tail,
                                     const unsigned long long* __restrict__ mask, const int64_t* __restrict__ woff,
                                     const uint32_t* __restrict__ slot_pair, const uint32_t* __restrict__ fw, int kb,
                                     const int64_t* __restrict__ pos,
                                     uint64_t* __restrict__ keys, uint64_t* __restrict__ fkeys,
                                     uint32_t* __restrict__ vals) {
  for (int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; j < d.G; j += int64_t(gridDim.x) * blockDim.x) {
    int32_t r, f;
    const int64_t end = seq_end(d, j, &r, &f);
    uint64_t k[2];
    const int n = windows_at(d, head, tail, j, end, kb, k);
    if (n == 0) continue;
    int64_t o = pos[j];
    if (r == 0) {
      for (int i = 0; i < n; ++i, ++o) {
        keys[o] = k[i];
        fkeys[o] = uint64_t(uint32_t(f));
        vals[o] = 1u;
      }
    } else {
      unsigned long long m = mask[r];
      int64_t slot = woff[r];
      while (m) {
        const int ff = __ffsll(m) - 1;
        m &= m - 1;
        const uint32_t w = fw[slot_pair[slot++]];
        for (int i = 0; i < n; ++i, ++o) {
          keys[o] = k[i];
          fkeys[o] = uint64_t(uint32_t(ff));
          vals[o] = w;
        }
      }
    }
  }
}

__global__ void pad_tail_kernel(uint64_t* __restrict__ keys, uint64_t* __restrict__ fkeys,
                                uint32_t* __restrict__ vals, const int64_t* __restrict__ n_dev, int64_t bound,
                                uint64_t key_pad, uint64_t file_pad) {
  const int64_t n = *n_dev;
  for (int64_t i = n + blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < bound; i += int64_t(gridDim.x) * blockDim.x) {
    keys[i] = key_pad;
    if (fkeys) fkeys[i] = file_pad;
    if (vals) vals[i] = 0;
  }
}

// Rows that are already one per (file, key): keys to 21-bit fields, copied.
__global__ void reduced_rows_out_kernel(const uint64_t* __restrict__ keys, const int32_t* __restrict__ file,
                                        const uint64_t* __restrict__ cnt, const int64_t* __restrict__ n_dev, int kb,
                                        uint64_t* __restrict__ okey, int32_t* __restrict__ ofile,
                                        uint64_t* __restrict__ ocnt) {
  const int64_t n = *n_dev;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    okey[i] = to_output_key(keys[i], kb);
    if (ofile) ofile[i] = file[i];
    ocnt[i] = cnt[i];
  }
}

__global__ void last_total2_kernel(const int64_t* __restrict__ ex, const int64_t* __restrict__ cnt, int64_t n,
                                   int64_t* __restrict__ out, int64_t* __restrict__ out2) {
  const int64_t t = n > 0 ? ex[n - 1] + cnt[n - 1] : 0;
  *out = t;
  if (out2) *out2 = t;
}

__global__ void pack_hi_lo_kernel(const uint64_t* __restrict__ hi, const uint32_t* __restrict__ lo, int64_t n,
                                  uint64_t* __restrict__ out) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    out[i] = (hi[i] << 32) | lo[i];
}

__global__ void unpack_hi_lo_kernel(const uint64_t* __restrict__ in, int64_t n, uint64_t* __restrict__ hi,
                                    uint32_t* __restrict__ lo) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const uint64_t x = in[i];
    hi[i] = x >> 32;
    lo[i] = uint32_t(x);
  }
}

int bits_for(int64_t x) {
  int b = 1;
  while ((int64_t(1) << b) <= x) ++b;
  return b;
}

// Segmented sum over sorted rows: one output row per run of equal (file, key),
// pad-key rows skipped.  Pass 1, per tile of 2048 rows: the number of run
// heads, the sum of the rows before the first head (the tail of a run that
// started in an earlier tile) and whether the whole tile continues such a run.
// After a scan of the head counts, pass 2 stages the tile in shared memory,
// gives each head its output index and sums its run up to the tile end, then
// adds the leading sums of the following tiles while the run continues - so a
// hot key's long run costs one pass over its tiles, not one thread per row.
constexpr int kRedThreads = 256;
constexpr int kRedItems = 8;
constexpr int kRedTile = kRedThreads * kRedItems;

__device__ __forceinline__ bool red_same(const uint64_t* __restrict__ keys, const uint64_t* __restrict__ fkeys,
                                         int64_t i, int64_t j) {
  return keys[i] == keys[j] && (!fkeys || fkeys[i] == fkeys[j]);
}

__device__ __forceinline__ int red_block_scan(int v, int* total) {
  __shared__ int warp_tot[kRedThreads / 32];
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
  for (int w = 0; w < kRedThreads / 32; ++w) {
    const int t = warp_tot[w];
    before += w < warp ? t : 0;
    all += t;
  }
  __syncthreads();
  *total = all;
  return before + incl - v;
}

__global__ void __launch_bounds__(kRedThreads) red_count_kernel(const uint64_t* __restrict__ keys,
                                                                const uint64_t* __restrict__ fkeys,
                                                                const uint32_t* __restrict__ vals, int64_t n,
                                                                uint64_t key_pad, int64_t* __restrict__ tcnt,
                                                                unsigned long long* __restrict__ lead,
                                                                int* __restrict__ passes) {
  __shared__ int first_head, any_pad;
  __shared__ unsigned long long lsum;
  const int64_t base = int64_t(blockIdx.x) * kRedTile;
  const int64_t end = min(n, base + kRedTile);
  if (threadIdx.x == 0) {
    first_head = kRedTile;
    any_pad = 0;
    lsum = 0;
  }
  __syncthreads();
  int c = 0;
#pragma unroll
  for (int k = 0; k < kRedItems; ++k) {  // consecutive threads, consecutive rows
    const int64_t i = base + k * kRedThreads + threadIdx.x;
    if (i >= end) continue;
    const bool pad = keys[i] == key_pad;
    const bool head = !pad && (i == 0 || !red_same(keys, fkeys, i, i - 1));
    c += head;
    if (head) atomicMin(&first_head, int(i - base));
    if (pad) any_pad = 1;
  }
  int total;
  red_block_scan(c, &total);  // also orders the shared updates above
  unsigned long long part = 0;
#pragma unroll
  for (int k = 0; k < kRedItems; ++k) {
    const int64_t i = base + k * kRedThreads + threadIdx.x;
    if (i < end && i - base < first_head && keys[i] != key_pad) part += vals[i];
  }
  if (part) atomicAdd(&lsum, part);
  __syncthreads();
  if (threadIdx.x == 0) {
    tcnt[blockIdx.x] = total;
    lead[blockIdx.x] = lsum;
    passes[blockIdx.x] = (total == 0 && !any_pad && end - base == kRedTile) ? 1 : 0;
  }
}

__global__ void __launch_bounds__(kRedThreads) red_write_kernel(const uint64_t* __restrict__ keys,
                                                                const uint64_t* __restrict__ fkeys,
                                                                const uint32_t* __restrict__ vals, int64_t n,
                                                                uint64_t key_pad, const int64_t* __restrict__ toff,
                                                                const unsigned long long* __restrict__ lead,
                                                                const int* __restrict__ passes, int64_t tiles, int kb,
                                                                uint64_t* __restrict__ out_key,
                                                                int32_t* __restrict__ out_file,
                                                                uint64_t* __restrict__ out_count) {
  __shared__ uint64_t sk[kRedTile];
  __shared__ uint32_t sv[kRedTile];
  __shared__ uint32_t sf[kRedTile];  // files fit 32 bits
  const int64_t base = int64_t(blockIdx.x) * kRedTile;
  const int len = int(min(n - base, int64_t(kRedTile)));
  int64_t o0 = toff[blockIdx.x];  // requested with the tile, before the barrier
  for (int r = threadIdx.x; r < len; r += kRedThreads) {
    sk[r] = keys[base + r];
    sv[r] = vals[base + r];
    if (fkeys) sf[r] = uint32_t(fkeys[base + r]);
  }
  __syncthreads();
  for (int k = 0; k < kRedItems; ++k) {  // one 256-row step at a time, in row order
    const int r = k * kRedThreads + threadIdx.x;
    const int64_t i = base + r;
    bool h = false;
    if (r < len && sk[r] != key_pad) {
      if (r > 0)
        h = sk[r] != sk[r - 1] || (fkeys && sf[r] != sf[r - 1]);
      else
        h = i == 0 || !red_same(keys, fkeys, i, i - 1);
    }
    int step;
    const int64_t o = o0 + red_block_scan(h ? 1 : 0, &step);
    o0 += step;
    if (!h) continue;
    const uint64_t key = sk[r];
    const uint32_t f = fkeys ? sf[r] : 0u;
    unsigned long long sum = sv[r];
    int q = r + 1;
    while (q < len && sk[q] == key && (!fkeys || sf[q] == f)) sum += sv[q++];
    if (q == len)  // the run reaches the tile end: add the leading sums of the next tiles
      for (int64_t t = int64_t(blockIdx.x) + 1; t < tiles; ++t) {
        sum += lead[t];
        if (!passes[t]) break;
      }
    out_key[o] = to_output_key(key, kb);
    if (out_file) out_file[o] = int32_t(f);
    out_count[o] = sum;
  }
}

void reduce_rows(gt_ctx* ctx, uint64_t* keys, uint64_t* fkeys, uint32_t* vals, int64_t n, int kb, uint64_t key_pad,
                 uint64_t* out_key, int32_t* out_file, uint64_t* out_count, int64_t* nrows_slot, cudaStream_t s,
                 bool output_keys = true) {
  if (n == 0) {
    GT_CUDA(cudaMemsetAsync(nrows_slot, 0, 8, s));
    return;
  }
  const int64_t tiles = (n + kRedTile - 1) / kRedTile;
  Buf tcnt(ctx, size_t(tiles + 1) * 8, s), toff(ctx, size_t(tiles + 1) * 8, s), sc(ctx, scan_scratch_bytes(tiles + 1), s);
  Buf lead(ctx, size_t(tiles) * 8, s), pass(ctx, size_t(tiles) * 4, s);
  GT_CUDA(cudaMemsetAsync(tcnt.as<int64_t>() + tiles, 0, 8, s));
  red_count_kernel<<<unsigned(tiles), kRedThreads, 0, s>>>(keys, fkeys, vals, n, key_pad, tcnt.as<int64_t>(),
                                                            lead.as<unsigned long long>(), pass.as<int>());
  GT_LAUNCH_CHECK();
  exclusive_scan_i64(tcnt.as<int64_t>(), toff.as<int64_t>(), tiles + 1, sc.p, s);
  GT_CUDA(cudaMemcpyAsync(nrows_slot, toff.as<int64_t>() + tiles, 8, cudaMemcpyDeviceToDevice, s));
  red_write_kernel<<<unsigned(tiles), kRedThreads, 0, s>>>(keys, fkeys, vals, n, key_pad, toff.as<int64_t>(),
                                                            lead.as<unsigned long long>(), pass.as<int>(), tiles,
                                                            output_keys ? kb : 0, out_key, out_file, out_count);
  GT_LAUNCH_CHECK();
}

}  // namespace

// Rows sorted by (file, key): a stable sort by key carrying (file << 32 |
// value) as a 64-bit payload, then a stable sort of that payload on its file
// bits carrying the key - no permutation is applied afterwards.
void sort_by_file_key(gt_ctx* ctx, Buf& k0, Buf& f0, Buf& v0, int64_t bound, int key_bits, int file_bits,
                      cudaStream_t s, Windows& out) {
  const int threads = 256, cap = ctx->num_sms * 16;
  out.keys = Buf(ctx, size_t(bound) * 8, s);
  out.fkeys = Buf(ctx, size_t(bound) * 8, s);
  out.vals = Buf(ctx, size_t(bound) * 4, s);
  out.n = bound;
  if (bound == 0) return;
  Phase ph2(ctx, "seq_sort", s);
  Buf p0(ctx, size_t(bound) * 8, s), p1(ctx, size_t(bound) * 8, s), k1(ctx, size_t(bound) * 8, s);
  Buf q(ctx, size_t(bound) * 8, s), rs(ctx, radix_scratch_bytes(bound, true, 8), s);
  pack_hi_lo_kernel<<<grid_for(bound, threads, cap), threads, 0, s>>>(f0.as<uint64_t>(), v0.as<uint32_t>(), bound,
                                                                       p0.as<uint64_t>());
  GT_LAUNCH_CHECK();
  radix_sort_u64(k0.as<uint64_t>(), k1.as<uint64_t>(), p0.p, p1.p, 8, bound, 0, key_bits, rs.p, s);
  radix_sort_u64(p1.as<uint64_t>(), q.as<uint64_t>(), k1.p, out.keys.p, 8, bound, 32, 32 + file_bits, rs.p, s);
  unpack_hi_lo_kernel<<<grid_for(bound, threads, cap), threads, 0, s>>>(q.as<uint64_t>(), bound,
                                                                         out.fkeys.as<uint64_t>(),
                                                                         out.vals.as<uint32_t>());
  GT_LAUNCH_CHECK();
}

namespace {

// Device-detected failures go to *status (the result's own status word).
void sorted_windows(gt_grammar* g, bool per_file, cudaStream_t s, Windows& out, uint32_t* status) {
  gt_ctx* ctx = g->ctx;
  const DevGrammar& d = g->d;
  const int threads = 256, cap = ctx->num_sms * 16;
  if (d.V > (1 << 21)) fail(GT_EOVERFLOW, "3-word keys need num_words <= 2^21");
  if (d.N >= (uint64_t(1) << 32)) fail(GT_EOVERFLOW, "sequence count needs fewer than 2^32 tokens per grammar");
  const int kb = bits_for(d.V > 1 ? d.V - 1 : 1);  // bits per word id
  out.kb = kb;
  out.key_pad = uint64_t(1) << (3 * kb);  // above every real key: unused rows sort last
  const int key_bits = 3 * kb + 1;
  Buf head(ctx, size_t(d.R) * 8, s), tail(ctx, size_t(d.R) * 8, s);
  {
    Phase ph(ctx, "seq_headtail", s);
    run_head_tail(g, head.as<int32_t>(), tail.as<int32_t>(), s);
  }
  if (!per_file) {
    // exactly the owned windows (Eq. 1's count, known since load); the pad
    // key fills any rows the emit pass leaves
    const int64_t n = g->info.owned_windows;
    Buf k0(ctx, size_t(n) * 8, s), v0(ctx, size_t(n) * 4, s);
    out.keys = Buf(ctx, size_t(n) * 8, s);
    out.vals = Buf(ctx, size_t(n) * 4, s);
    out.n = n;
    if (n == 0) return;
    {
      Phase ph(ctx, "seq_emit", s);
      Buf wt(ctx, size_t(d.R) * 8, s);
      run_rule_weights(g, wt.as<uint64_t>(), s);
      const int64_t nt = d.ntiles;
      // each tile's first row: structure of the grammar, counted once and kept
      const int64_t* toff = seq_tile_offsets(g, head.as<int32_t>(), tail.as<int32_t>(), kb, s);
      win_emit_kernel<<<unsigned(nt), kWinThreads, 0, s>>>(d, head.as<int32_t>(), tail.as<int32_t>(),
                                                            wt.as<uint64_t>(), kb, out.key_pad, toff, n,
                                                            k0.as<uint64_t>(), v0.as<uint32_t>(), status);
      GT_LAUNCH_CHECK();
      pad_tail_kernel<<<grid_for(n, threads, cap), threads, 0, s>>>(k0.as<uint64_t>(), nullptr, v0.as<uint32_t>(),
                                                                     toff + nt, n, out.key_pad, 0);
      GT_LAUNCH_CHECK();
    }
    Phase ph(ctx, "seq_sort", s);
    Buf rs(ctx, radix_scratch_bytes(n, true, 4), s);
    radix_sort_u64(k0.as<uint64_t>(), out.keys.as<uint64_t>(), v0.p, out.vals.p, 4, n, 0, key_bits, rs.p, s);
    return;
  }
  if (file_strategy(g) == 2) {
    bu_window_rows(g, head, tail, kb, out.key_pad, s, out);
    return;
  }
  // ---- per file, top-down: count, scan, emit (windows x files of the rule) ----
  Phase ph(ctx, "seq_emit", s);
  FileWeights fw;
  file_weights(g, s, fw);
  const int64_t bound = 2 * d.root_len + 2 * g->fsym_bound;
  if (bound == 0) {
    out.n = 0;
    return;
  }
  Buf cnt(ctx, size_t(d.G) * 8, s), pos(ctx, size_t(d.G) * 8, s), sc(ctx, scan_scratch_bytes(d.G), s), nd(ctx, 8, s);
  GT_CUDA(cudaMemsetAsync(nd.p, 0, 8, s));
  Buf k0(ctx, size_t(bound) * 8, s), f0(ctx, size_t(bound) * 8, s), v0(ctx, size_t(bound) * 4, s);
  if (d.G > 0) {
    win_count_file_kernel<<<grid_for(d.G, threads, cap), threads, 0, s>>>(
        d, head.as<int32_t>(), tail.as<int32_t>(), fw.mask, kb, cnt.as<int64_t>());
    GT_LAUNCH_CHECK();
    exclusive_scan_i64(cnt.as<int64_t>(), pos.as<int64_t>(), d.G, sc.p, s);
    last_total2_kernel<<<1, 1, 0, s>>>(pos.as<int64_t>(), cnt.as<int64_t>(), d.G, nd.as<int64_t>(), nullptr);
    GT_LAUNCH_CHECK();
    win_emit_file_kernel<<<grid_for(d.G, threads, cap), threads, 0, s>>>(
        d, head.as<int32_t>(), tail.as<int32_t>(), fw.mask, fw.off, fw.slot_pair,
        fw.w.as<uint32_t>(), kb, pos.as<int64_t>(), k0.as<uint64_t>(), f0.as<uint64_t>(), v0.as<uint32_t>());
    GT_LAUNCH_CHECK();
  }
  pad_tail_kernel<<<grid_for(bound, threads, cap), threads, 0, s>>>(k0.as<uint64_t>(), f0.as<uint64_t>(),
                                                                     v0.as<uint32_t>(), nd.as<int64_t>(), bound,
                                                                     out.key_pad, uint64_t(d.F));
  GT_LAUNCH_CHECK();
  sort_by_file_key(ctx, k0, f0, v0, bound, key_bits, bits_for(d.F), s, out);
}

// (max_count - count) << 32 | file: ascending = count descending (counts of a
// key in a file never exceed max_count, the longest file's length).
__global__ void rank_keys_kernel(const uint64_t* __restrict__ cnt, const int32_t* __restrict__ file,
                                 const int64_t* __restrict__ n_dev, int64_t bound, uint64_t max_count,
                                 uint64_t* __restrict__ k) {
  const int64_t n = *n_dev;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < bound; i += int64_t(gridDim.x) * blockDim.x)
    k[i] = i < n ? ((max_count - cnt[i]) << 32) | uint32_t(file[i]) : (max_count << 32);
}

__global__ void rank_unpack_kernel(const uint64_t* __restrict__ pay, int64_t n, uint64_t max_count,
                                   int32_t* __restrict__ file, uint64_t* __restrict__ cnt) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const uint64_t x = pay[i];
    file[i] = int32_t(uint32_t(x));
    cnt[i] = max_count - (x >> 32);
  }
}

__global__ void key_heads_kernel(const uint64_t* __restrict__ key, const int64_t* __restrict__ n_dev, int64_t bound,
                                 int64_t* __restrict__ flag) {
  const int64_t n = *n_dev;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < bound; i += int64_t(gridDim.x) * blockDim.x)
    flag[i] = (i < n && (i == 0 || key[i] != key[i - 1])) ? 1 : 0;
}

__global__ void key_offsets_kernel(const uint64_t* __restrict__ key, const int64_t* __restrict__ flag,
                                   const int64_t* __restrict__ pos, const int64_t* __restrict__ n_dev, int64_t bound,
                                   int kb, bool windows, int64_t* __restrict__ off, uint64_t* __restrict__ okey,
                                   int64_t* __restrict__ nkeys, int64_t* __restrict__ nkeys1) {
  const int64_t n = *n_dev;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < bound; i += int64_t(gridDim.x) * blockDim.x)
    if (flag[i]) {
      off[pos[i]] = i;
      okey[pos[i]] = windows ? to_output_key(key[i], kb) : key[i];
    }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const int64_t nk = bound > 0 ? pos[bound - 1] + flag[bound - 1] : 0;
    off[nk] = n;
    *nkeys = nk;
    *nkeys1 = nk + 1;
  }
}

}  // namespace

// Rows (key, file, count), n_dev of them (bound allocated) -> ranked index:
// keys ascending; inside a key, count descending then file ascending.
gt_result* ranked_from_rows(gt_ctx* ctx, Buf& rkey, Buf& rfile, Buf& rcnt, const int64_t* n_dev, int64_t bound,
                            int kb, bool windows, uint64_t key_pad, uint64_t max_count, cudaStream_t s) {
  const int threads = 256, cap = ctx->num_sms * 16;
  ResultBuilder rb(ctx, s);
  Phase ph(ctx, "ranked", s);
  auto* off = static_cast<int64_t*>(rb.alloc(size_t(bound + 1) * 8));
  auto* okey = static_cast<uint64_t*>(rb.alloc(size_t(bound) * 8));
  auto* ofile = static_cast<int32_t*>(rb.alloc(size_t(bound) * 4));
  auto* ocnt = static_cast<uint64_t*>(rb.alloc(size_t(bound) * 8));
  int64_t* len_off = rb.new_len_slot();
  int64_t* len_key = rb.new_len_slot();
  int64_t* len_row = rb.new_len_slot();
  GT_CUDA(cudaMemcpyAsync(len_row, n_dev, 8, cudaMemcpyDeviceToDevice, s));
  if (bound == 0) {
    GT_CUDA(cudaMemsetAsync(off, 0, 8, s));
    GT_CUDA(cudaMemsetAsync(len_key, 0, 8, s));
    const int64_t one = 1;
    GT_CUDA(cudaMemcpyAsync(len_off, &one, 8, cudaMemcpyHostToDevice, s));
  } else {
    // sort 1: stable by count descending, key ((max_count - count) << 32 |
    // file), payload the row key; sort 2: stable by row key, payload sort 1's key
    Buf k0(ctx, size_t(bound) * 8, s), k1(ctx, size_t(bound) * 8, s), v1(ctx, size_t(bound) * 8, s);
    Buf pay(ctx, size_t(bound) * 8, s), rs(ctx, radix_scratch_bytes(bound, true, 8), s), skey(ctx, size_t(bound) * 8, s);
    Buf flag(ctx, size_t(bound) * 8, s), pos(ctx, size_t(bound) * 8, s), sc(ctx, scan_scratch_bytes(bound), s);
    // rows past n_dev must carry the pad key so they sort last
    pad_tail_kernel<<<grid_for(bound, threads, cap), threads, 0, s>>>(rkey.as<uint64_t>(), nullptr, nullptr, n_dev,
                                                                       bound, key_pad, 0);
    GT_LAUNCH_CHECK();
    if (max_count >= (uint64_t(1) << 31)) fail(GT_EOVERFLOW, "ranked index counts need files below 2^31 tokens");
    rank_keys_kernel<<<grid_for(bound, threads, cap), threads, 0, s>>>(rcnt.as<uint64_t>(), rfile.as<int32_t>(), n_dev,
                                                                        bound, max_count, k0.as<uint64_t>());
    GT_LAUNCH_CHECK();
    int cbits = 1;
    while (cbits < 32 && (uint64_t(1) << cbits) <= max_count) ++cbits;
    radix_sort_u64(k0.as<uint64_t>(), k1.as<uint64_t>(), rkey.p, v1.p, 8, bound, 32, 32 + cbits, rs.p, s);
    int kbits = 1;
    while (kbits < 64 && (uint64_t(1) << kbits) <= key_pad) ++kbits;
    radix_sort_u64(v1.as<uint64_t>(), skey.as<uint64_t>(), k1.p, pay.p, 8, bound, 0, kbits, rs.p, s);
    rank_unpack_kernel<<<grid_for(bound, threads, cap), threads, 0, s>>>(pay.as<uint64_t>(), bound, max_count, ofile,
                                                                          ocnt);
    GT_LAUNCH_CHECK();
    key_heads_kernel<<<grid_for(bound, threads, cap), threads, 0, s>>>(skey.as<uint64_t>(), n_dev, bound,
                                                                        flag.as<int64_t>());
    GT_LAUNCH_CHECK();
    exclusive_scan_i64(flag.as<int64_t>(), pos.as<int64_t>(), bound, sc.p, s);
    key_offsets_kernel<<<grid_for(bound, threads, cap), threads, 0, s>>>(
        skey.as<uint64_t>(), flag.as<int64_t>(), pos.as<int64_t>(), n_dev, bound, kb, windows, off, okey, len_key,
        len_off);
    GT_LAUNCH_CHECK();
  }
  rb.field_dyn("offsets", off, len_off);
  rb.field_dyn("key", okey, len_key);
  rb.field_dyn("file", ofile, len_row);
  rb.field_dyn("count", ocnt, len_row);
  return rb.finish();
}

gt_result* reduce_key_rows(gt_ctx* ctx, Buf& keys, Buf& vals, int64_t n, int key_bits, uint64_t key_pad,
                           cudaStream_t s, const uint32_t* status_in) {
  ResultBuilder rb(ctx, s);
  auto* key = static_cast<uint64_t*>(rb.alloc(size_t(n) * 8));
  auto* count = static_cast<uint64_t*>(rb.alloc(size_t(n) * 8));
  int64_t* len = rb.new_len_slot();
  if (n > 0) {
    Phase ph(ctx, "rows_sort", s);
    Buf k1(ctx, size_t(n) * 8, s), v1(ctx, size_t(n) * 4, s), rs(ctx, radix_scratch_bytes(n, true, 4), s);
    radix_sort_u64(keys.as<uint64_t>(), k1.as<uint64_t>(), vals.p, v1.p, 4, n, 0, key_bits, rs.p, s);
    reduce_rows(ctx, k1.as<uint64_t>(), nullptr, v1.as<uint32_t>(), n, 0, key_pad, key, nullptr, count, len, s,
                false);
  } else {
    GT_CUDA(cudaMemsetAsync(len, 0, 8, s));
  }
  rb.field_dyn("key", key, len);
  rb.field_dyn("count", count, len);
  if (status_in) GT_CUDA(cudaMemcpyAsync(rb.status(), status_in, 4, cudaMemcpyDeviceToDevice, s));
  return rb.finish();
}

gt_result* run_ranked_windows(gt_grammar* g, cudaStream_t s) {
  gt_ctx* ctx = g->ctx;
  Windows w;
  Buf st(ctx, 4, s);  // no kernel of the per-file window paths raises a flag
  GT_CUDA(cudaMemsetAsync(st.p, 0, 4, s));
  sorted_windows(g, true, s, w, st.as<uint32_t>());
  if (w.reduced)
    return ranked_from_rows(ctx, w.keys, w.rfile, w.rcnt, w.total.as<int64_t>(), w.n, w.kb, true, w.key_pad,
                            uint64_t(g->max_file_len), s);
  // per-file 3-gram rows (file, key, count) in (file, key) order
  Buf rkey(ctx, size_t(w.n) * 8, s), rfile(ctx, size_t(w.n) * 4, s), rcnt(ctx, size_t(w.n) * 8, s), nd(ctx, 8, s);
  reduce_rows(ctx, w.keys.as<uint64_t>(), w.fkeys.as<uint64_t>(), w.vals.as<uint32_t>(), w.n, w.kb, w.key_pad,
              rkey.as<uint64_t>(), rfile.as<int32_t>(), rcnt.as<uint64_t>(), nd.as<int64_t>(), s, false);
  return ranked_from_rows(ctx, rkey, rfile, rcnt, nd.as<int64_t>(), w.n, w.kb, true, w.key_pad,
                          uint64_t(g->max_file_len), s);
}

gt_result* run_sequence_count(gt_grammar* g, int per_file, cudaStream_t s) {
  // global count: the one-row-per-window radix sort (default, measured faster
  // on the 500M-token corpus) or the sample-sort buckets (seq_path = 2)
  if (!per_file && gparam(g, "seq_path", 1) == 2) return run_sequence_count_global(g, s);
  gt_ctx* ctx = g->ctx;
  ResultBuilder rb(ctx, s);
  Windows w;
  sorted_windows(g, per_file != 0, s, w, rb.status());
  Phase ph(ctx, "seq_reduce", s);
  auto* key = static_cast<uint64_t*>(rb.alloc(size_t(w.n) * 8));
  auto* count = static_cast<uint64_t*>(rb.alloc(size_t(w.n) * 8));
  int32_t* file = per_file ? static_cast<int32_t*>(rb.alloc(size_t(w.n) * 4)) : nullptr;
  int64_t* len = rb.new_len_slot();
  if (w.reduced) {
    GT_CUDA(cudaMemcpyAsync(len, w.total.p, 8, cudaMemcpyDeviceToDevice, s));
    if (w.n > 0) {
      reduced_rows_out_kernel<<<grid_for(w.n, 256, ctx->num_sms * 16), 256, 0, s>>>(
          w.keys.as<uint64_t>(), w.rfile.as<int32_t>(), w.rcnt.as<uint64_t>(), w.total.as<int64_t>(), w.kb, key, file,
          count);
      GT_LAUNCH_CHECK();
    }
  } else {
    reduce_rows(ctx, w.keys.as<uint64_t>(), per_file ? w.fkeys.as<uint64_t>() : nullptr, w.vals.as<uint32_t>(), w.n,
                w.kb, w.key_pad, key, file, count, len, s);
  }
  if (per_file) rb.field_dyn("file", file, len);
  rb.field_dyn("key", key, len);
  rb.field_dyn("count", count, len);
  return rb.finish();
}

}  // namespace gt
