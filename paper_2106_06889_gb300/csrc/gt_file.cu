// Per-file analytics: term vector and inverted index (Section VI), with the
// top-down traversal of Section IV-A, which carries per-rule file information
// from the root down (the strategy the paper picks when there are few files).
//
// GB300 form, for up to 64 files.  At load (structure only):
//   1. file masks, top-down: mask[r] = files whose expansion contains rule r,
//      a 64-bit set per rule, ORed over parents level by level;
//   2. memory pool: popcount(mask) slots per rule, level by level, each slot's
//      (file, rule) pair in file-major order, the root's references by pair,
//      and each slot's row of (parent's pair, mult);
//   3. every file's rule words, bucket-sorted per chunk, each entry naming its
//      pair.
// Per query:
//   4. per-file weights, level by level: weight (r, f) = occurrences of r in
//      file f = the root's references plus the row's mult * parent weight;
//   5. the root's chunks sorted by 2^14-word bucket; one CTA per (file,
//      bucket) builds a dense shared-memory histogram from the file's root
//      runs and weighted rule-word runs - the CTAs of one file run together,
//      so the file's data is read from HBM once and from L2 by the others -
//      and writes the bucket's nonzero counts in word order plus a bit per
//      word for the inverted index;
//   6. the (file, bucket) pieces are copied into the term vector (adding the
//      word count on the way when it is asked for) and the bits become
//      ascending file lists for the inverted index (one pass, bounded
//      look-back for the offsets).
#include <algorithm>

#include <vector>

#include "gt_device.cuh"

namespace gt {
namespace {

constexpr int kFBLog2 = 14;
constexpr int kFBucket = 1 << kFBLog2;
constexpr int kTvThreads = 512;
constexpr int kBinsPerThread = kFBucket / kTvThreads;  // 32: one mask word per thread
static_assert(kBinsPerThread == 32, "one 32-bit mask word per thread");

__global__ void fmask_root_kernel(const int64_t* __restrict__ rfile_off, const int32_t* __restrict__ rfile_f,
                                  int32_t R, unsigned long long* __restrict__ mask) {
  for (int64_t c = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; c < R; c += int64_t(gridDim.x) * blockDim.x) {
    unsigned long long m = 0;
    for (int64_t e = rfile_off[c]; e < rfile_off[c + 1]; ++e) m |= 1ull << rfile_f[e];
    mask[c] = m;
  }
}

// OR of the parents' masks for the children on one level (edges grouped by
// child; the root's own mask is 0, its references came from fmask_root).
__global__ void fmask_edges_kernel(const int32_t* __restrict__ lchild, const int32_t* __restrict__ lpar, int64_t a,
                                   int64_t b, unsigned long long* __restrict__ mask) {
  const int lane = threadIdx.x & 31;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t i = a + blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i - lane < b; i += stride) {
    const bool in = i < b;
    const int32_t c = in ? lchild[i] : -1;
    unsigned long long v = in ? mask[lpar[i]] : 0ull;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long u = __shfl_down_sync(0xffffffffu, v, o);
      const int32_t c2 = __shfl_down_sync(0xffffffffu, c, o);
      if (lane + o < 32 && c2 == c) v |= u;
    }
    const int32_t cp = __shfl_up_sync(0xffffffffu, c, 1);
    if (in && (lane == 0 || cp != c) && v) atomicOr(&mask[c], v);
  }
}

__global__ void mask_totals_kernel(const unsigned long long* __restrict__ mask, const int32_t* __restrict__ W,
                                   const int32_t* __restrict__ S, int32_t R, unsigned long long* __restrict__ out) {
  unsigned long long a = 0, x = 0, y = 0;
  for (int64_t r = 1 + blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < R; r += int64_t(gridDim.x) * blockDim.x) {
    const unsigned long long f = __popcll(mask[r]);
    a += f;
    x += f * (unsigned long long)W[r];
    y += f * (unsigned long long)(W[r] + S[r]);
  }
  for (int o = 16; o; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    x += __shfl_xor_sync(0xffffffffu, x, o);
    y += __shfl_xor_sync(0xffffffffu, y, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&out[0], a);
    atomicAdd(&out[1], x);
    atomicAdd(&out[2], y);
  }
}

// Per-file weights are computed level by level from a structure built at
// load: every (rule, file) slot has a row listing, for each non-root parent
// p of the rule that holds the file, p's slot for that file and the edge's
// multiplicity.  A level pass then computes, per slot, its starting value (the
// root's references of that file, copied in) plus the sum of mult times the
// parent slots' weights (parents are on lower levels, so their weights are
// final).  A rule with few parent edges ("light": at most kHeavyParents, the
// root's included) has rows of at most that many entries and gets one thread
// per slot; the rows of a "heavy" rule (a frequent digram used by up to
// thousands of rules) are summed by a warp each.
constexpr int kHeavyParents = 4;

__device__ __forceinline__ bool heavy_rule(const int64_t* __restrict__ pedge_off, int32_t r) {
  return r != 0 && pedge_off[r + 1] - pedge_off[r] > kHeavyParents;
}

// Slot layout: the light rules' slots level by level (rules in level order,
// each rule's files ascending), then the heavy rules' slots, also level by
// level, so that the slots of one class and level are contiguous.  cnt[k] =
// slots of the k-th rule in level order of the selected class.
__global__ void level_popc_kernel(const int32_t* __restrict__ lvl_order, const unsigned long long* __restrict__ mask,
                                  const int64_t* __restrict__ pedge_off, int32_t R, int64_t* __restrict__ cnt_light,
                                  int64_t* __restrict__ cnt_heavy) {
  for (int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; k < R; k += int64_t(gridDim.x) * blockDim.x) {
    const int32_t r = lvl_order[k];
    const int64_t n = r == 0 ? 0 : __popcll(mask[r]);
    const bool h = heavy_rule(pedge_off, r);
    cnt_light[k] = h ? 0 : n;
    cnt_heavy[k] = h ? n : 0;
  }
}

// off[r] from the scans (heavy slots after all light ones) and the owner
// (rule, file) of every slot.
__global__ void slot_owner_kernel(const int32_t* __restrict__ lvl_order, const int64_t* __restrict__ scan_light,
                                  const int64_t* __restrict__ scan_heavy, const int64_t* __restrict__ n_light,
                                  const unsigned long long* __restrict__ mask, const int64_t* __restrict__ pedge_off,
                                  int32_t R, int64_t* __restrict__ off, int32_t* __restrict__ slot_rule,
                                  uint8_t* __restrict__ slot_file) {
  const int64_t nl = *n_light;
  for (int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; k < R; k += int64_t(gridDim.x) * blockDim.x) {
    const int32_t r = lvl_order[k];
    int64_t o = heavy_rule(pedge_off, r) ? nl + scan_heavy[k] : scan_light[k];
    off[r] = o;
    unsigned long long m = r == 0 ? 0ull : mask[r];
    while (m) {
      const int f = __ffsll(m) - 1;
      m &= m - 1;
      slot_rule[o] = r;
      slot_file[o] = uint8_t(f);
      ++o;
    }
  }
}

// Per level l: first light slot lvl_slot[l] = scan_light[lvl_off[l]] and
// first heavy slot lvl_heavy[l] = n_light + scan_heavy[lvl_off[l]]; index
// depth holds the ends.
__global__ void level_slot_off_kernel(const int64_t* __restrict__ lvl_off, int32_t depth,
                                      const int64_t* __restrict__ scan_light, const int64_t* __restrict__ scan_heavy,
                                      const int64_t* __restrict__ n, int32_t R, int64_t* __restrict__ lvl_slot,
                                      int64_t* __restrict__ lvl_heavy) {
  for (int l = threadIdx.x; l <= depth; l += blockDim.x) {
    lvl_slot[l] = lvl_off[l] < R ? scan_light[lvl_off[l]] : n[0];
    lvl_heavy[l] = n[0] + (lvl_off[l] < R ? scan_heavy[lvl_off[l]] : n[1]);
  }
}

// Rows, edge-parallel over the non-root parent edges p -> c: every file f
// of p gets an entry (p's slot for f, mult) in the row of c's slot for f.
// With fill == false only the row lengths are counted; with fill == true the
// entries are placed (their order inside a row is whatever the atomics give:
// the row is a sum of integers).
template <bool kFill>
__global__ void slot_rows_kernel(const int32_t* __restrict__ lchild, const int32_t* __restrict__ lpar,
                                 const uint32_t* __restrict__ lmult, int64_t E, const int64_t* __restrict__ off,
                                 const unsigned long long* __restrict__ mask, uint32_t* __restrict__ cnt,
                                 const int64_t* __restrict__ row_off, uint2* __restrict__ entries) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < E; e += int64_t(gridDim.x) * blockDim.x) {
    const int32_t p = lpar[e];
    if (p == 0) continue;  // the root's references are the starting values
    const int32_t c = lchild[e];
    const unsigned long long cm = mask[c];
    unsigned long long pm = mask[p];
    const int64_t po = off[p], co = off[c];
    for (int k = 0; pm; ++k) {
      const int f = __ffsll(pm) - 1;
      pm &= pm - 1;
      const int64_t slot = co + __popcll(cm & ((1ull << f) - 1ull));
      const uint32_t at = atomicAdd(&cnt[slot], 1u);
      if (kFill) entries[row_off[slot] + at] = make_uint2(uint32_t(po + k), lmult[e]);
    }
  }
}

__global__ void widen_u32_kernel(const uint32_t* __restrict__ x, int64_t n, int64_t* __restrict__ y) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    y[i] = x[i];
}

__global__ void narrow_off_kernel(const int64_t* __restrict__ x, int64_t n, uint32_t* __restrict__ y) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i <= n; i += int64_t(gridDim.x) * blockDim.x)
    y[i] = uint32_t(x[i]);
}


struct WeightRows {
  const uint32_t* row_off;    // [slots + 1]
  const uint2* entries;       // (parent's pair, mult)
  const uint4* pieces;        // heavy rows cut into pieces: (pair, first entry, end entry, 0)
  const uint32_t* slot_pair;  // [slots]: the pair of each slot (weights are kept by pair)
};

// Heavy rows are cut into pieces of at most kPieceEntries entries, one warp
// each, so that a rule with thousands of parents does not set the length of
// its level's pass; the pieces of a slot add their sums atomically.
constexpr uint32_t kPieceEntries = 128;

// At load: pieces of the heavy slots [h0, h1) (counted with fill == false).
template <bool kFill>
__global__ void row_pieces_kernel(const uint32_t* __restrict__ row_off, int64_t h0, int64_t h1,
                                  int64_t* __restrict__ cnt, const int64_t* __restrict__ pscan,
                                  uint4* __restrict__ pieces) {
  for (int64_t i = h0 + blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < h1; i += int64_t(gridDim.x) * blockDim.x) {
    const uint32_t r0 = row_off[i], r1 = row_off[i + 1];
    const int64_t np = (int64_t(r1 - r0) + kPieceEntries - 1) / kPieceEntries;
    if (!kFill) {
      cnt[i - h0] = np;
      continue;
    }
    int64_t o = pscan[i - h0];
    for (uint32_t e = r0; e < r1; e += kPieceEntries, ++o)
      pieces[o] = make_uint4(uint32_t(i), e, min(e + kPieceEntries, r1), 0u);
  }
}

// At load: the root's references in the slot layout, w0[slot (c, f)] = how
// often the root of file f references rule c (0 if it does not): the
// starting value of every per-file weight.
__global__ void root_slots_kernel(const int64_t* __restrict__ rfile_off, const int32_t* __restrict__ rfile_f,
                                  const uint32_t* __restrict__ rfile_m, int32_t R, const int64_t* __restrict__ off,
                                  const unsigned long long* __restrict__ mask, uint32_t* __restrict__ w0) {
  for (int64_t c = 1 + blockIdx.x * int64_t(blockDim.x) + threadIdx.x; c < R; c += int64_t(gridDim.x) * blockDim.x) {
    const unsigned long long cm = mask[c];
    const int64_t o = off[c];
    for (int64_t e = rfile_off[c]; e < rfile_off[c + 1]; ++e)
      w0[o + __popcll(cm & ((1ull << rfile_f[e]) - 1ull))] = rfile_m[e];
  }
}

// At load, once the pairs are in file-major order: every slot's pair (the
// weights of a query live in pair order, so that the rule-word entries of a
// chunk, which come from a run of consecutive pairs, gather them from a
// small window), the root's references in pair order, and the rows' and
// pieces' slots replaced by their pairs.
__global__ void slot_pair_kernel(const uint32_t* __restrict__ pair_slot, int64_t n, uint32_t* __restrict__ slot_pair) {
  for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < n; q += int64_t(gridDim.x) * blockDim.x)
    slot_pair[pair_slot[q]] = uint32_t(q);
}

__global__ void pair_gather_kernel(const uint32_t* __restrict__ by_slot, const uint32_t* __restrict__ pair_slot,
                                   int64_t n, uint32_t* __restrict__ by_pair) {
  for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < n; q += int64_t(gridDim.x) * blockDim.x)
    by_pair[q] = by_slot[pair_slot[q]];
}

__global__ void rows_to_pairs_kernel(uint2* __restrict__ entries, int64_t ne, uint4* __restrict__ pieces, int64_t np,
                                     const uint32_t* __restrict__ slot_pair) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < ne + np; i += int64_t(gridDim.x) * blockDim.x) {
    if (i < ne) entries[i].x = slot_pair[entries[i].x];
    else pieces[i - ne].x = slot_pair[pieces[i - ne].x];
  }
}

// One level: blocks [0, light_blocks) take the light slots [a, b), one
// thread per slot (rows of at most kHeavyParents entries, all loads issued
// together); the other blocks take the pieces [ha, hb) of the heavy slots'
// rows, one warp per piece.  Every slot already holds the root's references
// of its file.
__global__ void __launch_bounds__(256) fweight_level_kernel(WeightRows L, int64_t a, int64_t b, int light_blocks,
                                                            int64_t ha, int64_t hb, uint32_t* __restrict__ w) {
  if (int(blockIdx.x) < light_blocks) {
    for (int64_t i = a + blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < b;
         i += int64_t(light_blocks) * blockDim.x) {
      const uint32_t r0 = L.row_off[i], n = L.row_off[i + 1] - r0;  // <= kHeavyParents
      if (n == 0) continue;
      uint2 en[kHeavyParents];
#pragma unroll
      for (int k = 0; k < kHeavyParents; ++k) en[k] = k < int(n) ? L.entries[r0 + k] : make_uint2(0u, 0u);
      uint32_t x[kHeavyParents];
#pragma unroll
      for (int k = 0; k < kHeavyParents; ++k) x[k] = k < int(n) ? w[en[k].x] : 0u;
      const uint32_t q = L.slot_pair[i];
      uint32_t v = w[q];
#pragma unroll
      for (int k = 0; k < kHeavyParents; ++k) v += en[k].y * x[k];
      w[q] = v;
    }
    return;
  }
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = int64_t(int(gridDim.x) - light_blocks) * (blockDim.x >> 5);
  for (int64_t q = ha + (int64_t(int(blockIdx.x) - light_blocks) * blockDim.x + threadIdx.x) / 32; q < hb;
       q += nwarps) {
    const uint4 pc = L.pieces[q];
    uint32_t v = 0;
    for (uint32_t e0 = pc.y; e0 < pc.z; e0 += 4 * 32) {  // four entries per lane in flight
      uint2 en[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const uint32_t e = e0 + u * 32 + lane;
        en[u] = e < pc.z ? L.entries[e] : make_uint2(0u, 0u);
      }
      uint32_t x[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) x[u] = en[u].y ? w[en[u].x] : 0u;
#pragma unroll
      for (int u = 0; u < 4; ++u) v += en[u].y * x[u];
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0 && v) atomicAdd(&w[pc.x], v);
  }
}

// (file << 32 | rule) keys of every (rule, file) slot, rule-major.
// Pairs of rules without words of their own get file F: sorted after every
// file's pairs, they stay out of the rule-word chunks.
__global__ void fentry_keys_kernel(const unsigned long long* __restrict__ mask, const int64_t* __restrict__ off,
                                   const int32_t* __restrict__ W, int32_t R, int32_t F, uint64_t* __restrict__ keys) {
  for (int64_t r = 1 + blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < R; r += int64_t(gridDim.x) * blockDim.x) {
    unsigned long long m = mask[r];
    int64_t o = off[r];
    const bool none = W[r] == 0;
    while (m) {
      const int f = __ffsll(m) - 1;
      m &= m - 1;
      keys[o++] = (uint64_t(none ? F : f) << 32) | uint64_t(r);
    }
  }
}

// The rules' own words, rule after rule (the root's excluded): rule r's are
// rule_words[woff[r], woff[r] + W_r).  They are at most N < 2^32.
__global__ void rule_words_kernel(DevGrammar d, const int64_t* __restrict__ woff64, uint32_t* __restrict__ woff,
                                  int32_t* __restrict__ rule_words) {
  for (int64_t r = 1 + blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < d.R; r += int64_t(gridDim.x) * blockDim.x) {
    int64_t o = woff64[r];
    woff[r] = uint32_t(o);
    for (int64_t j = d.rule_off[r]; j < d.rule_off[r + 1]; ++j) {
      const int32_t sy = d.sym[j];
      if (sy < d.V) rule_words[o++] = sy;
    }
  }
}

__global__ void rule_word_counts_kernel(const int32_t* __restrict__ W, int32_t R, int64_t* __restrict__ cnt) {
  for (int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < R; r += int64_t(gridDim.x) * blockDim.x)
    cnt[r] = r == 0 ? 0 : W[r];
}

__global__ void entry_words_kernel(const uint64_t* __restrict__ keys, int64_t n, const int32_t* __restrict__ W,
                                   int32_t F, int64_t* __restrict__ cnt) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    cnt[i] = int32_t(keys[i] >> 32) < F ? W[uint32_t(keys[i])] : 0;
}

__global__ void iota_u32_kernel(uint32_t* __restrict__ x, int64_t n) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    x[i] = uint32_t(i);
}

// xoff[f] = position of file f's first emitted word.
__global__ void file_starts_kernel(const int64_t* __restrict__ fstart, const int64_t* __restrict__ pos,
                                   const int64_t* __restrict__ wcnt, int64_t n, int32_t F, int64_t* __restrict__ xoff) {
  for (int32_t f = blockIdx.x * blockDim.x + threadIdx.x; f <= F; f += gridDim.x * blockDim.x) {
    const int64_t i = fstart[f];
    xoff[f] = i < n ? pos[i] : (n > 0 ? pos[n - 1] + wcnt[n - 1] : 0);
  }
}

struct TvSlots {
  int32_t* word;   // [F * nb * kFBucket]
  uint32_t* cnt;   // same
  int64_t* nnz;    // [F * nb]
  uint32_t* bits;  // [F * nb * kTvThreads]: bit l of word t = word (bucket base + 32 t + l) occurs
};

constexpr int kChunk = 4096;  // rule words per chunk of the weighted sort
// root chunks (kFileChunk symbols) are sorted by 1024-thread CTAs, rule-word
// chunks (kChunk words) by 512-thread CTAs: 8 items per thread either way
template <bool kWeighted>
struct ChunkShape {
  static constexpr int kItemsPerChunk = kWeighted ? kChunk : kFileChunk;
  static constexpr int kThreads = kWeighted ? 512 : 1024;
  static constexpr int kPer = kItemsPerChunk / kThreads;
  static constexpr int kWarps = kThreads / 32;
  static_assert(kPer * kThreads == kItemsPerChunk, "whole items per thread");
};
constexpr int kMaxNb = 128;

// A stream of (file-ordered) word items cut into chunks that never cross a
// file: chunk c covers items [start[c], start[c] + len[c]) of file file_of(c);
// the chunks of file f are [foff[f], foff[f+1]).  For the rule words, chunk c
// also names the (file, rule) pairs whose words overlap it: [p0[c], p1[c]).
struct Chunks {
  const int64_t* start;
  const int32_t* len;
  const int64_t* foff;
  const int64_t* count;  // device: number of chunks
  const int64_t* p0 = nullptr;
  const int64_t* p1 = nullptr;
};

// Where the rule words of a chunk come from: the (file, rule) pairs in
// file-major order (rule in the key's low half), the weight slot of each pair,
// the position of its first word, the per-file weights, and the rules' own
// words (rule r's at rule_words[woff[r]], W_r of them).
struct PairWords {
  const uint32_t* wbeg;   // [pairs]: the pair's rule's first own word in rule_words
  const uint32_t* slot;   // [pairs]: the pair's weight slot
  const uint32_t* pos;    // [pairs + 1]: first word of each pair in the file-major stream (< N < 2^32)
  const uint32_t* w;      // per-file weights (slot layout)
  const int32_t* rule_words;
};

// Counting sort of one chunk by word bucket, in shared memory, written back
// to the chunk's own item range (one entry per word, so it always fits):
// root words become their 14-bit index (uint16), rule words (index | weight
// << 16) as uint64.  runs[c * nb + b] = (start, length) of bucket b's entries.
// Root chunks read their words from the root body.  A rule-word chunk first
// expands the (file, rule) pairs that overlap it into shared memory: each
// pair writes its rule's own words (a contiguous run of the words-only rule
// array) with the pair's weight at their positions in the chunk; pairs are
// contiguous in the word stream, so a pair's words end where the next pair's
// begin.
template <bool kWeighted>
__global__ void __launch_bounds__(ChunkShape<kWeighted>::kThreads, kWeighted ? 3 : 2) chunk_sort_kernel(
    Chunks ch, const int32_t* __restrict__ items, PairWords pw, int nb, int32_t V, void* __restrict__ out,
    int64_t* __restrict__ run_start, int32_t* __restrict__ run_len) {
  constexpr int kCsThreads = ChunkShape<kWeighted>::kThreads;
  constexpr int kCsWarps = ChunkShape<kWeighted>::kWarps;
  constexpr int kItems = ChunkShape<kWeighted>::kItemsPerChunk;
  constexpr int kPer = ChunkShape<kWeighted>::kPer;
  __shared__ uint32_t wcnt[kCsWarps][kMaxNb + 1];
  __shared__ uint32_t bstart[kMaxNb + 1];
  // rule chunks: the expanded (word, weight) items, then the sorted entries
  __shared__ __align__(16) unsigned char stage_raw[size_t(kItems) * (kWeighted ? 8 : 2)];
  int32_t* const ex_word = reinterpret_cast<int32_t*>(stage_raw);
  uint32_t* const ex_wt = reinterpret_cast<uint32_t*>(stage_raw) + kItems;
  const int64_t nch = *ch.count;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int64_t c = blockIdx.x; c < nch; c += gridDim.x) {
    for (int i = tid; i < kCsWarps * (kMaxNb + 1); i += kCsThreads) (&wcnt[0][0])[i] = 0;
    const int64_t base = ch.start[c];
    const int n = ch.len[c];
    if (kWeighted) {
      const int64_t q0 = ch.p0[c], q1 = ch.p1[c];
      // two pairs per thread at a time: every load of a level is issued
      // before the next level's (slot -> weight)
      for (int64_t k0 = q0; k0 < q1; k0 += 2 * kCsThreads) {
        uint32_t wb[2], sl[2], wv[2];
        int64_t a[2], b[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int64_t q = k0 + u * kCsThreads + tid;
          const bool in = q < q1;
          wb[u] = in ? pw.wbeg[q] : 0u;
          sl[u] = in ? pw.slot[q] : 0u;
          a[u] = in ? int64_t(pw.pos[q]) - base : 0;
          b[u] = in ? int64_t(pw.pos[q + 1]) - base : 0;
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) wv[u] = a[u] < b[u] ? pw.w[sl[u]] : 0u;
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int64_t j0 = a[u] > 0 ? a[u] : 0, j1 = b[u] < n ? b[u] : n;  // clipped to the chunk
          for (int64_t j = j0; j < j1; ++j) {
            ex_word[j] = pw.rule_words[wb[u] + uint32_t(j - a[u])];
            ex_wt[j] = wv[u];
          }
        }
      }
    }
    __syncthreads();
    // item j of this thread: word (21 bits, V <= 2^21) | rank inside its
    // (warp, bucket) << 21 (a warp holds 256 items, so the rank takes 8
    // bits); kNone for no item or a rule reference
    constexpr uint32_t kNone = 0xffffffffu;
    static_assert(32 * kPer <= 256, "rank fits 8 bits");
    uint32_t it[kPer];
    uint32_t wt[kWeighted ? kPer : 1];
    if (kWeighted) {
#pragma unroll
      for (int j = 0; j < kPer; ++j) {
        const int i = j * kCsThreads + tid;  // warp-contiguous: item order inside a warp is lane order
        const int32_t x = i < n ? ex_word[i] : -1;
        wt[j] = i < n ? ex_wt[i] : 0u;
        it[j] = uint32_t(x) < uint32_t(V) ? uint32_t(x) : kNone;
      }
    } else {
      // the chunk's 16-byte-aligned window (from at most 3 symbols before the
      // chunk), read as int4: only vectors that start inside the window, so
      // the last read ends at most 3 symbols past the chunk (the array is
      // padded by 4); symbols outside the chunk are dropped
      const int64_t a0 = base & ~int64_t(3);
      const int lead = int(base - a0);
      static_assert(kPer % 4 == 0, "whole vectors per thread");
#pragma unroll
      for (int j = 0; j < kPer / 4; ++j) {
        const int v = j * kCsThreads + tid;
        const int4 q = 4 * v < lead + n ? *reinterpret_cast<const int4*>(items + a0 + 4 * int64_t(v))
                                        : make_int4(-1, -1, -1, -1);
        const int32_t xs[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = 4 * v + u - lead;  // position in the chunk
          const int32_t x = (i >= 0 && i < n) ? xs[u] : -1;
          it[4 * j + u] = uint32_t(x) < uint32_t(V) ? uint32_t(x) : kNone;
        }
      }
    }
    // rank inside (warp, bucket) by an atomic on the warp's own counter: the
    // histograms that read the runs do not depend on the order inside a run
#pragma unroll
    for (int j = 0; j < kPer; ++j)
      if (it[j] != kNone) it[j] |= atomicAdd(&wcnt[warp][it[j] >> kFBLog2], 1u) << 21;
    __syncthreads();  // also: the expanded items are in registers, the stage may be overwritten
    // exclusive prefix over (bucket, warp): warp b0.. scans bucket b over the warps
    for (int b = warp; b < nb; b += kCsWarps) {
      const uint32_t x = lane < kCsWarps ? wcnt[lane][b] : 0u;
      uint32_t incl = x;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
      }
      if (lane < kCsWarps) wcnt[lane][b] = incl - x;
      if (lane == 31) bstart[b] = incl;  // bucket total, turned into a start below
    }
    __syncthreads();
    if (warp == 0) {
      uint32_t run = 0;
      for (int b0 = 0; b0 < nb; b0 += 32) {
        const int b = b0 + lane;
        const uint32_t x = b < nb ? bstart[b] : 0u;
        uint32_t incl = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += u;
        }
        if (b < nb) {
          bstart[b] = run + incl - x;
          // rule chunks are written back to their own item range, root
          // chunks to slot c of kFileChunk entries (16-byte aligned)
          run_start[c * nb + b] = (kWeighted ? base : c * int64_t(kFileChunk)) + run + incl - x;
          run_len[c * nb + b] = int32_t(x);
        }
        run += __shfl_sync(0xffffffffu, incl, 31);
      }
      if (lane == 0) bstart[kMaxNb] = run;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      if (it[j] == kNone) continue;
      const uint32_t word = it[j] & ((1u << 21) - 1u);
      const int b = int(word >> kFBLog2);
      const uint32_t pos = bstart[b] + wcnt[warp][b] + (it[j] >> 21);
      const uint32_t local = word & (kFBucket - 1);
      if (kWeighted)
        reinterpret_cast<uint64_t*>(stage_raw)[pos] = (uint64_t(wt[j]) << 16) | local;
      else
        reinterpret_cast<uint16_t*>(stage_raw)[pos] = uint16_t(local);
    }
    __syncthreads();
    const uint32_t total = bstart[kMaxNb];
    if (kWeighted) {
      uint64_t* o = static_cast<uint64_t*>(out) + base;
      for (uint32_t i = tid; i < total; i += kCsThreads) o[i] = reinterpret_cast<uint64_t*>(stage_raw)[i];
    } else {
      static_assert(kItems == 8 * kCsThreads, "one 16-byte store per thread");
      int4* o = reinterpret_cast<int4*>(static_cast<uint16_t*>(out) + c * int64_t(kFileChunk));
      if (8 * uint32_t(tid) < total) o[tid] = reinterpret_cast<const int4*>(stage_raw)[tid];
    }
    __syncthreads();
  }
}

template <bool kWeighted>
void launch_chunk_sort(unsigned grid, cudaStream_t s, const Chunks& ch, const int32_t* items, const PairWords& pw,
                       int nb, int32_t V, void* out, int64_t* run_start, int32_t* run_len) {
  if (nb > kMaxNb) fail(GT_EOVERFLOW, "more than 128 word buckets");
  chunk_sort_kernel<kWeighted><<<grid, ChunkShape<kWeighted>::kThreads, 0, s>>>(ch, items, pw, nb, V, out,
                                                                               run_start, run_len);
  GT_LAUNCH_CHECK();
}

// Chunk table of the emitted rule words: file f's words [xoff[f], xoff[f+1]).
// One block; thread f cuts file f (F <= 64 on this path).
__global__ void rule_chunks_kernel(const int64_t* __restrict__ xoff, int32_t F, int64_t* __restrict__ start,
                                   int32_t* __restrict__ len, int64_t* __restrict__ foff, int64_t* __restrict__ count) {
  __shared__ int64_t nch[65];
  const int f = threadIdx.x;
  if (f < F) nch[f] = (xoff[f + 1] - xoff[f] + kChunk - 1) / kChunk;
  __syncthreads();
  if (f == 0) {
    int64_t c = 0;
    for (int32_t i = 0; i < F; ++i) {
      const int64_t n = nch[i];
      nch[i] = c;
      c += n;
    }
    nch[F] = c;
    *count = c;
  }
  __syncthreads();
  if (f <= F) foff[f] = nch[f];
  if (f < F) {
    int64_t c = nch[f];
    for (int64_t p = xoff[f]; p < xoff[f + 1]; p += kChunk, ++c) {
      start[c] = p;
      len[c] = int32_t(min(int64_t(kChunk), xoff[f + 1] - p));
    }
  }
}

// The pairs whose words overlap each rule-word chunk: p0 = the pair holding
// the chunk's first word (the last pair starting at or before it; pairs
// without words start where the next one does, so it is never one of them),
// p1 = the first pair starting at or after the chunk's end.
__global__ void chunk_pairs_kernel(const int64_t* __restrict__ start, const int32_t* __restrict__ len,
                                   const int64_t* __restrict__ count, const int64_t* __restrict__ pos, int64_t n,
                                   int64_t* __restrict__ p0, int64_t* __restrict__ p1) {
  const int64_t nch = *count;
  for (int64_t c = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; c < nch; c += int64_t(gridDim.x) * blockDim.x) {
    const int64_t s0 = start[c], s1 = s0 + len[c];
    int64_t lo = 0, hi = n;  // first i with pos[i] > s0
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (pos[mid] <= s0) lo = mid + 1;
      else hi = mid;
    }
    p0[c] = lo - 1;
    lo = 0, hi = n;  // first i with pos[i] >= s1
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (pos[mid] < s1) lo = mid + 1;
      else hi = mid;
    }
    p1[c] = lo;
  }
}

// At load: the rule-word entries of each chunk narrowed to 32 bits, the
// pair made relative to the chunk's first pair (a chunk holds at most
// kChunk + 1 pairs, every one with a word) above the 14-bit index.
constexpr int kRelShift = 14;
__global__ void narrow_entries_kernel(const uint64_t* __restrict__ wide, const int64_t* __restrict__ start,
                                      const int32_t* __restrict__ len, const int64_t* __restrict__ count,
                                      const int64_t* __restrict__ p0, uint32_t* __restrict__ out) {
  const int64_t nch = *count;
  for (int64_t c = blockIdx.x; c < nch; c += gridDim.x) {
    const int64_t b = start[c], q0 = p0[c];
    for (int i = threadIdx.x; i < len[c]; i += blockDim.x) {
      const uint64_t e = wide[b + i];
      out[b + i] = (uint32_t(int64_t(e >> 16) - q0) << kRelShift) | uint32_t(e & (kFBucket - 1));
    }
  }
}

// Per pair, what the rule-word chunks read: the first own word of its rule
// and its first word in the stream as uint32 (both below N < 2^32).
__global__ void pair_records_kernel(const uint64_t* __restrict__ keys, const int64_t* __restrict__ pos, int64_t n,
                                    const uint32_t* __restrict__ woff, uint32_t* __restrict__ wbeg,
                                    uint32_t* __restrict__ pos32) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i <= n; i += int64_t(gridDim.x) * blockDim.x) {
    pos32[i] = uint32_t(pos[i]);
    if (i < n) wbeg[i] = woff[uint32_t(keys[i])];
  }
}

// CTA (f, b): dense histogram of file f's words in bucket b, from the bucket-b
// runs of f's root chunks and rule-word chunks.  Run descriptors are staged
// in shared memory a batch at a time, so each warp's next run starts without
// a dependent global load.
constexpr int kTvBatch = kTvThreads;

// Root entries (uint16) add 1; rule-word entries (uint32) carry their
// (file, rule) pair, relative to their chunk's first pair p0, above the
// 14-bit index, and add that pair's weight: the entries of a run come from
// one chunk, a run of consecutive pairs, so the gathers fall in a small
// window of the weights.
template <bool kRule>
__device__ __forceinline__ void tv_runs(uint32_t* hist, int64_t c0, int64_t c1, int nb, int b,
                                        const int64_t* __restrict__ rs, const int32_t* __restrict__ rl,
                                        const void* __restrict__ entv, const int64_t* __restrict__ p0,
                                        const uint32_t* __restrict__ wts, int64_t* s_start, int32_t* s_len,
                                        uint32_t* s_p0) {
  using E = typename std::conditional<kRule, uint32_t, uint16_t>::type;
  const E* __restrict__ ent = static_cast<const E*>(entv);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int64_t cb = c0; cb < c1; cb += kTvBatch) {
    const int nbatch = int(min(int64_t(kTvBatch), c1 - cb));
    __syncthreads();  // previous batch consumed
    if (tid < nbatch) {
      s_start[tid] = rs[(cb + tid) * nb + b];
      s_len[tid] = rl[(cb + tid) * nb + b];
      if (kRule) s_p0[tid] = uint32_t(p0[cb + tid]);  // pairs < 2^32 (checked at load)
    }
    __syncthreads();
    for (int q = warp; q < nbatch; q += kTvThreads / 32) {
      const int64_t s0 = s_start[q];
      const int32_t n = s_len[q];
      const uint32_t* wq = kRule ? wts + s_p0[q] : nullptr;
      // 4 independent loads per lane in flight, then their weights
      for (int i0 = 0; i0 < n; i0 += 128) {
        uint32_t e[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int i = i0 + k * 32 + lane;
          e[k] = i < n ? uint32_t(ent[s0 + i]) : 0u;
        }
        uint32_t x[4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
          x[k] = !kRule ? 1u : (i0 + k * 32 + lane < n ? __ldg(wq + (e[k] >> 14)) : 0u);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          if (i0 + k * 32 + lane >= n) break;
          atomicAdd(&hist[e[k] & (kFBucket - 1)], x[k]);
        }
      }
    }
  }
}

__global__ void __launch_bounds__(kTvThreads) tv_hist_kernel(int32_t F, int nb, Chunks rc, const int64_t* __restrict__ rrs,
                                                             const int32_t* __restrict__ rrl,
                                                             const uint16_t* __restrict__ rent, Chunks xc,
                                                             const int64_t* __restrict__ xrs,
                                                             const int32_t* __restrict__ xrl,
                                                             const uint32_t* __restrict__ xent,
                                                             const uint32_t* __restrict__ xw,
                                                             const int32_t* __restrict__ order, TvSlots out) {
  __shared__ uint32_t hist[kFBucket];
  __shared__ int64_t warp_tot[kTvThreads / 32 + 1];
  __shared__ int64_t s_start[kTvBatch];
  __shared__ int32_t s_len[kTvBatch];
  __shared__ uint32_t s_p0[kTvBatch];
  // pieces of the longest files first (order: files by length, descending)
  const int f = order[blockIdx.x / nb], b = blockIdx.x % nb;
  const int64_t piece = int64_t(f) * nb + b;
  const int tid = threadIdx.x;
  for (int i = tid; i < kFBucket; i += kTvThreads) hist[i] = 0;
  tv_runs<false>(hist, rc.foff[f], rc.foff[f + 1], nb, b, rrs, rrl, rent, nullptr, nullptr, s_start, s_len, s_p0);
  tv_runs<true>(hist, xc.foff[f], xc.foff[f + 1], nb, b, xrs, xrl, xent, xc.p0, xw, s_start, s_len, s_p0);
  __syncthreads();
  // compaction in word order: warp w owns bins [1024 w, 1024 w + 1024), read
  // 32 consecutive bins per round (no bank conflicts); the round masks are the
  // inverted index's occupancy bits
  constexpr int kBinsPerWarp = kFBucket / (kTvThreads / 32);
  constexpr int kRounds = kBinsPerWarp / 32;
  static_assert(kRounds == 32, "one round mask per lane");
  const int lane = tid & 31, warp = tid >> 5;
  uint32_t my_mask = 0;  // lane r keeps the mask of round r
  int wcount = 0;
#pragma unroll 8
  for (int r = 0; r < kRounds; ++r) {
    const uint32_t m = __ballot_sync(0xffffffffu, hist[warp * kBinsPerWarp + r * 32 + lane] != 0u);
    if (lane == r) my_mask = m;
    wcount += __popc(m);
  }
  out.bits[piece * kTvThreads + warp * 32 + lane] = my_mask;
  if (lane == 0) warp_tot[warp] = wcount;
  __syncthreads();
  if (warp == 0) {
    const int64_t wv = lane < kTvThreads / 32 ? warp_tot[lane] : 0;
    int64_t wi = wv;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t u = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += u;
    }
    if (lane < kTvThreads / 32) warp_tot[lane] = wi - wv;
    if (lane == kTvThreads / 32 - 1) warp_tot[kTvThreads / 32] = wi;
  }
  __syncthreads();
  const int64_t slot = piece * kFBucket;
  const int32_t wbase = b << kFBLog2;
  int64_t o = slot + warp_tot[warp];
  const uint32_t below = (1u << lane) - 1u;
#pragma unroll 4
  for (int r = 0; r < kRounds; ++r) {
    const uint32_t m = __shfl_sync(0xffffffffu, my_mask, r);
    const int bin = warp * kBinsPerWarp + r * 32 + lane;
    if ((m >> lane) & 1u) {
      const int64_t p = o + __popc(m & below);
      out.word[p] = wbase + bin;
      out.cnt[p] = hist[bin];
    }
    o += __popc(m);
  }
  if (tid == 0) out.nnz[piece] = warp_tot[kTvThreads / 32];
}

// Copy every (file, bucket) piece to its place in the term vector.
// Copy every (file, bucket) piece to its place in the term vector; with wc
// (zeroed), each entry's count is also added to its word's count (the word
// count as the sum of the files' counts, one 32-bit reduction per entry:
// counts stay below N < 2^32 on this path).
__global__ void tv_gather_kernel(TvSlots in, const int64_t* __restrict__ off, int32_t* __restrict__ word,
                                 uint64_t* __restrict__ cnt, unsigned* __restrict__ wc) {
  const int64_t slot = int64_t(blockIdx.x) * kFBucket;
  const int64_t n = in.nnz[blockIdx.x], o = off[blockIdx.x];
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const int32_t w = in.word[slot + i];
    const uint32_t c = in.cnt[slot + i];
    word[o + i] = w;
    cnt[o + i] = c;
    if (wc) atomicAdd(&wc[w], c);
  }
}

__global__ void tv_file_off_kernel(const int64_t* __restrict__ off, int nb, int32_t F,
                                   const int64_t* __restrict__ total, int64_t* __restrict__ tv_off) {
  for (int32_t f = blockIdx.x * blockDim.x + threadIdx.x; f <= F; f += gridDim.x * blockDim.x)
    tv_off[f] = f < F ? off[int64_t(f) * nb] : *total;
}

// Inverted index: files holding each word (bit set in that file's piece).
// A warp takes 32 consecutive words - one 32-bit occupancy word per file -
// lane f loads file f's (and file f + 32's) word, and one ballot per bit
// position gives each word's set of files.
__device__ __forceinline__ void ii_masks(const uint32_t* __restrict__ bits, int nb, int32_t F, int64_t w0, int lane,
                                         uint32_t& m_lo, uint32_t& m_hi) {
  const int64_t b = w0 >> kFBLog2, t = (w0 & (kFBucket - 1)) >> 5;
  m_lo = lane < F ? bits[(int64_t(lane) * nb + b) * kTvThreads + t] : 0u;
  m_hi = lane + 32 < F ? bits[(int64_t(lane + 32) * nb + b) * kTvThreads + t] : 0u;
}

__global__ void ii_count_kernel(const uint32_t* __restrict__ bits, int nb, int32_t F, int32_t V,
                                int64_t* __restrict__ cnt) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t w0 = ((blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5) * 32; w0 < V; w0 += nwarps * 32) {
    uint32_t lo, hi;
    ii_masks(bits, nb, F, w0, lane, lo, hi);
    int mine = 0;
#pragma unroll
    for (int l = 0; l < 32; ++l) {
      const int c = __popc(__ballot_sync(0xffffffffu, (lo >> l) & 1u)) + __popc(__ballot_sync(0xffffffffu, (hi >> l) & 1u));
      if (lane == l) mine = c;
    }
    if (w0 + lane < V) cnt[w0 + lane] = mine;
  }
}

__global__ void ii_fill_kernel(const uint32_t* __restrict__ bits, int nb, int32_t F, int32_t V,
                               const int64_t* __restrict__ off, int32_t* __restrict__ files) {
  const int lane = threadIdx.x & 31;
  const unsigned below = (1u << lane) - 1u;
  const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t w0 = ((blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5) * 32; w0 < V; w0 += nwarps * 32) {
    uint32_t lo, hi;
    ii_masks(bits, nb, F, w0, lane, lo, hi);
    const int64_t my_off = w0 + lane < V ? off[w0 + lane] : 0;
    for (int l = 0; l < 32 && w0 + l < V; ++l) {
      const unsigned a = __ballot_sync(0xffffffffu, (lo >> l) & 1u);
      const unsigned c = __ballot_sync(0xffffffffu, (hi >> l) & 1u);
      const int64_t o = __shfl_sync(0xffffffffu, my_off, l);
      if ((a >> lane) & 1u) files[o + __popc(a & below)] = lane;
      if ((c >> lane) & 1u) files[o + __popc(a) + __popc(c & below)] = lane + 32;
    }
  }
}

// The inverted index in one pass: CTAs take blocks of kIiWords words in
// ticket order; each counts the files of its words (one ballot per bit, as
// above), scans the counts, gets the block's first posting by a bounded
// decoupled look-back over the preceding blocks, writes the words' offsets
// and fills their postings.
constexpr int kIiThreads = 256;
constexpr int kIiWords = kIiThreads;  // a warp per 32 words

__global__ void __launch_bounds__(kIiThreads) ii_build_kernel(const uint32_t* __restrict__ bits, int nb, int32_t F,
                                                              int32_t V, unsigned long long* __restrict__ flags,
                                                              unsigned long long* __restrict__ ticket,
                                                              int64_t* __restrict__ off, int32_t* __restrict__ files,
                                                              unsigned* __restrict__ status) {
  __shared__ int64_t s_item, s_prefix;
  __shared__ int s_wsum[kIiThreads / 32 + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_item = int64_t(atomicAdd(ticket, 1ull));
  __syncthreads();
  const int64_t item = s_item;
  const int64_t w0 = item * kIiWords + warp * 32;
  uint32_t lo = 0, hi = 0;
  if (w0 < V) ii_masks(bits, nb, F, w0, lane, lo, hi);
  int mine = 0;
#pragma unroll
  for (int l = 0; l < 32; ++l) {
    const int c = __popc(__ballot_sync(0xffffffffu, (lo >> l) & 1u)) + __popc(__ballot_sync(0xffffffffu, (hi >> l) & 1u));
    if (lane == l) mine = c;
  }
  if (w0 + lane >= V) mine = 0;
  // exclusive prefix of the counts over the block
  int incl = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int u = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += u;
  }
  if (lane == 31) s_wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const int x = lane < kIiThreads / 32 ? s_wsum[lane] : 0;
    int wi = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += u;
    }
    if (lane < kIiThreads / 32) s_wsum[lane] = wi - x;
    if (lane == kIiThreads / 32 - 1) s_wsum[kIiThreads / 32] = wi;
    const uint64_t total = uint64_t(__shfl_sync(0xffffffffu, wi, kIiThreads / 32 - 1));
    if (lane == 0) publish_aggregate(flags, item, total);
    __syncwarp();
    const int64_t p = warp_look_back(flags, item, total, status);
    if (lane == 0) s_prefix = p < 0 ? 0 : p;
  }
  __syncthreads();
  const int64_t my_off = s_prefix + s_wsum[warp] + incl - mine;
  if (w0 + lane < V) off[w0 + lane] = my_off;
  if (w0 + lane == V - 1) off[V] = my_off + mine;
  const unsigned below = (1u << lane) - 1u;
  for (int l = 0; l < 32 && w0 + l < V; ++l) {
    const unsigned a = __ballot_sync(0xffffffffu, (lo >> l) & 1u);
    const unsigned c = __ballot_sync(0xffffffffu, (hi >> l) & 1u);
    const int64_t o = __shfl_sync(0xffffffffu, my_off, l);
    if ((a >> lane) & 1u) files[o + __popc(a & below)] = lane;
    if ((c >> lane) & 1u) files[o + __popc(a) + __popc(c & below)] = lane + 32;
  }
}

__global__ void last_total_kernel(const int64_t* __restrict__ ex, const int64_t* __restrict__ cnt, int64_t n,
                                  int64_t* __restrict__ out, int64_t* __restrict__ out2) {
  const int64_t t = n > 0 ? ex[n - 1] + cnt[n - 1] : 0;
  *out = t;
  if (out2) *out2 = t;
}

// top-k: key = file << 32 | (2^32 - 1 - count), sorted stably over entries that
// are already in ascending word order inside each file.
__global__ void topk_keys_kernel(const int32_t* __restrict__ word, const uint64_t* __restrict__ cnt,
                                 const int64_t* __restrict__ tv_off, int32_t F, int64_t bound,
                                 uint64_t* __restrict__ keys, uint32_t* __restrict__ idx) {
  const int64_t n = tv_off[F];
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < bound; i += int64_t(gridDim.x) * blockDim.x) {
    idx[i] = uint32_t(i);
    if (i >= n) {
      keys[i] = uint64_t(uint32_t(F)) << 32;  // padding sorts last
      continue;
    }
    int32_t lo = 0, hi = F;  // file of entry i: last f with tv_off[f] <= i
    while (hi - lo > 1) {
      const int32_t mid = (lo + hi) >> 1;
      if (tv_off[mid] <= i) lo = mid;
      else hi = mid;
    }
    keys[i] = (uint64_t(lo) << 32) | uint64_t(0xffffffffu - uint32_t(cnt[i]));
  }
}

__global__ void topk_count_kernel(const int64_t* __restrict__ tv_off, int32_t F, int k, int64_t* __restrict__ cnt) {
  for (int32_t f = blockIdx.x * blockDim.x + threadIdx.x; f < F; f += gridDim.x * blockDim.x)
    cnt[f] = min(int64_t(k), tv_off[f + 1] - tv_off[f]);
}

__global__ void topk_gather_kernel(const uint32_t* __restrict__ idx, const int64_t* __restrict__ tv_off,
                                   const int64_t* __restrict__ k_off, int32_t F, const int32_t* __restrict__ word,
                                   const uint64_t* __restrict__ cnt, int32_t* __restrict__ kw,
                                   uint64_t* __restrict__ kc) {
  for (int32_t f = blockIdx.x; f < F; f += gridDim.x) {
    const int64_t n = k_off[f + 1] - k_off[f];
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
      const uint32_t j = idx[tv_off[f] + i];
      kw[k_off[f] + i] = word[j];
      kc[k_off[f] + i] = cnt[j];
    }
  }
}

struct FileHist {
  Buf slot_word, slot_cnt, nnz, bits, off, total;
  int nb = 0;
  int64_t bound = 0;  // bound on term-vector entries (= inverted-index postings)
};

int bits_for(int64_t x) {
  int b = 1;
  while ((int64_t(1) << b) <= x) ++b;
  return b;
}

// Steps 1-5: the dense (file, bucket) pieces, their sizes and the II bits.
// Nothing here waits for the GPU: buffers are sized by bounds computed when
// the grammar was loaded, and sorts run over padded, bound-sized arrays.
}  // namespace

// At load: the file masks once, to size every per-file buffer exactly (pairs,
// their words, their body symbols), and the structure the per-file weights
// and the rule-word chunks are computed over.  Grammars with more than 64
// files keep 0.
void file_sizes(gt_grammar* g, cudaStream_t s) {
  gt_ctx* ctx = g->ctx;
  const DevGrammar& d = g->d;
  g->fentry_bound = g->fword_bound = g->fsym_bound = 0;
  if (d.F > 64) return;
  const int threads = 256, cap = ctx->num_sms * 16;
  // structure used only while the layout is built (released on return)
  Buf owners, w0b, pairs, words, recs;
  const int32_t* rule_words = nullptr;
  const uint32_t* fe_wbeg = nullptr;
  const uint32_t* fe_pos32 = nullptr;
  // persistent: masks, slot offsets and the pair count (freed with the grammar)
  void* p = grammar_alloc(g, size_t(d.R) * 16 + 16, s);
  auto* M = static_cast<unsigned long long*>(p);
  auto* off = reinterpret_cast<int64_t*>(M + d.R);
  auto* nnz = off + d.R;
  Buf tot(ctx, 32, s), sc(ctx, scan_scratch_bytes(d.R), s), ntot(ctx, 32, s);
  Buf cl(ctx, size_t(d.R) * 8, s), ch(ctx, size_t(d.R) * 8, s);
  Buf sl(ctx, size_t(d.R) * 8, s), sh(ctx, size_t(d.R) * 8, s);
  fmask_root_kernel<<<grid_for(d.R, threads, cap), threads, 0, s>>>(d.rfile_off, d.rfile_f, d.R, M);
  GT_LAUNCH_CHECK();
  for (int lv = 2; lv < d.depth; ++lv) {
    const int64_t a = g->ledge_off[lv], b = g->ledge_off[lv + 1];
    if (b > a) {
      fmask_edges_kernel<<<grid_for(b - a, threads, cap), threads, 0, s>>>(d.ledge_child, d.ledge_par, a, b, M);
      GT_LAUNCH_CHECK();
    }
  }
  // slots level by level, light rules first: popcounts in level order, scanned
  auto* nl = ntot.as<int64_t>();  // [0] light slots, [1] heavy slots
  level_popc_kernel<<<grid_for(d.R, threads, cap), threads, 0, s>>>(d.lvl_order, M, d.pedge_off, d.R,
                                                                     cl.as<int64_t>(), ch.as<int64_t>());
  GT_LAUNCH_CHECK();
  exclusive_scan_i64(cl.as<int64_t>(), sl.as<int64_t>(), d.R, sc.p, s);
  last_total_kernel<<<1, 1, 0, s>>>(sl.as<int64_t>(), cl.as<int64_t>(), d.R, nl, nullptr);
  GT_LAUNCH_CHECK();
  exclusive_scan_i64(ch.as<int64_t>(), sh.as<int64_t>(), d.R, sc.p, s);
  last_total_kernel<<<1, 1, 0, s>>>(sh.as<int64_t>(), ch.as<int64_t>(), d.R, nl + 1, nullptr);
  GT_LAUNCH_CHECK();
  GT_CUDA(cudaMemsetAsync(tot.p, 0, 32, s));
  mask_totals_kernel<<<grid_for(d.R, threads, cap), threads, 0, s>>>(M, d.nwords, d.nrefs, d.R,
                                                                      tot.as<unsigned long long>());
  GT_LAUNCH_CHECK();
  unsigned long long h[3];
  int64_t hn[2];
  GT_CUDA(cudaMemcpyAsync(h, tot.p, 24, cudaMemcpyDeviceToHost, s));
  GT_CUDA(cudaMemcpyAsync(hn, nl, 16, cudaMemcpyDeviceToHost, s));
  GT_CUDA(cudaStreamSynchronize(s));
  g->fentry_bound = int64_t(h[0]);
  g->fword_bound = int64_t(h[1]);
  g->fsym_bound = int64_t(h[2]);
  const int64_t EB = g->fentry_bound;
  if (hn[0] + hn[1] != EB) fail(GT_EINVAL, "per-file slot count mismatch");
  if (EB >= (int64_t(1) << 32)) fail(GT_EOVERFLOW, "2^32 or more (rule, file) pairs");
  g->light_slots = hn[0];
  GT_CUDA(cudaMemcpyAsync(nnz, &EB, 8, cudaMemcpyHostToDevice, s));
  // owners of the slots and each level's first light and heavy slot
  void* po = grammar_alloc(g, size_t(2 * (d.depth + 1)) * 8 + 64, s);
  auto* lslot = static_cast<int64_t*>(po);
  auto* lheavy = lslot + d.depth + 1;
  owners = Buf(ctx, size_t(EB) * 5 + 64, s);
  auto* srule = owners.as<int32_t>();
  auto* sfile = reinterpret_cast<uint8_t*>(srule + EB);
  slot_owner_kernel<<<grid_for(d.R, threads, cap), threads, 0, s>>>(d.lvl_order, sl.as<int64_t>(), sh.as<int64_t>(),
                                                                     nl, M, d.pedge_off, d.R, off, srule, sfile);
  GT_LAUNCH_CHECK();
  {
    Buf loff(ctx, size_t(d.depth + 1) * 8, s);
    GT_CUDA(cudaMemcpyAsync(loff.p, g->lvl_off.data(), size_t(d.depth + 1) * 8, cudaMemcpyHostToDevice, s));
    level_slot_off_kernel<<<1, 128, 0, s>>>(loff.as<int64_t>(), d.depth, sl.as<int64_t>(), sh.as<int64_t>(), nl, d.R,
                                            lslot, lheavy);
    GT_LAUNCH_CHECK();
    g->lvl_slot.assign(size_t(d.depth + 1), 0);
    g->lvl_heavy.assign(size_t(d.depth + 1), 0);
    GT_CUDA(cudaMemcpyAsync(g->lvl_slot.data(), lslot, size_t(d.depth + 1) * 8, cudaMemcpyDeviceToHost, s));
    GT_CUDA(cudaMemcpyAsync(g->lvl_heavy.data(), lheavy, size_t(d.depth + 1) * 8, cudaMemcpyDeviceToHost, s));
    GT_CUDA(cudaStreamSynchronize(s));  // loff, EB and lvl_off's host copy are read by now
  }
  // the root's references in slot layout (every weight's starting value)
  {
    w0b = Buf(ctx, size_t(EB) * 4 + 16, s);
    auto* w0 = w0b.as<uint32_t>();
    if (EB > 0) GT_CUDA(cudaMemsetAsync(w0, 0, size_t(EB) * 4, s));
    root_slots_kernel<<<grid_for(d.R, threads, cap), threads, 0, s>>>(d.rfile_off, d.rfile_f, d.rfile_m, d.R, off, M,
                                                                       w0);
    GT_LAUNCH_CHECK();
  }
  // every slot's row of (parent slot, mult): counted, scanned, filled
  {
    Buf rc(ctx, size_t(EB) * 4 + 16, s), rc64(ctx, size_t(EB) * 8 + 16, s), ro64(ctx, size_t(EB + 1) * 8, s);
    Buf sc5(ctx, scan_scratch_bytes(EB), s);
    if (EB > 0) GT_CUDA(cudaMemsetAsync(rc.p, 0, size_t(EB) * 4, s));
    slot_rows_kernel<false><<<grid_for(d.E, threads, cap), threads, 0, s>>>(
        d.ledge_child, d.ledge_par, d.ledge_mult, d.E, off, M, rc.as<uint32_t>(), nullptr, nullptr);
    GT_LAUNCH_CHECK();
    widen_u32_kernel<<<grid_for(EB, threads, cap), threads, 0, s>>>(rc.as<uint32_t>(), EB, rc64.as<int64_t>());
    GT_LAUNCH_CHECK();
    exclusive_scan_i64(rc64.as<int64_t>(), ro64.as<int64_t>(), EB, sc5.p, s);
    last_total_kernel<<<1, 1, 0, s>>>(ro64.as<int64_t>(), rc64.as<int64_t>(), EB, ro64.as<int64_t>() + EB, nullptr);
    GT_LAUNCH_CHECK();
    int64_t nent = 0;
    GT_CUDA(cudaMemcpyAsync(&nent, ro64.as<int64_t>() + EB, 8, cudaMemcpyDeviceToHost, s));
    GT_CUDA(cudaStreamSynchronize(s));
    if (nent >= (int64_t(1) << 32)) fail(GT_EOVERFLOW, "per-file weight rows hold 2^32 entries or more");
    void* pr = grammar_alloc(g, size_t(EB + 1) * 4 + 16 + size_t(nent) * 8 + 16, s);
    auto* roff = static_cast<uint32_t*>(pr);
    auto* ent = reinterpret_cast<uint2*>(roff + ((EB + 1 + 3) / 4) * 4);
    narrow_off_kernel<<<grid_for(EB + 1, threads, cap), threads, 0, s>>>(ro64.as<int64_t>(), EB, roff);
    GT_LAUNCH_CHECK();
    if (EB > 0) GT_CUDA(cudaMemsetAsync(rc.p, 0, size_t(EB) * 4, s));
    slot_rows_kernel<true><<<grid_for(d.E, threads, cap), threads, 0, s>>>(
        d.ledge_child, d.ledge_par, d.ledge_mult, d.E, off, M, rc.as<uint32_t>(), ro64.as<int64_t>(), ent);
    GT_LAUNCH_CHECK();
    g->row_off = roff;
    g->row_entries = ent;
    g->row_entries_n = nent;
    // the heavy slots' rows in pieces, and each level's first piece
    const int64_t NL = hn[0], NH = EB - NL;
    Buf pc(ctx, size_t(NH) * 8 + 16, s), ps(ctx, size_t(NH + 1) * 8, s), sc6(ctx, scan_scratch_bytes(NH), s);
    int64_t npieces = 0;
    if (NH > 0) {
      row_pieces_kernel<false><<<grid_for(NH, threads, cap), threads, 0, s>>>(roff, NL, EB, pc.as<int64_t>(),
                                                                               nullptr, nullptr);
      GT_LAUNCH_CHECK();
      exclusive_scan_i64(pc.as<int64_t>(), ps.as<int64_t>(), NH, sc6.p, s);
      last_total_kernel<<<1, 1, 0, s>>>(ps.as<int64_t>(), pc.as<int64_t>(), NH, ps.as<int64_t>() + NH, nullptr);
      GT_LAUNCH_CHECK();
      GT_CUDA(cudaMemcpyAsync(&npieces, ps.as<int64_t>() + NH, 8, cudaMemcpyDeviceToHost, s));
      GT_CUDA(cudaStreamSynchronize(s));
    }
    auto* pieces = static_cast<uint4*>(grammar_alloc(g, size_t(npieces) * 16 + 16, s));
    if (npieces > 0) {
      row_pieces_kernel<true><<<grid_for(NH, threads, cap), threads, 0, s>>>(roff, NL, EB, nullptr,
                                                                              ps.as<int64_t>(), pieces);
      GT_LAUNCH_CHECK();
    }
    g->row_pieces = pieces;
    g->row_pieces_n = npieces;
    g->lvl_piece.assign(size_t(d.depth + 1), 0);
    for (int l = 0; l <= d.depth; ++l) {
      const int64_t h = g->lvl_heavy[size_t(l)] - NL;  // heavy slots before level l
      if (NH > 0) GT_CUDA(cudaMemcpyAsync(&g->lvl_piece[size_t(l)], ps.as<int64_t>() + h, 8, cudaMemcpyDeviceToHost, s));
    }
    GT_CUDA(cudaStreamSynchronize(s));  // the scratch above is released on return
  }
  g->fmask = M;
  g->foff = off;
  g->fnnz = nnz;
  // the pairs in file-major order with their word offsets
  const size_t qbytes = size_t(EB) * 8 + size_t(EB) * 4 + size_t(EB + 1) * 8 + size_t(d.F + 1) * 8 + 64;
  pairs = Buf(ctx, qbytes, s);
  auto* fkeys = pairs.as<uint64_t>();
  auto* fslot = reinterpret_cast<uint32_t*>(fkeys + EB);
  auto* fpos = reinterpret_cast<int64_t*>(reinterpret_cast<char*>(fslot) + (size_t(EB) * 4 + 15) / 16 * 16);
  auto* fxoff = fpos + EB + 1;
  Buf keys(ctx, size_t(EB) * 8, s), slot0(ctx, size_t(EB) * 4, s), rs(ctx, radix_scratch_bytes(EB, true, 4), s);
  Buf wcnt(ctx, size_t(EB) * 8, s), sc2(ctx, scan_scratch_bytes(EB), s), fstart(ctx, size_t(d.F + 1) * 8, s);
  if (EB > 0) {
    fentry_keys_kernel<<<grid_for(d.R, threads, cap), threads, 0, s>>>(M, off, d.nwords, d.R, d.F,
                                                                        keys.as<uint64_t>());
    GT_LAUNCH_CHECK();
    iota_u32_kernel<<<grid_for(EB, threads, cap), threads, 0, s>>>(slot0.as<uint32_t>(), EB);
    GT_LAUNCH_CHECK();
    radix_sort_u64(keys.as<uint64_t>(), fkeys, slot0.p, fslot, 4, EB, 32, 32 + bits_for(d.F), rs.p, s);
    entry_words_kernel<<<grid_for(EB, threads, cap), threads, 0, s>>>(fkeys, EB, d.nwords, d.F, wcnt.as<int64_t>());
    GT_LAUNCH_CHECK();
    exclusive_scan_i64(wcnt.as<int64_t>(), fpos, EB, sc2.p, s);
    last_total_kernel<<<1, 1, 0, s>>>(fpos, wcnt.as<int64_t>(), EB, fpos + EB, nullptr);
    GT_LAUNCH_CHECK();
  } else {
    GT_CUDA(cudaMemsetAsync(fpos, 0, 8, s));
  }
  csr_offsets_hi(fkeys, EB, d.F, fstart.as<int64_t>(), s);
  file_starts_kernel<<<1, 128, 0, s>>>(fstart.as<int64_t>(), fpos, wcnt.as<int64_t>(), EB, d.F, fxoff);
  GT_LAUNCH_CHECK();
  // weights by pair: each slot's pair, the root's references by pair, and the
  // rows and pieces re-addressed to pairs
  {
    auto* sp = static_cast<uint32_t*>(grammar_alloc(g, size_t(EB) * 8 + 32, s));
    auto* r0 = sp + EB + 4;
    if (EB > 0) {
      slot_pair_kernel<<<grid_for(EB, threads, cap), threads, 0, s>>>(fslot, EB, sp);
      GT_LAUNCH_CHECK();
      pair_gather_kernel<<<grid_for(EB, threads, cap), threads, 0, s>>>(w0b.as<uint32_t>(), fslot, EB, r0);
      GT_LAUNCH_CHECK();
    }
    const int64_t ne = g->row_entries_n, np = g->row_pieces_n;
    if (ne + np > 0) {
      rows_to_pairs_kernel<<<grid_for(ne + np, threads, cap), threads, 0, s>>>(
          const_cast<uint2*>(g->row_entries), ne, const_cast<uint4*>(g->row_pieces), np, sp);
      GT_LAUNCH_CHECK();
    }
    g->slot_pair = sp;
    g->root_pairs = r0;
  }
  // the rule words cut into chunks of at most kChunk words inside each file,
  // with the pairs that overlap each chunk
  const int64_t nxc = g->fword_bound / kChunk + d.F + 1;  // bound on the chunks
  void* pc = grammar_alloc(g, size_t(nxc) * 28 + size_t(d.F + 1) * 8 + 64, s);
  auto* xcs = static_cast<int64_t*>(pc);
  auto* xp0 = xcs + nxc;
  auto* xp1 = xp0 + nxc;
  auto* xcf = xp1 + nxc;
  auto* xcn = xcf + d.F + 1;
  auto* xcl = reinterpret_cast<int32_t*>(xcn + 1);
  rule_chunks_kernel<<<1, 128, 0, s>>>(fxoff, d.F, xcs, xcl, xcf, xcn);
  GT_LAUNCH_CHECK();
  chunk_pairs_kernel<<<grid_for(nxc, threads, cap), threads, 0, s>>>(xcs, xcl, xcn, fpos, EB, xp0, xp1);
  GT_LAUNCH_CHECK();
  GT_CUDA(cudaMemcpyAsync(&g->rule_chunks, xcn, 8, cudaMemcpyDeviceToHost, s));
  // the rules' own words, for the chunks' expansion
  {
    Buf wc(ctx, size_t(d.R) * 8, s), wo(ctx, size_t(d.R) * 8 + 8, s), sc4(ctx, scan_scratch_bytes(d.R), s);
    rule_word_counts_kernel<<<grid_for(d.R, threads, cap), threads, 0, s>>>(d.nwords, d.R, wc.as<int64_t>());
    GT_LAUNCH_CHECK();
    exclusive_scan_i64(wc.as<int64_t>(), wo.as<int64_t>(), d.R, sc4.p, s);
    last_total_kernel<<<1, 1, 0, s>>>(wo.as<int64_t>(), wc.as<int64_t>(), d.R, wo.as<int64_t>() + d.R, nullptr);
    GT_LAUNCH_CHECK();
    int64_t nw = 0;
    GT_CUDA(cudaMemcpyAsync(&nw, wo.as<int64_t>() + d.R, 8, cudaMemcpyDeviceToHost, s));
    GT_CUDA(cudaStreamSynchronize(s));
    words = Buf(ctx, size_t(d.R) * 4 + size_t(nw) * 4 + 64, s);
    auto* woff = words.as<uint32_t>();
    auto* rw = reinterpret_cast<int32_t*>(woff + d.R + (d.R & 3 ? 4 - (d.R & 3) : 0));
    rule_words_kernel<<<grid_for(d.R, threads, cap), threads, 0, s>>>(d, wo.as<int64_t>(), woff, rw);
    GT_LAUNCH_CHECK();
    recs = Buf(ctx, size_t(EB) * 8 + 16, s);
    auto* rec = recs.as<uint32_t>();
    pair_records_kernel<<<grid_for(EB + 1, threads, cap), threads, 0, s>>>(fkeys, fpos, EB, woff, rec, rec + EB);
    GT_LAUNCH_CHECK();
    rule_words = rw;
    fe_wbeg = rec;
    fe_pos32 = rec + EB;
    GT_CUDA(cudaStreamSynchronize(s));  // the scratch above is released on return
  }
  g->xch_start = xcs;
  g->xch_len = xcl;
  g->xch_foff = xcf;
  g->xch_count = xcn;
  g->xch_p0 = xp0;
  g->xch_p1 = xp1;
  GT_CUDA(cudaStreamSynchronize(s));
  // the rule words of every file sorted by 16k-word bucket, each entry its
  // (file, rule) pair relative to the chunk's first pair above its 14-bit
  // index, in 32 bits (structure: a query gathers its weights by pair)
  {
    const int nb = int((d.V + kFBucket - 1) / kFBucket);
    const int64_t nxc2 = g->rule_chunks;
    void* px = grammar_alloc(g, size_t(g->fword_bound) * 4 + 16 + size_t(nxc2) * nb * 12 + 64, s);
    auto* xrs = static_cast<int64_t*>(px);
    auto* xrl = reinterpret_cast<int32_t*>(xrs + nxc2 * nb);
    auto* xent = reinterpret_cast<uint32_t*>(xrl + nxc2 * nb + 4);
    if (nxc2 > 0) {
      Buf ident(ctx, size_t(EB) * 4 + 16, s), wide(ctx, size_t(g->fword_bound) * 8 + 16, s);
      iota_u32_kernel<<<grid_for(EB, threads, cap), threads, 0, s>>>(ident.as<uint32_t>(), EB);
      GT_LAUNCH_CHECK();
      Chunks xc{xcs, xcl, xcf, xcn, xp0, xp1};
      // "weight" of pair q = ident[ident[q]] = q: every entry carries its pair
      const PairWords pw{fe_wbeg, ident.as<uint32_t>(), fe_pos32, ident.as<uint32_t>(), rule_words};
      launch_chunk_sort<true>(unsigned(std::min<int64_t>(nxc2, 65535)), s, xc, nullptr, pw, nb, d.V, wide.p, xrs,
                              xrl);
      narrow_entries_kernel<<<unsigned(std::min<int64_t>(nxc2, 65535)), 256, 0, s>>>(
          wide.as<uint64_t>(), xcs, xcl, xcn, xp0, xent);
      GT_LAUNCH_CHECK();
      GT_CUDA(cudaStreamSynchronize(s));  // ident and wide are released on return
    }
    g->xent = xent;
    g->xrun_start = xrs;
    g->xrun_len = xrl;
  }
  // files by length, longest first (launch order of per-file work)
  std::vector<uint64_t> hl(size_t(d.F));
  if (d.F > 0) {
    GT_CUDA(cudaMemcpyAsync(hl.data(), d.file_len, size_t(d.F) * 8, cudaMemcpyDeviceToHost, s));
    GT_CUDA(cudaStreamSynchronize(s));
  }
  std::vector<int32_t> ord(size_t(d.F));
  for (int32_t f = 0; f < d.F; ++f) ord[size_t(f)] = f;
  std::stable_sort(ord.begin(), ord.end(), [&](int32_t a, int32_t b) { return hl[size_t(a)] > hl[size_t(b)]; });
  void* pf = grammar_alloc(g, size_t(d.F) * 4 + 16, s);
  if (d.F > 0) GT_CUDA(cudaMemcpyAsync(pf, ord.data(), size_t(d.F) * 4, cudaMemcpyHostToDevice, s));
  GT_CUDA(cudaStreamSynchronize(s));  // ord is a host temporary
  g->file_order = static_cast<const int32_t*>(pf);
}

void file_weights(gt_grammar* g, cudaStream_t s, FileWeights& fw) {
  gt_ctx* ctx = g->ctx;
  const DevGrammar& d = g->d;
  const int threads = 256, cap = ctx->num_sms * 16;
  const int32_t F = d.F, V = d.V;
  if (F > 64) fail(GT_EOVERFLOW, "the top-down per-file strategy holds at most 64 files (file_strategy 0 or 2 selects bottom-up)");
  if (d.N >= (uint64_t(1) << 32)) fail(GT_EOVERFLOW, "per-file analytics need fewer than 2^32 tokens per grammar");
  if (V > (1 << 21)) fail(GT_EOVERFLOW, "per-file analytics support num_words <= 2^21");
  if (!g->fmask) fail(GT_EINVAL, "per-file layout missing");
  const int64_t EB = g->fentry_bound;
  fw.mask = g->fmask;
  fw.off = g->foff;
  fw.nnz = g->fnnz;
  fw.w = Buf(ctx, size_t(EB) * 4, s);
  fw.slot_pair = g->slot_pair;
  // every weight starts as the root's references of its file (weights by pair)
  if (EB > 0) GT_CUDA(cudaMemcpyAsync(fw.w.p, g->root_pairs, size_t(EB) * 4, cudaMemcpyDeviceToDevice, s));
  const WeightRows L{g->row_off, g->row_entries, g->row_pieces, g->slot_pair};
  // level by level from the root's children down; level-1 rules have no
  // parent but the root, so their weights are complete already
  for (int lv = 2; lv < d.depth; ++lv) {
    const int64_t a = g->lvl_slot[size_t(lv)], b = g->lvl_slot[size_t(lv) + 1];
    const int64_t ha = g->lvl_piece[size_t(lv)], hb = g->lvl_piece[size_t(lv) + 1];
    if (b <= a && hb <= ha) continue;
    const int lb = b > a ? int(grid_for(b - a, threads, cap)) : 0;
    const int hblk = hb > ha ? int(grid_for((hb - ha) * 32, threads, cap)) : 0;  // a warp per heavy piece
    fweight_level_kernel<<<unsigned(lb + hblk), threads, 0, s>>>(L, a, b, lb, ha, hb, fw.w.as<uint32_t>());
    GT_LAUNCH_CHECK();
  }
}

namespace {

void file_hist(gt_grammar* g, cudaStream_t s, FileHist& fh) {
  gt_ctx* ctx = g->ctx;
  const DevGrammar& d = g->d;
  const int32_t F = d.F, V = d.V;
  FileWeights fwt;
  {
    Phase ph(ctx, "file_weights", s);
    file_weights(g, s, fwt);
  }
  // ---- bucket-sorted chunks, then dense (file, bucket) histograms ----
  const int nb = int((V + kFBucket - 1) / kFBucket);
  const int64_t pieces = int64_t(F) * nb;
  fh.nb = nb;
  fh.bound = std::min<int64_t>(int64_t(d.N), pieces * kFBucket);
  fh.slot_word = Buf(ctx, size_t(pieces) * kFBucket * 4, s);
  fh.slot_cnt = Buf(ctx, size_t(pieces) * kFBucket * 4, s);
  fh.nnz = Buf(ctx, size_t(pieces) * 8, s);
  fh.bits = Buf(ctx, size_t(pieces) * kTvThreads * 4, s);
  fh.off = Buf(ctx, size_t(pieces) * 8, s);
  fh.total = Buf(ctx, 8, s);
  TvSlots ts{fh.slot_word.as<int32_t>(), fh.slot_cnt.as<uint32_t>(), fh.nnz.as<int64_t>(), fh.bits.as<uint32_t>()};
  {
    Phase ph2(ctx, "tv_hist", s);
    const int64_t nrc = g->root_chunks;
    Chunks rc{d.rch_start, d.rch_len, d.rch_foff, d.rch_count};
    Chunks xc{g->xch_start, g->xch_len, g->xch_foff, g->xch_count, g->xch_p0, g->xch_p1};
    const PairWords pw{};  // unused by the root chunks
    Buf rent(ctx, size_t(nrc) * kFileChunk * 2 + 16, s), rrs(ctx, size_t(nrc) * nb * 8, s),
        rrl(ctx, size_t(nrc) * nb * 4, s);
    if (nrc > 0) {
      Phase ph4(ctx, "chunk_sort_root", s);
      launch_chunk_sort<false>(unsigned(std::min<int64_t>(nrc, 65535)), s, rc, d.sym, pw, nb, V, rent.p,
                               rrs.as<int64_t>(), rrl.as<int32_t>());
    }
    // the rule words: bucket-sorted at load, weighted here by their pairs
    Phase ph3(ctx, "tv_hist_kernel", s);
    tv_hist_kernel<<<unsigned(pieces), kTvThreads, 0, s>>>(F, nb, rc, rrs.as<int64_t>(), rrl.as<int32_t>(),
                                                           rent.as<uint16_t>(), xc, g->xrun_start, g->xrun_len,
                                                           g->xent, fwt.w.as<uint32_t>(), g->file_order, ts);
    GT_LAUNCH_CHECK();
  }
  Buf sc3(ctx, scan_scratch_bytes(pieces), s);
  exclusive_scan_i64(fh.nnz.as<int64_t>(), fh.off.as<int64_t>(), pieces, sc3.p, s);
  last_total_kernel<<<1, 1, 0, s>>>(fh.off.as<int64_t>(), fh.nnz.as<int64_t>(), pieces, fh.total.as<int64_t>(),
                                    nullptr);
  GT_LAUNCH_CHECK();
}

// With wc (top_k == 0 only), the word counts are written too: the sum over
// files of the term vectors' counts, added while the pieces are copied.
gt_result* term_vector_from(gt_grammar* g, FileHist& fh, int top_k, cudaStream_t s, uint64_t* wc = nullptr) {
  gt_ctx* ctx = g->ctx;
  const DevGrammar& d = g->d;
  const int64_t pieces = int64_t(d.F) * fh.nb;
  const int64_t nb_ = fh.bound;
  TvSlots ts{fh.slot_word.as<int32_t>(), fh.slot_cnt.as<uint32_t>(), fh.nnz.as<int64_t>(), fh.bits.as<uint32_t>()};
  if (top_k != 0) {  // top-k selection or TF-IDF: from the gathered arrays
    Buf tw(ctx, size_t(nb_) * 4, s), tc(ctx, size_t(nb_) * 8, s), full_off(ctx, size_t(d.F + 1) * 8, s);
    {
      Phase ph(ctx, "tv_out", s);
      tv_gather_kernel<<<unsigned(pieces), 256, 0, s>>>(ts, fh.off.as<int64_t>(), tw.as<int32_t>(),
                                                        tc.as<uint64_t>(), nullptr);
      GT_LAUNCH_CHECK();
      tv_file_off_kernel<<<1, 256, 0, s>>>(fh.off.as<int64_t>(), fh.nb, d.F, fh.total.as<int64_t>(),
                                           full_off.as<int64_t>());
      GT_LAUNCH_CHECK();
    }
    return tv_from_arrays(ctx, tw.as<int32_t>(), tc.as<uint64_t>(), full_off.as<int64_t>(), fh.total.as<int64_t>(),
                          nb_, d.F, top_k, s, d.V);
  }
  ResultBuilder rb(ctx, s);
  Phase ph(ctx, "tv_out", s);
  auto* tv_off = static_cast<int64_t*>(rb.alloc(size_t(d.F + 1) * 8));
  auto* word = static_cast<int32_t*>(rb.alloc(size_t(nb_) * 4));
  auto* cnt = static_cast<uint64_t*>(rb.alloc(size_t(nb_) * 8));
  int64_t* len = rb.new_len_slot();
  Buf wc32(ctx, wc ? size_t(d.V) * 4 + 16 : 16, s);
  if (wc) GT_CUDA(cudaMemsetAsync(wc32.p, 0, size_t(d.V) * 4, s));
  tv_gather_kernel<<<unsigned(pieces), 256, 0, s>>>(ts, fh.off.as<int64_t>(), word, cnt,
                                                    wc ? wc32.as<unsigned>() : nullptr);
  GT_LAUNCH_CHECK();
  if (wc) {
    widen_u32_kernel<<<grid_for(d.V, 256, ctx->num_sms * 8), 256, 0, s>>>(wc32.as<uint32_t>(), d.V,
                                                                          reinterpret_cast<int64_t*>(wc));
    GT_LAUNCH_CHECK();
  }
  tv_file_off_kernel<<<1, 256, 0, s>>>(fh.off.as<int64_t>(), fh.nb, d.F, fh.total.as<int64_t>(), tv_off);
  GT_LAUNCH_CHECK();
  GT_CUDA(cudaMemcpyAsync(len, fh.total.p, 8, cudaMemcpyDeviceToDevice, s));
  rb.field("offsets", tv_off, int64_t(d.F) + 1);
  rb.field_dyn("word", word, len);
  rb.field_dyn("count", cnt, len);
  return rb.finish();
}

gt_result* inverted_index_from(gt_grammar* g, FileHist& fh, cudaStream_t s) {
  gt_ctx* ctx = g->ctx;
  const DevGrammar& d = g->d;
  ResultBuilder rb(ctx, s);
  Phase ph(ctx, "ii_out", s);
  const int threads = 256, cap = ctx->num_sms * 16;
  const int64_t V = d.V;
  auto* ii_off = static_cast<int64_t*>(rb.alloc(size_t(V + 1) * 8));
  auto* files = static_cast<int32_t*>(rb.alloc(size_t(fh.bound) * 4));
  int64_t* len = rb.new_len_slot();
  if (V == 0) {
    GT_CUDA(cudaMemsetAsync(ii_off, 0, 8, s));
  } else {
    const int64_t blocks = (V + kIiWords - 1) / kIiWords;
    Buf lb(ctx, size_t(blocks + 1) * 8, s);  // look-back words, then the ticket
    GT_CUDA(cudaMemsetAsync(lb.p, 0, size_t(blocks + 1) * 8, s));
    auto* fl = lb.as<unsigned long long>();
    ii_build_kernel<<<unsigned(blocks), kIiThreads, 0, s>>>(fh.bits.as<uint32_t>(), fh.nb, d.F, d.V, fl,
                                                             fl + blocks, ii_off, files, rb.status());
    GT_LAUNCH_CHECK();
  }
  GT_CUDA(cudaMemcpyAsync(len, fh.total.p, 8, cudaMemcpyDeviceToDevice, s));
  rb.field("offsets", ii_off, V + 1);
  rb.field_dyn("file", files, len);
  return rb.finish();
}

__global__ void tv_rows_kernel(const int32_t* __restrict__ word, const int64_t* __restrict__ tv_off, int32_t F,
                               int64_t bound, uint64_t* __restrict__ rkey, int32_t* __restrict__ rfile) {
  const int64_t n = tv_off[F];
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < bound && i < n;
       i += int64_t(gridDim.x) * blockDim.x) {
    int32_t lo = 0, hi = F;  // file of row i: last f with tv_off[f] <= i
    while (hi - lo > 1) {
      const int32_t mid = (lo + hi) >> 1;
      if (tv_off[mid] <= i) lo = mid;
      else hi = mid;
    }
    rkey[i] = uint64_t(uint32_t(word[i]));
    rfile[i] = lo;
  }
}

}  // namespace

gt_result* run_ranked_words(gt_grammar* g, cudaStream_t s) {
  if (file_strategy(g) == 2) return run_ranked_words_bu(g, s);
  gt_ctx* ctx = g->ctx;
  const DevGrammar& d = g->d;
  const int threads = 256, cap = ctx->num_sms * 16;
  FileHist fh;
  file_hist(g, s, fh);
  const int64_t pieces = int64_t(d.F) * fh.nb, bound = fh.bound;
  TvSlots ts{fh.slot_word.as<int32_t>(), fh.slot_cnt.as<uint32_t>(), fh.nnz.as<int64_t>(), fh.bits.as<uint32_t>()};
  Buf tw(ctx, size_t(bound) * 4, s), tc(ctx, size_t(bound) * 8, s), toff(ctx, size_t(d.F + 1) * 8, s);
  Buf rkey(ctx, size_t(bound) * 8, s), rfile(ctx, size_t(bound) * 4, s);
  tv_gather_kernel<<<unsigned(pieces), 256, 0, s>>>(ts, fh.off.as<int64_t>(), tw.as<int32_t>(), tc.as<uint64_t>(),
                                                    nullptr);
  GT_LAUNCH_CHECK();
  tv_file_off_kernel<<<1, 256, 0, s>>>(fh.off.as<int64_t>(), fh.nb, d.F, fh.total.as<int64_t>(), toff.as<int64_t>());
  GT_LAUNCH_CHECK();
  if (bound > 0) {
    tv_rows_kernel<<<grid_for(bound, threads, cap), threads, 0, s>>>(tw.as<int32_t>(), toff.as<int64_t>(), d.F, bound,
                                                                      rkey.as<uint64_t>(), rfile.as<int32_t>());
    GT_LAUNCH_CHECK();
  }
  return ranked_from_rows(ctx, rkey, rfile, tc, fh.total.as<int64_t>(), bound, 0, false, uint64_t(d.V),
                          uint64_t(g->max_file_len), s);
}

__global__ void copy_rows_kernel(const int32_t* __restrict__ w, const uint64_t* __restrict__ c,
                                 const int64_t* __restrict__ n_dev, int32_t* __restrict__ ow,
                                 uint64_t* __restrict__ oc) {
  const int64_t n = *n_dev;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    ow[i] = w[i];
    oc[i] = c[i];
  }
}

// Term-vector result from (word, count) rows in (file, word) order with file
// offsets; top_k > 0 keeps each file's top_k counts (count desc, word asc).
// df[w] += 1 for every term-vector entry of w (the files containing w).
__global__ void df_kernel(const int32_t* __restrict__ word, const int64_t* __restrict__ total,
                          uint32_t* __restrict__ df) {
  const int64_t n = *total;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    atomicAdd(&df[word[i]], 1u);
}

// TF-IDF of every term-vector entry: count * ln(F / df(word)).
__global__ void tfidf_kernel(const int32_t* __restrict__ word, const uint64_t* __restrict__ cnt,
                             const int64_t* __restrict__ total, const uint32_t* __restrict__ df, int32_t F,
                             double* __restrict__ out) {
  const int64_t n = *total;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    out[i] = double(cnt[i]) * log(double(F) / double(df[word[i]]));
}

gt_result* tv_from_arrays(gt_ctx* ctx, const int32_t* word, const uint64_t* cnt, const int64_t* tv_off_in,
                          const int64_t* total, int64_t bound, int32_t F, int top_k, cudaStream_t s,
                          int32_t V) {
  const int threads = 256, cap = ctx->num_sms * 16;
  ResultBuilder rb(ctx, s);
  Phase ph(ctx, "tv_out", s);
  auto* tv_off = static_cast<int64_t*>(rb.alloc(size_t(F + 1) * 8));
  if (top_k <= 0) {
    auto* ow = static_cast<int32_t*>(rb.alloc(size_t(bound) * 4));
    auto* oc = static_cast<uint64_t*>(rb.alloc(size_t(bound) * 8));
    int64_t* len = rb.new_len_slot();
    GT_CUDA(cudaMemcpyAsync(tv_off, tv_off_in, size_t(F + 1) * 8, cudaMemcpyDeviceToDevice, s));
    GT_CUDA(cudaMemcpyAsync(len, total, 8, cudaMemcpyDeviceToDevice, s));
    if (bound > 0) {
      copy_rows_kernel<<<grid_for(bound, threads, cap), threads, 0, s>>>(word, cnt, total, ow, oc);
      GT_LAUNCH_CHECK();
    }
    rb.field("offsets", tv_off, int64_t(F) + 1);
    rb.field_dyn("word", ow, len);
    rb.field_dyn("count", oc, len);
    if (top_k == kTfIdf) {
      if (V <= 0) fail(GT_EINVAL, "TF-IDF needs the vocabulary size");
      auto* tf = static_cast<double*>(rb.alloc(size_t(bound) * 8));
      Buf df(ctx, size_t(V) * 4, s);
      GT_CUDA(cudaMemsetAsync(df.p, 0, size_t(V) * 4, s));
      if (bound > 0) {
        df_kernel<<<grid_for(bound, threads, cap), threads, 0, s>>>(ow, total, df.as<uint32_t>());
        GT_LAUNCH_CHECK();
        tfidf_kernel<<<grid_for(bound, threads, cap), threads, 0, s>>>(ow, oc, total, df.as<uint32_t>(), F, tf);
        GT_LAUNCH_CHECK();
      }
      rb.field_dyn("tfidf", tf, len);
    }
  } else {
    Buf k0(ctx, size_t(bound) * 8, s), k1(ctx, size_t(bound) * 8, s), i0(ctx, size_t(bound) * 4, s);
    Buf i1(ctx, size_t(bound) * 4, s), rs(ctx, radix_scratch_bytes(bound, true, 4), s);
    Buf kc(ctx, size_t(F) * 8 + 8, s), sc(ctx, scan_scratch_bytes(F + 1), s);
    if (bound > 0) {
      topk_keys_kernel<<<grid_for(bound, threads, cap), threads, 0, s>>>(word, cnt, tv_off_in, F, bound,
                                                                          k0.as<uint64_t>(), i0.as<uint32_t>());
      GT_LAUNCH_CHECK();
      radix_sort_u64(k0.as<uint64_t>(), k1.as<uint64_t>(), i0.p, i1.p, 4, bound, 0, 32 + bits_for(F), rs.p, s);
    }
    topk_count_kernel<<<grid_for(F, 256, cap), 256, 0, s>>>(tv_off_in, F, top_k, kc.as<int64_t>());
    GT_LAUNCH_CHECK();
    GT_CUDA(cudaMemsetAsync(kc.as<int64_t>() + F, 0, 8, s));
    exclusive_scan_i64(kc.as<int64_t>(), tv_off, F + 1, sc.p, s);
    const int64_t kb = std::min<int64_t>(int64_t(top_k) * F, bound);
    auto* kw = static_cast<int32_t*>(rb.alloc(size_t(kb) * 4));
    auto* kcnt = static_cast<uint64_t*>(rb.alloc(size_t(kb) * 8));
    int64_t* len = rb.new_len_slot();
    topk_gather_kernel<<<std::max(1, std::min(F, cap)), 256, 0, s>>>(i1.as<uint32_t>(), tv_off_in, tv_off, F, word,
                                                                     cnt, kw, kcnt);
    GT_LAUNCH_CHECK();
    GT_CUDA(cudaMemcpyAsync(len, tv_off + F, 8, cudaMemcpyDeviceToDevice, s));
    rb.field("offsets", tv_off, int64_t(F) + 1);
    rb.field_dyn("word", kw, len);
    rb.field_dyn("count", kcnt, len);
  }
  return rb.finish();
}

namespace {

// Word counts as the sum of the per-file counts (top-down pieces): CTA
// (bucket, file group) adds its files' compacted (word, count) entries of the
// bucket into a dense shared histogram - words are distinct inside a piece,
// so updates rarely collide - and stores it as one partial.
constexpr int kWcFileGroup = 8;

__global__ void __launch_bounds__(kTvThreads) tvwc_hist_kernel(TvSlots ts, int32_t F, int nb, int groups,
                                                               uint32_t* __restrict__ partial) {
  __shared__ uint32_t hist[kFBucket];
  const int b = blockIdx.x / groups, grp = blockIdx.x % groups;
  for (int i = threadIdx.x; i < kFBucket; i += kTvThreads) hist[i] = 0;
  __syncthreads();
  const int f1 = min(F, (grp + 1) * kWcFileGroup);
  for (int f = grp * kWcFileGroup; f < f1; ++f) {
    const int64_t piece = int64_t(f) * nb + b;
    const int64_t n = ts.nnz[piece];
    const int32_t* __restrict__ w = ts.word + piece * kFBucket;
    const uint32_t* __restrict__ c = ts.cnt + piece * kFBucket;
    for (int64_t i = threadIdx.x; i < n; i += kTvThreads) atomicAdd(&hist[w[i] & (kFBucket - 1)], c[i]);
  }
  __syncthreads();
  uint32_t* dst = partial + int64_t(blockIdx.x) * kFBucket;
  for (int i = threadIdx.x; i < kFBucket; i += kTvThreads) dst[i] = hist[i];
}

__global__ void tvwc_reduce_kernel(const uint32_t* __restrict__ partial, int groups, int32_t V,
                                   unsigned long long* __restrict__ counts) {
  for (int64_t w = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; w < V; w += int64_t(gridDim.x) * blockDim.x) {
    const int64_t b = w >> kFBLog2, l = w & (kFBucket - 1);
    unsigned long long s = 0;
    for (int k = 0; k < groups; ++k) s += partial[(b * groups + k) * kFBucket + l];
    counts[w] = s;
  }
}

}  // namespace

bool run_file_batch(gt_grammar* g, const int* tv_topk, int n_tv, gt_result** tv_out, gt_result** ii_out,
                    cudaStream_t s, uint64_t* wc_out) {
  if (file_strategy(g) == 2) {
    run_file_batch_bu(g, tv_topk, n_tv, tv_out, ii_out, s);
    return false;
  }
  FileHist fh;
  file_hist(g, s, fh);
  // the word count rides on the first full term vector's copy when there is one
  int fused = -1;
  for (int i = 0; i < n_tv && wc_out && fused < 0; ++i)
    if (tv_topk[i] == 0) fused = i;
  for (int i = 0; i < n_tv; ++i) tv_out[i] = term_vector_from(g, fh, tv_topk[i], s, i == fused ? wc_out : nullptr);
  if (ii_out) *ii_out = inverted_index_from(g, fh, s);
  if (!wc_out) return false;
  if (fused >= 0) return true;
  gt_ctx* ctx = g->ctx;
  const DevGrammar& d = g->d;
  Phase ph(ctx, "wc_from_files", s);
  const int groups = (d.F + kWcFileGroup - 1) / kWcFileGroup;
  if (groups == 0 || fh.nb == 0) {
    GT_CUDA(cudaMemsetAsync(wc_out, 0, size_t(d.V) * 8, s));
    return true;
  }
  TvSlots ts{fh.slot_word.as<int32_t>(), fh.slot_cnt.as<uint32_t>(), fh.nnz.as<int64_t>(), fh.bits.as<uint32_t>()};
  Buf partial(ctx, size_t(fh.nb) * groups * kFBucket * 4, s);
  tvwc_hist_kernel<<<unsigned(fh.nb * groups), kTvThreads, 0, s>>>(ts, d.F, fh.nb, groups, partial.as<uint32_t>());
  GT_LAUNCH_CHECK();
  tvwc_reduce_kernel<<<grid_for(d.V, 256, ctx->num_sms * 8), 256, 0, s>>>(
      partial.as<uint32_t>(), groups, d.V, reinterpret_cast<unsigned long long*>(wc_out));
  GT_LAUNCH_CHECK();
  return true;
}

gt_result* run_term_vector(gt_grammar* g, int top_k, cudaStream_t s) {
  gt_result* r = nullptr;
  run_file_batch(g, &top_k, 1, &r, nullptr, s);
  return r;
}

gt_result* run_inverted_index(gt_grammar* g, cudaStream_t s) {
  gt_result* r = nullptr;
  run_file_batch(g, nullptr, 0, nullptr, &r, s);
  return r;
}

}  // namespace gt
