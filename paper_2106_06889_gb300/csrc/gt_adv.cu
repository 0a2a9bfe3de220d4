// Analytics built on the same traversals (the Introduction and Related Work
// name TF-IDF and word co-occurrence as the analytics that follow the six of
// Section VI).
//
// TF-IDF: the term vector of every file (Section VI, either per-file
// strategy) with, per entry, count * ln(F / df(word)), df(word) = the number
// of files whose term vector holds the word (a histogram over the entries).
//
// Word co-occurrence within a window of three words: the ordered pairs
// (t[i], t[j]) with j - i in {1, 2} inside one file.  Every such pair is the
// (first, second) or (first, third) pair of exactly one 3-word window, except
// the last pair of each file, which starts no window.  So the pairs come from
// the global 3-word counts (Section IV-D's sequence support, gt_seq*.cu): two
// rows per distinct 3-gram weighted by its count, plus each file's last pair
// (from the root's last symbols and the children's tail buffers), sorted by
// pair key and summed.
#include "gt_device.cuh"

namespace gt {
namespace {

// Rows of the pairs of every 3-gram: (a, b) and (a, c) of key a|b|c with its
// count; rows past the number of 3-grams get the pad key.
__global__ void cooc_rows_kernel(const uint64_t* __restrict__ key3, const uint64_t* __restrict__ cnt3,
                                 const int64_t* __restrict__ n3_dev, int64_t bound, uint64_t key_pad,
                                 uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  const int64_t n3 = *n3_dev;
  const uint64_t m = (uint64_t(1) << 21) - 1;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < bound; i += int64_t(gridDim.x) * blockDim.x) {
    uint64_t k0 = key_pad, k1 = key_pad;
    uint32_t c = 0;
    if (i < n3) {
      const uint64_t k = key3[i];
      const uint64_t a = k >> 42, b = (k >> 21) & m, cw = k & m;
      k0 = (a << 21) | b;
      k1 = (a << 21) | cw;
      c = uint32_t(cnt3[i]);  // below 2^32: fewer than 2^32 tokens
    }
    keys[2 * i] = k0;
    keys[2 * i + 1] = k1;
    vals[2 * i] = c;
    vals[2 * i + 1] = c;
  }
}

// Last word of body symbol x (a word, or a rule's last word).
__device__ __forceinline__ int32_t last_word(const DevGrammar& d, const int32_t* __restrict__ tail, int32_t x) {
  return x < d.V ? x : tail[2 * (x - d.V) + 1];
}

// The last pair (second-to-last word, last word) of every file of two or more
// words, one row each (pad key otherwise).
__global__ void file_last_pair_kernel(DevGrammar d, const int32_t* __restrict__ tail, uint64_t key_pad,
                                      uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  for (int32_t f = blockIdx.x * blockDim.x + threadIdx.x; f < d.F; f += gridDim.x * blockDim.x) {
    const int64_t fo = d.file_off[f], fe = d.file_off[f + 1];
    int32_t last = -1, prev = -1;
    if (fe > fo) {
      const int32_t x = d.sym[fe - 1];
      last = last_word(d, tail, x);
      if (x >= d.V) prev = tail[2 * (x - d.V)];  // -1 for a rule of one word
      if (prev < 0 && fe - 2 >= fo) prev = last_word(d, tail, d.sym[fe - 2]);
    }
    const bool ok = last >= 0 && prev >= 0;
    keys[f] = ok ? (uint64_t(uint32_t(prev)) << 21) | uint64_t(uint32_t(last)) : key_pad;
    vals[f] = ok ? 1u : 0u;
  }
}

}  // namespace

gt_result* run_tfidf(gt_grammar* g, cudaStream_t s) {
  const int k = kTfIdf;
  gt_result* tv = nullptr;
  run_file_batch(g, &k, 1, &tv, nullptr, s);
  return tv;
}

gt_result* run_cooccurrence(gt_grammar* g, cudaStream_t s) {
  gt_ctx* ctx = g->ctx;
  const DevGrammar& d = g->d;
  if (d.V > (1 << 21)) fail(GT_EOVERFLOW, "pair keys need num_words <= 2^21");
  gt_result* seq = run_sequence_count(g, 0, s);
  try {
    void *k3 = nullptr, *c3 = nullptr;
    const int64_t* n3 = nullptr;
    result_device_field(seq, "key", &k3, &n3);
    result_device_field(seq, "count", &c3, &n3);
    const int64_t U = g->info.owned_windows;  // distinct 3-grams at most
    const int64_t n = 2 * U + d.F;
    const uint64_t key_pad = uint64_t(1) << 42;  // above every pair key
    Buf keys(ctx, size_t(n) * 8, s), vals(ctx, size_t(n) * 4, s);
    Buf tail(ctx, size_t(d.R) * 8, s), head(ctx, size_t(d.R) * 8, s);
    {
      Phase ph(ctx, "cooc_rows", s);
      run_head_tail(g, head.as<int32_t>(), tail.as<int32_t>(), s);
      const int threads = 256, cap = ctx->num_sms * 16;
      if (U > 0) {
        cooc_rows_kernel<<<grid_for(U, threads, cap), threads, 0, s>>>(
            static_cast<uint64_t*>(k3), static_cast<uint64_t*>(c3), n3, U, key_pad, keys.as<uint64_t>(),
            vals.as<uint32_t>());
        GT_LAUNCH_CHECK();
      }
      file_last_pair_kernel<<<grid_for(d.F, threads, cap), threads, 0, s>>>(
          d, tail.as<int32_t>(), key_pad, keys.as<uint64_t>() + 2 * U, vals.as<uint32_t>() + 2 * U);
      GT_LAUNCH_CHECK();
    }
    gt_result* out = reduce_key_rows(ctx, keys, vals, n, 43, key_pad, s, reinterpret_cast<uint32_t*>(seq->d_lens));
    out->deps.push_back(seq);  // the 3-gram result's buffers live until this result is freed
    return out;
  } catch (...) {
    gt_free_result(seq);
    throw;
  }
}

// Device pointer and device length slot of a field of a result under construction.
void result_device_field(gt_result* r, const char* field, void** ptr, const int64_t** d_len) {
  for (auto& f : r->fields)
    if (f.name == field) {
      *ptr = f.ptr;
      if (!f.len_src) fail(GT_EINVAL, "field has a fixed length");
      *d_len = r->d_lens + (f.len_src - r->h_lens);
      return;
    }
  fail(GT_ENOTFOUND, std::string("unknown result field: ") + field);
}

}  // namespace gt
