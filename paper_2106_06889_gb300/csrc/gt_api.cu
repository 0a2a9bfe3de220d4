// The gt_* C ABI: contexts, grammar load, result objects and the host-side
// orchestration of each analytic.  Every step of every analytic runs in this
// library's CUDA kernels; there is no CPU path.
#include <algorithm>
#include <cstring>
#include <memory>
#include <new>

#include <unordered_map>

#include "gt_device.cuh"

using gt::Buf;
using gt::fail;

namespace gt {
std::atomic<long long> g_launches{0};
thread_local gt_ctx* t_call_ctx = nullptr;
}

namespace {

template <class F>
gt_status guard(gt_ctx* ctx, F&& f) {
  try {
    f();
    if (ctx) ctx->last_error.clear();
    return GT_OK;
  } catch (const gt::Error& e) {
    if (ctx) ctx->last_error = e.msg;
    return e.code;
  } catch (const std::bad_alloc&) {
    if (ctx) ctx->last_error = "host allocation failed";
    return GT_ENOMEM;
  } catch (...) {
    if (ctx) ctx->last_error = "unexpected failure";
    return GT_ECUDA;
  }
}

cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

void use_device(gt_ctx* ctx) {
  GT_CUDA(cudaSetDevice(ctx->device));
  gt::t_call_ctx = ctx;
}

gt_status status_to_code(uint32_t st) {
  if (st & gt::ST_INVALID) return GT_EINVAL;
  if (st & gt::ST_TIMEOUT) return GT_ETIMEOUT;
  if (st & gt::ST_TABLE_FULL) return GT_ETABLE_FULL;
  if (st & gt::ST_OVERFLOW) return GT_EOVERFLOW;
  return GT_OK;
}

const char* status_text(uint32_t st) {
  if (st & gt::ST_INVALID) return "device detected an invalid input";
  if (st & gt::ST_TIMEOUT) return "a bounded device wait timed out";
  if (st & gt::ST_TABLE_FULL) return "a device hash table ran out of slots";
  if (st & gt::ST_OVERFLOW) return "a device counter overflowed";
  return "";
}

__global__ void nonzero_flags_kernel(const uint64_t* __restrict__ c, int64_t n, int64_t* __restrict__ flag) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    flag[i] = c[i] != 0;
}

__global__ void compact_words_kernel(const uint64_t* __restrict__ c, int64_t n, const int64_t* __restrict__ pos,
                                     int32_t* __restrict__ words, uint64_t* __restrict__ counts,
                                     int64_t* __restrict__ total) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const uint64_t v = c[i];
    if (v) {
      words[pos[i]] = int32_t(i);
      counts[pos[i]] = v;
    }
    if (i == n - 1) *total = pos[i] + (v != 0);
  }
}

// key = N - count: ascending key order is descending count; words with count
// zero get key N and sort last.
__global__ void count_keys_kernel(const uint64_t* __restrict__ c, int64_t n, uint64_t N, uint64_t* __restrict__ keys,
                                  uint32_t* __restrict__ vals) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    keys[i] = N - c[i];
    vals[i] = uint32_t(i);
  }
}

__global__ void count_unkey_kernel(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ vals, int64_t n,
                                   uint64_t N, int32_t* __restrict__ words, uint64_t* __restrict__ counts,
                                   int64_t* __restrict__ total) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const uint64_t cnt = N - keys[i];
    words[i] = int32_t(vals[i]);
    counts[i] = cnt;
    if (cnt != 0 && (i == n - 1 || keys[i + 1] == N)) *total = i + 1;
  }
}

int bits_for(uint64_t x) {
  int b = 0;
  while (b < 64 && (uint64_t(1) << b) <= x) ++b;
  return b;
}

}  // namespace

// ============================================================================
// context
// ============================================================================

GT_API gt_status gt_create(gt_ctx** out, int device, size_t pool_bytes) {
  if (!out) return GT_EINVAL;
  *out = nullptr;
  gt_ctx* ctx = new (std::nothrow) gt_ctx();
  if (!ctx) return GT_ENOMEM;
  gt_status st = guard(ctx, [&] {
    int n = 0;
    GT_CUDA(cudaGetDeviceCount(&n));
    if (device < 0 || device >= n) fail(GT_ECUDA, "no such CUDA device");
    cudaDeviceProp prop;
    GT_CUDA(cudaGetDeviceProperties(&prop, device));
    if (prop.major != 10 || prop.minor != 3)
      fail(GT_ECUDA, "libgtadoc.so is built for sm_103a (GB300); this device is sm_" + std::to_string(prop.major) +
                         std::to_string(prop.minor));
    ctx->device = device;
    ctx->num_sms = prop.multiProcessorCount;
    GT_CUDA(cudaSetDevice(device));
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    GT_CUDA(cudaMemPoolCreate(&ctx->pool, &props));
    uint64_t thr = pool_bytes ? uint64_t(pool_bytes) : ~uint64_t(0);
    GT_CUDA(cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, &thr));
    GT_CUDA(cudaMalloc(&ctx->d_status, 64));
    GT_CUDA(cudaMemset(ctx->d_status, 0, 64));
  });
  if (st != GT_OK) {
    gt_destroy(ctx);
    return st;
  }
  *out = ctx;
  return GT_OK;
}

GT_API gt_status gt_destroy(gt_ctx* ctx) {
  if (!ctx) return GT_EINVAL;
  cudaSetDevice(ctx->device);
  for (cudaEvent_t e : ctx->free_events) cudaEventDestroy(e);
  for (void* p : ctx->pinned_chunks) cudaFreeHost(p);
  gt_profile_reset(ctx);
  if (ctx->d_status) cudaFree(ctx->d_status);
  if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
  delete ctx;
  return GT_OK;
}

GT_API const char* gt_last_error(const gt_ctx* ctx) { return ctx ? ctx->last_error.c_str() : "null context"; }

GT_API gt_status gt_sync(gt_ctx* ctx, void* stream) {
  if (!ctx) return GT_EINVAL;
  uint32_t st = 0;
  gt_status rc = guard(ctx, [&] {
    use_device(ctx);
    GT_CUDA(cudaStreamSynchronize(as_stream(stream)));
    GT_CUDA(cudaMemcpy(&st, ctx->d_status, 4, cudaMemcpyDeviceToHost));
    GT_CUDA(cudaMemset(ctx->d_status, 0, 4));
  });
  if (rc != GT_OK) return rc;
  if (st) ctx->last_error = status_text(st);
  return status_to_code(st);
}

// ============================================================================
// grammar
// ============================================================================

GT_API gt_status gt_load_grammar(gt_ctx* ctx, const gt_grammar_desc* desc, void* stream, gt_grammar** out) {
  if (!ctx || !desc || !out) return GT_EINVAL;
  *out = nullptr;
  gt_grammar* g = new (std::nothrow) gt_grammar();
  if (!g) return GT_ENOMEM;
  g->ctx = ctx;
  cudaStream_t s = as_stream(stream);
  gt_status st = guard(ctx, [&] {
    use_device(ctx);
    const int32_t V = desc->num_words, R = desc->num_rules, F = desc->num_files;
    if (V < 1 || R < 1 || F < 1) fail(GT_EINVAL, "num_words, num_rules and num_files must be >= 1");
    if (int64_t(V) + int64_t(R) >= (int64_t(1) << 31)) fail(GT_EOVERFLOW, "num_words + num_rules must be < 2^31");
    if (!desc->rule_off || !desc->file_off) fail(GT_EINVAL, "null offsets");
    // validate the offsets on the host: the caller's arrays in place, or a
    // copy when they live on the device
    std::vector<int64_t> roff_copy, foff_copy;
    const int64_t* roff = desc->rule_off;
    const int64_t* foff = desc->file_off;
    if (desc->on_device) {
      roff_copy.resize(size_t(R) + 1);
      foff_copy.resize(size_t(F) + 1);
      GT_CUDA(cudaMemcpy(roff_copy.data(), desc->rule_off, roff_copy.size() * 8, cudaMemcpyDeviceToHost));
      GT_CUDA(cudaMemcpy(foff_copy.data(), desc->file_off, foff_copy.size() * 8, cudaMemcpyDeviceToHost));
      roff = roff_copy.data();
      foff = foff_copy.data();
    }
    if (roff[0] != 0) fail(GT_EINVAL, "rule_off[0] must be 0");
    for (int32_t r = 0; r < R; ++r) {
      if (roff[r + 1] < roff[r]) fail(GT_EINVAL, "rule_off must be non-decreasing");
      if (r > 0 && roff[r + 1] == roff[r]) fail(GT_EINVAL, "every non-root rule body must be non-empty");
      // edge multiplicities are 32-bit: a body (the root included) holds fewer than 2^32 symbols
      if (roff[r + 1] - roff[r] >= (int64_t(1) << 32)) fail(GT_EOVERFLOW, "a rule body of 2^32 symbols or more");
    }
    const int64_t G = roff[R], root_len = roff[1];
    if (G >= (int64_t(1) << 40)) fail(GT_EOVERFLOW, "grammar too large");
    if (foff[0] != 0 || foff[F] != root_len) fail(GT_EINVAL, "file_off must start at 0 and end at the root length");
    for (int32_t f = 0; f < F; ++f)
      if (foff[f + 1] < foff[f]) fail(GT_EINVAL, "file_off must be non-decreasing");
    if (G > 0 && !desc->sym) fail(GT_EINVAL, "null sym");

    gt::DevGrammar& d = g->d;
    d.V = V;
    d.R = R;
    d.F = F;
    d.G = G;
    d.root_len = root_len;
    // symbols padded to whole tiles, plus 16 bytes, with -1 (never a word,
    // never a rule): a 16-byte vector load that starts at a symbol stays in
    // the array; uploads go straight from the caller's arrays (DMA when they
    // are pinned)
    const cudaMemcpyKind up = desc->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    auto upload_phase = std::make_unique<gt::Phase>(ctx, "load_upload", s);
    const int64_t Gp = std::max<int64_t>((G + gt::kTile - 1) / gt::kTile, 1) * gt::kTile + 4;
    void* p = gt::grammar_alloc(g, size_t(Gp) * 4, s);
    GT_CUDA(cudaMemsetAsync(static_cast<int32_t*>(p) + G, 0xff, size_t(Gp - G) * 4, s));
    if (G > 0) GT_CUDA(cudaMemcpyAsync(p, desc->sym, size_t(G) * 4, up, s));
    d.sym = static_cast<int32_t*>(p);
    p = gt::grammar_alloc(g, size_t(R + 1) * 8, s);
    GT_CUDA(cudaMemcpyAsync(p, desc->rule_off, size_t(R + 1) * 8, up, s));
    d.rule_off = static_cast<int64_t*>(p);
    p = gt::grammar_alloc(g, size_t(F + 1) * 8, s);
    GT_CUDA(cudaMemcpyAsync(p, desc->file_off, size_t(F + 1) * 8, up, s));
    d.file_off = static_cast<int64_t*>(p);
    {
      // file-pure chunks of the root (per-file analytics), one upload
      std::vector<int64_t> cs, cf(size_t(F) + 2);
      std::vector<int32_t> cl;
      for (int32_t f = 0; f < F; ++f) {
        cf[f] = int64_t(cs.size());
        for (int64_t q = foff[f]; q < foff[f + 1]; q += gt::kRootChunk) {
          cs.push_back(q);
          cl.push_back(int32_t(std::min<int64_t>(gt::kRootChunk, foff[f + 1] - q)));
        }
      }
      const int64_t nc = int64_t(cs.size());
      cf[F] = nc;
      cf[F + 1] = nc;
      g->root_chunks = nc;
      std::vector<char> blob(size_t(nc + 1) * 8 + size_t(F + 2) * 8 + size_t(nc + 1) * 4);
      char* bp = blob.data();
      std::memcpy(bp, cs.data(), size_t(nc) * 8);
      std::memcpy(bp + size_t(nc + 1) * 8, cf.data(), size_t(F + 2) * 8);
      std::memcpy(bp + size_t(nc + 1) * 8 + size_t(F + 2) * 8, cl.data(), size_t(nc) * 4);
      char* q = static_cast<char*>(gt::grammar_alloc(g, blob.size(), s));
      GT_CUDA(cudaMemcpyAsync(q, blob.data(), blob.size(), cudaMemcpyHostToDevice, s));
      upload_phase.reset();
      GT_CUDA(cudaStreamSynchronize(s));  // blob is a host temporary
      d.rch_start = reinterpret_cast<int64_t*>(q);
      d.rch_foff = reinterpret_cast<int64_t*>(q + size_t(nc + 1) * 8);
      d.rch_count = d.rch_foff + F + 1;
      d.rch_len = reinterpret_cast<int32_t*>(q + size_t(nc + 1) * 8 + size_t(F + 2) * 8);
    }
    {
      gt::Phase ph(ctx, "load_dag", s);
      gt::load_build_dag(g, s);
    }
    {
      // the top-down per-file layout (<= 64 files): DAG facts every per-file query reuses
      gt::Phase ph(ctx, "load_file_layout", s);
      gt::file_sizes(g, s);
    }
    g->info.file_pairs = g->fentry_bound;
    g->info.file_words = g->fword_bound;
    g->info.num_words = V;
    g->info.num_rules = R;
    g->info.num_files = F;
    g->info.num_syms = G;
  });
  if (st != GT_OK) {
    gt_free_grammar(g);
    return st;
  }
  *out = g;
  return GT_OK;
}

GT_API gt_status gt_free_grammar(gt_grammar* g) {
  if (!g) return GT_EINVAL;
  cudaSetDevice(g->ctx->device);
  cudaDeviceSynchronize();
  for (auto& e : g->wc_graphs)
    if (e.exec) cudaGraphExecDestroy(e.exec);
  if (g->seq_tile_ev) cudaEventDestroy(g->seq_tile_ev);
  for (void* p : g->owned) cudaFreeAsync(p, nullptr);  // grammar memory comes from the context pool
  delete g;
  return GT_OK;
}

GT_API gt_status gt_grammar_info_get(const gt_grammar* g, gt_grammar_info* info) {
  if (!g || !info) return GT_EINVAL;
  *info = g->info;
  return GT_OK;
}

// ============================================================================
// analytics
// ============================================================================

GT_API gt_status gt_rule_weights(gt_grammar* g, uint64_t* d_weights, void* stream) {
  if (!g || !d_weights) return GT_EINVAL;
  return guard(g->ctx, [&] {
    use_device(g->ctx);
    gt::run_rule_weights(g, d_weights, as_stream(stream));
  });
}

namespace {

void word_count_direct(gt_grammar* g, uint64_t* d_counts, cudaStream_t s, uint32_t* status = nullptr) {
  Buf wt(g->ctx, size_t(g->d.R) * 8, s);
  gt::run_rule_weights(g, wt.as<uint64_t>(), s);
  gt::run_word_count(g, wt.as<uint64_t>(), d_counts, s, status);
}

__global__ void or_status_kernel(uint32_t* __restrict__ dst, const uint32_t* __restrict__ src) {
  if (*src) atomicOr(dst, *src);
}

// The whole word-count launch sequence of one grammar into one output buffer,
// captured once as a CUDA graph (scratch allocations and frees included as
// graph memory nodes) and replayed: one launch instead of about a dozen.
// Launches the replay on s and returns true, or returns false (first call
// with this buffer, or the sequence cannot be captured).  The lock is held
// through the launch, so an eviction by another thread cannot free the exec
// in between.
bool word_count_graph(gt_grammar* g, uint64_t* d_counts, cudaStream_t s) {
  std::lock_guard<std::mutex> lk(g->graph_mu);
  gt_grammar::WcGraph* ent = nullptr;
  for (auto& e : g->wc_graphs)
    if (e.out == d_counts) ent = &e;
  const uint64_t now = ++g->graph_tick;
  if (ent) ent->last_use = now;
  auto replay = [&](const gt_grammar::WcGraph& e) {
    GT_CUDA(cudaGraphLaunch(e.exec, s));
    gt::g_launches.fetch_add(e.kernels);
    return true;
  };
  if (ent && ent->exec) return replay(*ent);
  if (!ent) {  // first call with this buffer: run directly, capture on the next one
    if (g->wc_graphs.size() >= gt_grammar::kMaxWcGraphs) {
      // evict the least recently used entry (an exec still running is freed
      // by CUDA once it completes)
      auto lru = std::min_element(g->wc_graphs.begin(), g->wc_graphs.end(),
                                  [](const auto& a, const auto& b) { return a.last_use < b.last_use; });
      if (lru->exec) cudaGraphExecDestroy(lru->exec);
      g->wc_graphs.erase(lru);
    }
    g->wc_graphs.push_back({d_counts, nullptr, now, 0});
    return false;
  }
  const long long l0 = gt::g_launches.load();
  cudaStream_t cs;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return false;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  if (ok) {
    try {
      word_count_direct(g, d_counts, cs);
    } catch (const gt::Error&) {
      ok = false;
    }
    const cudaError_t e = cudaStreamEndCapture(cs, &graph);
    ok = ok && e == cudaSuccess && graph;
  }
  if (ok) ok = cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(cs);
  cudaGetLastError();  // a refused capture leaves no sticky error
  // kernels recorded during capture did not run; replays account for them
  const long long recorded = gt::g_launches.load() - l0;
  gt::g_launches.fetch_sub(recorded);
  if (!ok) return false;
  ent->exec = exec;
  ent->kernels = int(recorded);
  return replay(*ent);
}

// Word count into d_counts: replayed from a graph when allowed (not while
// profiling, so that phase timers keep seeing each launch).
void word_count_any(gt_grammar* g, uint64_t* d_counts, cudaStream_t s) {
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  GT_CUDA(cudaStreamIsCapturing(s, &cap));
  const bool replayed = g->ctx->param("use_graphs", 1) && !g->ctx->prof_on && cap == cudaStreamCaptureStatusNone &&
                        word_count_graph(g, d_counts, s);
  if (!replayed) word_count_direct(g, d_counts, s);
}

}  // namespace

GT_API gt_status gt_word_count(gt_grammar* g, uint64_t* d_counts, void* stream) {
  if (!g || !d_counts) return GT_EINVAL;
  return guard(g->ctx, [&] {
    use_device(g->ctx);
    word_count_any(g, d_counts, as_stream(stream));
  });
}

GT_API gt_status gt_word_count_batch(gt_grammar* const* gs, uint64_t* const* d_counts, int n, void* stream) {
  if (!gs || !d_counts || n < 1) return GT_EINVAL;
  for (int i = 0; i < n; ++i)
    if (!gs[i] || !d_counts[i] || gs[i]->ctx != gs[0]->ctx) return GT_EINVAL;
  return guard(gs[0]->ctx, [&] {
    use_device(gs[0]->ctx);
    for (int a = 0; a < n; a += 64)
      gt::run_word_count_multi(const_cast<gt_grammar**>(gs) + a, d_counts + a, std::min(64, n - a), as_stream(stream));
  });
}

GT_API gt_status gt_head_tail(gt_grammar* g, int32_t* d_head, int32_t* d_tail, void* stream) {
  if (!g || !d_head || !d_tail) return GT_EINVAL;
  return guard(g->ctx, [&] {
    use_device(g->ctx);
    gt::run_head_tail(g, d_head, d_tail, as_stream(stream));
  });
}

namespace {

// Sort result from already computed word counts.
// wc_status: device status word of the word count that produced wc.
gt_result* sort_from_counts(gt_grammar* g, const uint64_t* wc, int order, cudaStream_t s,
                            const uint32_t* wc_status) {
  gt_ctx* ctx = g->ctx;
  const int64_t V = g->d.V;
  const int threads = 256, cap = ctx->num_sms * 8;
  gt::ResultBuilder rb(ctx, s);
  auto* words = static_cast<int32_t*>(rb.alloc(size_t(V) * 4));
  auto* counts = static_cast<uint64_t*>(rb.alloc(size_t(V) * 8));
  int64_t* nlen = rb.new_len_slot();
  gt::Phase ph(ctx, "sort_canon", s);
  if (order == 0) {
    Buf flag(ctx, size_t(V) * 8, s), pos(ctx, size_t(V) * 8, s), sc(ctx, gt::scan_scratch_bytes(V), s);
    nonzero_flags_kernel<<<gt::grid_for(V, threads, cap), threads, 0, s>>>(wc, V, flag.as<int64_t>());
    GT_LAUNCH_CHECK();
    gt::exclusive_scan_i64(flag.as<int64_t>(), pos.as<int64_t>(), V, sc.p, s);
    compact_words_kernel<<<gt::grid_for(V, threads, cap), threads, 0, s>>>(wc, V, pos.as<int64_t>(), words, counts,
                                                                            nlen);
    GT_LAUNCH_CHECK();
  } else {
    const uint64_t N = g->d.N;
    Buf k0(ctx, size_t(V) * 8, s), k1(ctx, size_t(V) * 8, s), v0(ctx, size_t(V) * 4, s), v1(ctx, size_t(V) * 4, s);
    Buf rs(ctx, gt::radix_scratch_bytes(V, true, 4), s);
    count_keys_kernel<<<gt::grid_for(V, threads, cap), threads, 0, s>>>(wc, V, N, k0.as<uint64_t>(),
                                                                        v0.as<uint32_t>());
    GT_LAUNCH_CHECK();
    gt::radix_sort_u64(k0.as<uint64_t>(), k1.as<uint64_t>(), v0.p, v1.p, 4, V, 0, bits_for(N), rs.p, s);
    count_unkey_kernel<<<gt::grid_for(V, threads, cap), threads, 0, s>>>(k1.as<uint64_t>(), v1.as<uint32_t>(), V, N,
                                                                         words, counts, nlen);
    GT_LAUNCH_CHECK();
  }
  rb.field_dyn("word", words, nlen);
  rb.field_dyn("count", counts, nlen);
  GT_CUDA(cudaMemcpyAsync(rb.status(), wc_status, 4, cudaMemcpyDeviceToDevice, s));
  return rb.finish();
}

}  // namespace

GT_API gt_status gt_sort(gt_grammar* g, int order, void* stream, gt_result** out) {
  if (!g || !out || (order != 0 && order != 1)) return GT_EINVAL;
  *out = nullptr;
  return guard(g->ctx, [&] {
    use_device(g->ctx);
    cudaStream_t s = as_stream(stream);
    Buf wc(g->ctx, size_t(g->d.V) * 8, s), wst(g->ctx, 4, s);
    GT_CUDA(cudaMemsetAsync(wst.p, 0, 4, s));
    {
      Buf wt(g->ctx, size_t(g->d.R) * 8, s);
      gt::run_rule_weights(g, wt.as<uint64_t>(), s);
      gt::run_word_count(g, wt.as<uint64_t>(), wc.as<uint64_t>(), s, wst.as<uint32_t>());
    }
    *out = sort_from_counts(g, wc.as<uint64_t>(), order, s, wst.as<uint32_t>());
  });
}

GT_API gt_status gt_term_vector(gt_grammar* g, int top_k, void* stream, gt_result** out) {
  if (!g || !out || top_k < 0) return GT_EINVAL;
  *out = nullptr;
  return guard(g->ctx, [&] {
    use_device(g->ctx);
    *out = gt::run_term_vector(g, top_k, as_stream(stream));
  });
}

GT_API gt_status gt_sequence_count(gt_grammar* g, int per_file, void* stream, gt_result** out) {
  if (!g || !out || (per_file != 0 && per_file != 1)) return GT_EINVAL;
  *out = nullptr;
  return guard(g->ctx, [&] {
    use_device(g->ctx);
    *out = gt::run_sequence_count(g, per_file, as_stream(stream));
  });
}

GT_API gt_status gt_ranked_index(gt_grammar* g, int n, void* stream, gt_result** out) {
  if (!g || !out || (n != 1 && n != 3)) return GT_EINVAL;
  *out = nullptr;
  return guard(g->ctx, [&] {
    use_device(g->ctx);
    *out = n == 3 ? gt::run_ranked_windows(g, as_stream(stream)) : gt::run_ranked_words(g, as_stream(stream));
  });
}

GT_API gt_status gt_tfidf(gt_grammar* g, void* stream, gt_result** out) {
  if (!g || !out) return GT_EINVAL;
  *out = nullptr;
  return guard(g->ctx, [&] {
    use_device(g->ctx);
    *out = gt::run_tfidf(g, as_stream(stream));
  });
}

GT_API gt_status gt_cooccurrence(gt_grammar* g, void* stream, gt_result** out) {
  if (!g || !out) return GT_EINVAL;
  *out = nullptr;
  return guard(g->ctx, [&] {
    use_device(g->ctx);
    *out = gt::run_cooccurrence(g, as_stream(stream));
  });
}

GT_API gt_status gt_inverted_index(gt_grammar* g, void* stream, gt_result** out) {
  if (!g || !out) return GT_EINVAL;
  *out = nullptr;
  return guard(g->ctx, [&] {
    use_device(g->ctx);
    *out = gt::run_inverted_index(g, as_stream(stream));
  });
}

// ============================================================================
// batches: several analytics over one or more grammars, one traversal each
// ============================================================================

GT_API gt_status gt_run_batch(gt_ctx* ctx, const gt_query* q, int nq, void* stream, gt_result** out) {
  if (!ctx || (nq > 0 && (!q || !out)) || nq < 0) return GT_EINVAL;
  for (int i = 0; i < nq; ++i) {
    out[i] = nullptr;
    if (!q[i].grammar || q[i].grammar->ctx != ctx) return GT_EINVAL;
    if (q[i].kind < GT_Q_WORD_COUNT || q[i].kind > GT_Q_COOCCURRENCE) return GT_EINVAL;
    if (q[i].kind == GT_Q_SEQUENCE_COUNT && q[i].param != 0 && q[i].param != 1) return GT_EINVAL;
    if (q[i].kind == GT_Q_RANKED_INDEX && q[i].param != 1 && q[i].param != 3) return GT_EINVAL;
    if (q[i].kind == GT_Q_WORD_COUNT && !q[i].d_counts) return GT_EINVAL;
    if (q[i].kind == GT_Q_SORT && q[i].param != 0 && q[i].param != 1) return GT_EINVAL;
    if (q[i].kind == GT_Q_TERM_VECTOR && q[i].param < 0) return GT_EINVAL;
  }
  gt_status st = guard(ctx, [&] {
    use_device(ctx);
    cudaStream_t s = as_stream(stream);
    std::vector<bool> done(size_t(nq), false);
    // ---- word counts (and the sorts built on them): one counts buffer per
    // grammar, and the word counts of all grammars in one fused launch sequence ----
    std::vector<gt_grammar*> wg;
    std::vector<uint64_t*> wc;
    std::vector<Buf> wscratch;
    wscratch.reserve(size_t(nq));
    std::unordered_map<gt_grammar*, uint64_t*> counts_of;
    for (int i = 0; i < nq; ++i) {
      if (q[i].kind != GT_Q_WORD_COUNT && q[i].kind != GT_Q_SORT) continue;
      gt_grammar* g = q[i].grammar;
      if (counts_of.count(g)) continue;
      uint64_t* counts = nullptr;
      for (int j = i; j < nq && !counts; ++j)
        if (q[j].grammar == g && q[j].kind == GT_Q_WORD_COUNT) counts = q[j].d_counts;
      if (!counts) {
        wscratch.emplace_back(ctx, size_t(g->d.V) * 8, s);
        counts = wscratch.back().as<uint64_t>();
      }
      counts_of[g] = counts;
      wg.push_back(g);
      wc.push_back(counts);
    }
    // a grammar that also has term-vector / inverted-index queries takes its
    // counts from that traversal (the sum of the per-file counts, top-down)
    std::unordered_map<gt_grammar*, bool> from_files;
    for (int i = 0; i < nq; ++i) {
      gt_grammar* g = q[i].grammar;
      if ((q[i].kind == GT_Q_TERM_VECTOR || q[i].kind == GT_Q_INVERTED_INDEX) && counts_of.count(g) &&
          gt::file_strategy(g) == 1)
        from_files[g] = true;
    }
    std::vector<gt_grammar*> fg;
    std::vector<uint64_t*> fc;
    for (size_t k = 0; k < wg.size(); ++k)
      if (!from_files.count(wg[k])) {
        fg.push_back(wg[k]);
        fc.push_back(wc[k]);
      }
    // this batch's own status word: sorts report the flags of the word counts
    // they are built on, word-count queries also through the context's word
    Buf bst(ctx, 4, s);
    GT_CUDA(cudaMemsetAsync(bst.p, 0, 4, s));
    bool any_sort = false, used_bst = !fg.empty();
    for (int i = 0; i < nq; ++i) any_sort = any_sort || q[i].kind == GT_Q_SORT;
    if (fg.size() == 1) {
      bool caller = false;
      for (int i = 0; i < nq; ++i)
        if (q[i].grammar == fg[0] && q[i].kind == GT_Q_WORD_COUNT && q[i].d_counts == fc[0]) caller = true;
      if (caller && !any_sort) {
        word_count_any(fg[0], fc[0], s);  // caller buffer: graph-replayable (flags go to the context word)
        used_bst = false;
      } else
        word_count_direct(fg[0], fc[0], s, bst.as<uint32_t>());
    } else {
      for (size_t a = 0; a < fg.size(); a += 64)
        gt::run_word_count_multi(fg.data() + a, fc.data() + a, int(std::min<size_t>(64, fg.size() - a)), s,
                                 bst.as<uint32_t>());
    }
    for (int i = 0; i < nq; ++i) {
      if (done[i]) continue;
      gt_grammar* g = q[i].grammar;
      std::vector<int> same;
      for (int j = i; j < nq; ++j)
        if (!done[j] && q[j].grammar == g) same.push_back(j);
      // term vectors and inverted index share the per-file traversal
      std::vector<int> tv_idx, tv_k;
      int ii = -1;
      for (int j : same) {
        if (q[j].kind == GT_Q_TERM_VECTOR || q[j].kind == GT_Q_TFIDF) {  // TF-IDF: a term vector with idf
          tv_idx.push_back(j);
          tv_k.push_back(q[j].kind == GT_Q_TFIDF ? gt::kTfIdf : q[j].param);
        }
        if (q[j].kind == GT_Q_INVERTED_INDEX && ii < 0) ii = j;
      }
      if (!tv_idx.empty() || ii >= 0) {
        std::vector<gt_result*> tvr(tv_idx.size(), nullptr);
        gt_result* iir = nullptr;
        gt::run_file_batch(g, tv_k.data(), int(tv_k.size()), tvr.data(), ii >= 0 ? &iir : nullptr, s,
                           from_files.count(g) ? counts_of[g] : nullptr);
        for (size_t k = 0; k < tv_idx.size(); ++k) out[tv_idx[k]] = tvr[k];
        if (ii >= 0) out[ii] = iir;
        for (int j : same)  // a second inverted-index query on the same grammar gets its own copy
          if (q[j].kind == GT_Q_INVERTED_INDEX && j != ii) out[j] = gt::run_inverted_index(g, s);
      }
      for (int j : same) {
        if (q[j].kind == GT_Q_SEQUENCE_COUNT) out[j] = gt::run_sequence_count(g, q[j].param, s);
        if (q[j].kind == GT_Q_RANKED_INDEX)
          out[j] = q[j].param == 3 ? gt::run_ranked_windows(g, s) : gt::run_ranked_words(g, s);
        if (q[j].kind == GT_Q_COOCCURRENCE) out[j] = gt::run_cooccurrence(g, s);
      }
      for (int j : same) done[j] = true;
    }
    // word-count copies and sorts, once every grammar's counts are enqueued
    for (int j = 0; j < nq; ++j) {
      if (q[j].kind == GT_Q_WORD_COUNT && q[j].d_counts != counts_of[q[j].grammar])
        GT_CUDA(cudaMemcpyAsync(q[j].d_counts, counts_of[q[j].grammar], size_t(q[j].grammar->d.V) * 8,
                                cudaMemcpyDeviceToDevice, s));
      if (q[j].kind == GT_Q_SORT)
        out[j] = sort_from_counts(q[j].grammar, counts_of[q[j].grammar], q[j].param, s, bst.as<uint32_t>());
    }
    if (used_bst) {
      or_status_kernel<<<1, 1, 0, s>>>(ctx->d_status, bst.as<uint32_t>());
      GT_LAUNCH_CHECK();
    }
  });
  if (st != GT_OK)
    for (int i = 0; i < nq; ++i)
      if (out[i]) {
        gt_free_result(out[i]);
        out[i] = nullptr;
      }
  return st;
}

// ============================================================================
// results
// ============================================================================

GT_API gt_status gt_result_view(gt_result* r, const char* field, const void** d_ptr, int64_t* len) {
  if (!r || !field || !d_ptr || !len) return GT_EINVAL;
  gt_ctx* ctx = r->ctx;
  gt_status rc = guard(ctx, [&] {
    if (!r->ready) {
      GT_CUDA(cudaEventSynchronize(r->done));
      for (auto& f : r->fields)
        if (f.len_src) f.len = *f.len_src;
      r->ready = true;
    }
  });
  if (rc != GT_OK) return rc;
  const uint32_t st = uint32_t(r->h_lens[0]);
  if (st) {
    ctx->last_error = status_text(st);
    return status_to_code(st);
  }
  for (auto& f : r->fields)
    if (f.name == field) {
      *d_ptr = f.ptr;
      *len = f.len;
      return GT_OK;
    }
  ctx->last_error = std::string("unknown result field: ") + field;
  return GT_ENOTFOUND;
}

GT_API gt_status gt_free_result(gt_result* r) {
  if (!r) return GT_EINVAL;
  cudaSetDevice(r->ctx->device);
  if (r->done) cudaEventSynchronize(r->done);
  for (void* p : r->owned) cudaFreeAsync(p, nullptr);
  r->ctx->give_back(r->h_lens, r->done);
  for (gt_result* x : r->deps) gt_free_result(x);  // done before r: same stream, earlier work
  delete r;
  return GT_OK;
}

// ============================================================================
// profiling
// ============================================================================

GT_API gt_status gt_profile_enable(gt_ctx* ctx, int on) {
  if (!ctx) return GT_EINVAL;
  ctx->prof_on = on != 0;
  return GT_OK;
}

GT_API gt_status gt_profile_reset(gt_ctx* ctx) {
  if (!ctx) return GT_EINVAL;
  cudaSetDevice(ctx->device);
  for (auto& kv : ctx->prof)
    for (auto& sp : kv.second) {
      cudaEventSynchronize(sp.b);
      cudaEventDestroy(sp.a);
      cudaEventDestroy(sp.b);
    }
  ctx->prof.clear();
  return GT_OK;
}

GT_API gt_status gt_profile_read(gt_ctx* ctx, const char* phase, double* total_ms, int64_t* spans,
                                 int64_t* launches) {
  if (!ctx || !phase || !total_ms || !spans || !launches) return GT_EINVAL;
  *total_ms = 0;
  *spans = 0;
  *launches = 0;
  auto it = ctx->prof.find(phase);
  if (it == ctx->prof.end()) return GT_OK;
  return guard(ctx, [&] {
    use_device(ctx);
    for (auto& sp : it->second) {
      GT_CUDA(cudaEventSynchronize(sp.b));
      float ms = 0;
      GT_CUDA(cudaEventElapsedTime(&ms, sp.a, sp.b));
      *total_ms += ms;
      *spans += 1;
      *launches += sp.launches;
    }
  });
}

GT_API int64_t gt_kernel_launches(void) { return gt::g_launches.load(); }

// ============================================================================
// self-check of the bounded look-back wait
// ============================================================================

namespace {

// Item 1 looks back at item 0: flags[0] is either never published (the wait
// runs out after `polls` polls) or published with the prefix `pre`.
__global__ void wait_check_kernel(unsigned long long* flags, int publish, uint64_t pre, int polls,
                                  unsigned* status, int64_t* out) {
  if (publish && threadIdx.x == 0) gt::publish_aggregate(flags, 0, pre);
  __syncwarp();
  const int64_t p = gt::warp_look_back(flags, 1, 5, status, polls);
  if (threadIdx.x == 0) *out = p;
}

}  // namespace

GT_API gt_status gt_check_bounded_wait(gt_ctx* ctx, int publish, int64_t polls, int64_t* prefix) {
  if (!ctx || !prefix || polls < 1 || polls > (int64_t(1) << 24)) return GT_EINVAL;
  return guard(ctx, [&] {
    use_device(ctx);
    cudaStream_t s = nullptr;
    gt::Buf b(ctx, 64, s);
    GT_CUDA(cudaMemsetAsync(b.p, 0, 64, s));
    auto* flags = b.as<unsigned long long>();
    auto* st = reinterpret_cast<unsigned*>(flags + 2);
    auto* out = reinterpret_cast<int64_t*>(flags + 3);
    wait_check_kernel<<<1, 32, 0, s>>>(flags, publish, 7, int(polls), st, out);
    GT_LAUNCH_CHECK();
    unsigned h_st = 0;
    GT_CUDA(cudaMemcpyAsync(&h_st, st, 4, cudaMemcpyDeviceToHost, s));
    GT_CUDA(cudaMemcpyAsync(prefix, out, 8, cudaMemcpyDeviceToHost, s));
    GT_CUDA(cudaStreamSynchronize(s));
    if (h_st & gt::ST_TIMEOUT) gt::fail(GT_ETIMEOUT, "look-back wait gave up (as asked)");
  });
}

GT_API gt_status gt_set_param(gt_ctx* ctx, const char* name, int64_t value) {
  if (!ctx || !name) return GT_EINVAL;
  static const char* known[] = {"wc_aggregate", "use_graphs", "file_strategy", "wc_slices", "bu_local", "seq_path",
                                "seq_table_cap", "radix_items", "radix_prefetch"};
  if (std::strcmp(name, "radix_items") == 0 && value != 8 && value != 16) {
    ctx->last_error = "radix_items must be 8 or 16";
    return GT_EINVAL;
  }
  for (const char* k : known)
    if (std::strcmp(k, name) == 0) {
      ctx->params[name] = value;
      return GT_OK;
    }
  ctx->last_error = std::string("unknown parameter: ") + name;
  return GT_ENOTFOUND;
}

// ============================================================================
// plans: a batch captured once as a CUDA graph and replayed
// ============================================================================

struct gt_plan {
  gt_ctx* ctx = nullptr;
  std::vector<gt_query> q;
  std::vector<gt_result*> res;  // results of the captured batch, rewritten by every launch
  cudaGraphExec_t exec = nullptr;
  long long kernels = 0;         // kernels one launch runs
  int64_t launches = 0;
};

GT_API gt_status gt_plan_create(gt_ctx* ctx, const gt_query* q, int nq, void* stream, gt_plan** out) {
  if (!ctx || !q || nq < 1 || !out) return GT_EINVAL;
  *out = nullptr;
  gt_plan* p = new (std::nothrow) gt_plan();
  if (!p) return GT_ENOMEM;
  p->ctx = ctx;
  p->q.assign(q, q + nq);
  p->res.assign(size_t(nq), nullptr);
  gt_status st = guard(ctx, [&] {
    use_device(ctx);
    if (ctx->prof_on) fail(GT_EINVAL, "plans cannot be captured while profiling is enabled");
    // one eager run: validates the queries and builds any per-grammar state
    // that the first call of an analytic creates
    std::vector<gt_result*> warm(size_t(nq), nullptr);
    const gt_status w = gt_run_batch(ctx, q, nq, stream, warm.data());
    if (w != GT_OK) fail(w, ctx->last_error);
    GT_CUDA(cudaStreamSynchronize(as_stream(stream)));
    for (gt_result* r : warm)
      if (r) gt_free_result(r);
    cudaStream_t cs;
    GT_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    const long long l0 = gt::g_launches.load();
    gt_status rc = GT_OK;
    std::string msg;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      rc = gt_run_batch(ctx, q, nq, cs, p->res.data());
      msg = ctx->last_error;
      const cudaError_t e = cudaStreamEndCapture(cs, &graph);
      if (rc == GT_OK && (e != cudaSuccess || !graph)) {
        rc = GT_ECUDA;
        msg = std::string("stream capture failed: ") + cudaGetErrorString(e);
      }
    } else {
      rc = GT_ECUDA;
      msg = "stream capture could not begin";
    }
    p->kernels = gt::g_launches.load() - l0;
    gt::g_launches.fetch_sub(p->kernels);  // the captured launches did not run
    if (rc == GT_OK) {
      // a launch frees the allocations of the previous one: results are
      // valid until the next launch of the plan
      const cudaError_t e = cudaGraphInstantiate(&p->exec, graph, cudaGraphInstantiateFlagAutoFreeOnLaunch);
      if (e != cudaSuccess) {
        rc = GT_ECUDA;
        msg = std::string("graph instantiation failed: ") + cudaGetErrorString(e);
      }
    }
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    cudaGetLastError();
    if (rc != GT_OK) fail(rc, msg);
  });
  if (st != GT_OK) {
    for (gt_result* r : p->res)  // captured results hold no memory yet: release the host parts only
      if (r) {
        p->ctx->give_back(r->h_lens, r->done);
        delete r;
      }
    delete p;
    return st;
  }
  *out = p;
  return GT_OK;
}

GT_API gt_status gt_plan_launch(gt_plan* p, void* stream) {
  if (!p) return GT_EINVAL;
  return guard(p->ctx, [&] {
    use_device(p->ctx);
    for (gt_result* r : p->res)
      if (r) r->ready = false;  // lengths are read again after this launch
    GT_CUDA(cudaGraphLaunch(p->exec, as_stream(stream)));
    // a record made during capture only orders the captured work: the
    // completion of each result is recorded here, after the replay
    for (gt_result* r : p->res)
      if (r) GT_CUDA(cudaEventRecord(r->done, as_stream(stream)));
    gt::g_launches.fetch_add(p->kernels);
    ++p->launches;
  });
}

GT_API gt_status gt_plan_result(gt_plan* p, int i, const char* field, const void** d_ptr, int64_t* len) {
  if (!p || i < 0 || i >= int(p->res.size()) || !field || !d_ptr || !len) return GT_EINVAL;
  if (!p->res[size_t(i)]) return GT_ENOTFOUND;  // a word count writes into the caller's buffer
  if (p->launches == 0) return GT_EBUSY;       // nothing computed yet
  return gt_result_view(p->res[size_t(i)], field, d_ptr, len);
}

GT_API gt_status gt_plan_destroy(gt_plan* p) {
  if (!p) return GT_EINVAL;
  cudaSetDevice(p->ctx->device);
  cudaDeviceSynchronize();
  for (gt_result* r : p->res) {
    if (!r) continue;
    if (p->launches > 0)  // the last launch's allocations are still live
      for (void* x : r->owned) cudaFreeAsync(x, nullptr);
    p->ctx->give_back(r->h_lens, r->done);
    delete r;
  }
  if (p->exec) cudaGraphExecDestroy(p->exec);
  delete p;
  return GT_OK;
}
