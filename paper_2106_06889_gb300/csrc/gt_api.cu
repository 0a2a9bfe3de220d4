// The gt_* C ABI: contexts, grammar load, result objects and the host-side
// orchestration of each analytic.  Every step of every analytic runs in this
// library's CUDA kernels; there is no CPU path.
#include <algorithm>
#include <cstring>
#include <new>

#include "gt_device.cuh"

using gt::Buf;
using gt::fail;

namespace gt {
std::atomic<long long> g_launches{0};
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

void use_device(gt_ctx* ctx) { GT_CUDA(cudaSetDevice(ctx->device)); }

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

// ---- result construction ----------------------------------------------------

// A result under construction: buffers are allocated from the pool on the
// query's stream; data-dependent lengths are written by kernels into a small
// device array and copied to pinned host memory when the query ends.
struct ResultBuilder {
  gt_result* r;
  cudaStream_t s;
  int64_t* d_lens = nullptr;  // device slots for data-dependent lengths; slot 0 holds the status word
  int nslots = 0;
  static constexpr int kMaxSlots = 8;

  ResultBuilder(gt_ctx* ctx, cudaStream_t st) : s(st) {
    r = new gt_result();
    r->ctx = ctx;
    GT_CUDA(cudaMallocHost(&r->h_lens, kMaxSlots * sizeof(int64_t)));
    void* p = nullptr;
    GT_CUDA(cudaMallocFromPoolAsync(&p, kMaxSlots * sizeof(int64_t), ctx->pool, s));
    r->owned.push_back(p);
    d_lens = static_cast<int64_t*>(p);
    GT_CUDA(cudaMemsetAsync(d_lens, 0, kMaxSlots * sizeof(int64_t), s));
    nslots = 1;
  }
  uint32_t* status() { return reinterpret_cast<uint32_t*>(d_lens); }
  int64_t* new_len_slot() {
    if (nslots >= kMaxSlots) fail(GT_EINVAL, "too many result fields");
    return d_lens + nslots++;
  }
  void* alloc(size_t bytes) {
    void* p = nullptr;
    GT_CUDA(cudaMallocFromPoolAsync(&p, bytes ? bytes : 16, r->ctx->pool, s));
    r->owned.push_back(p);
    return p;
  }
  void field(const char* name, void* ptr, int64_t len) { r->fields.push_back({name, ptr, len, nullptr}); }
  void field_dyn(const char* name, void* ptr, int64_t* d_len_slot) {
    const int64_t idx = d_len_slot - d_lens;
    r->fields.push_back({name, ptr, -1, r->h_lens + idx});
  }
  gt_result* finish() {
    GT_CUDA(cudaMemcpyAsync(r->h_lens, d_lens, kMaxSlots * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    GT_CUDA(cudaEventCreateWithFlags(&r->done, cudaEventDisableTiming));
    GT_CUDA(cudaEventRecord(r->done, s));
    gt_result* out = r;
    r = nullptr;
    return out;
  }
  ~ResultBuilder() {
    if (r) gt_free_result(r);
  }
};

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
    const cudaMemcpyKind kind = desc->on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
    std::vector<int64_t> roff(size_t(R) + 1), foff(size_t(F) + 1);
    GT_CUDA(cudaMemcpy(roff.data(), desc->rule_off, roff.size() * 8, kind));
    GT_CUDA(cudaMemcpy(foff.data(), desc->file_off, foff.size() * 8, kind));
    if (roff[0] != 0) fail(GT_EINVAL, "rule_off[0] must be 0");
    for (int32_t r = 0; r < R; ++r) {
      if (roff[r + 1] < roff[r]) fail(GT_EINVAL, "rule_off must be non-decreasing");
      if (r > 0 && roff[r + 1] == roff[r]) fail(GT_EINVAL, "every non-root rule body must be non-empty");
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
    // symbols padded to whole tiles with -1 (never a word, never a rule)
    const int64_t Gp = std::max<int64_t>((G + gt::kTile - 1) / gt::kTile, 1) * gt::kTile;
    void* p;
    GT_CUDA(cudaMalloc(&p, size_t(Gp) * 4));
    g->owned.push_back(p);
    GT_CUDA(cudaMemsetAsync(p, 0xff, size_t(Gp) * 4, s));
    if (G > 0)
      GT_CUDA(cudaMemcpyAsync(p, desc->sym, size_t(G) * 4,
                              desc->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    d.sym = static_cast<int32_t*>(p);
    GT_CUDA(cudaMalloc(&p, roff.size() * 8));
    g->owned.push_back(p);
    GT_CUDA(cudaMemcpyAsync(p, roff.data(), roff.size() * 8, cudaMemcpyHostToDevice, s));
    d.rule_off = static_cast<int64_t*>(p);
    GT_CUDA(cudaMalloc(&p, foff.size() * 8));
    g->owned.push_back(p);
    GT_CUDA(cudaMemcpyAsync(p, foff.data(), foff.size() * 8, cudaMemcpyHostToDevice, s));
    d.file_off = static_cast<int64_t*>(p);
    g->info.device_bytes = Gp * 4 + int64_t(roff.size() + foff.size()) * 8;
    gt::load_build_dag(g, s);
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
  for (void* p : g->owned) cudaFree(p);
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

GT_API gt_status gt_word_count(gt_grammar* g, uint64_t* d_counts, void* stream) {
  if (!g || !d_counts) return GT_EINVAL;
  return guard(g->ctx, [&] {
    use_device(g->ctx);
    cudaStream_t s = as_stream(stream);
    Buf wt(g->ctx, size_t(g->d.R) * 8, s);
    gt::run_rule_weights(g, wt.as<uint64_t>(), s);
    gt::run_word_count(g, wt.as<uint64_t>(), d_counts, s);
  });
}

GT_API gt_status gt_head_tail(gt_grammar* g, int32_t* d_head, int32_t* d_tail, void* stream) {
  if (!g || !d_head || !d_tail) return GT_EINVAL;
  return guard(g->ctx, [&] {
    use_device(g->ctx);
    gt::run_head_tail(g, d_head, d_tail, as_stream(stream));
  });
}

GT_API gt_status gt_sort(gt_grammar* g, int order, void* stream, gt_result** out) {
  if (!g || !out || (order != 0 && order != 1)) return GT_EINVAL;
  *out = nullptr;
  return guard(g->ctx, [&] {
    gt_ctx* ctx = g->ctx;
    use_device(ctx);
    cudaStream_t s = as_stream(stream);
    const int64_t V = g->d.V;
    const int threads = 256, cap = ctx->num_sms * 8;
    ResultBuilder rb(ctx, s);
    auto* words = static_cast<int32_t*>(rb.alloc(size_t(V) * 4));
    auto* counts = static_cast<uint64_t*>(rb.alloc(size_t(V) * 8));
    int64_t* nlen = rb.new_len_slot();
    Buf wc(ctx, size_t(V) * 8, s);
    {
      Buf wt(ctx, size_t(g->d.R) * 8, s);
      gt::run_rule_weights(g, wt.as<uint64_t>(), s);
      gt::run_word_count(g, wt.as<uint64_t>(), wc.as<uint64_t>(), s);
    }
    gt::Phase ph(ctx, "sort_canon", s);
    if (order == 0) {
      Buf flag(ctx, size_t(V) * 8, s), pos(ctx, size_t(V) * 8, s), sc(ctx, gt::scan_scratch_bytes(V), s);
      nonzero_flags_kernel<<<gt::grid_for(V, threads, cap), threads, 0, s>>>(wc.as<uint64_t>(), V, flag.as<int64_t>());
      GT_LAUNCH_CHECK();
      gt::exclusive_scan_i64(flag.as<int64_t>(), pos.as<int64_t>(), V, sc.p, s);
      compact_words_kernel<<<gt::grid_for(V, threads, cap), threads, 0, s>>>(wc.as<uint64_t>(), V, pos.as<int64_t>(),
                                                                              words, counts, nlen);
      GT_LAUNCH_CHECK();
    } else {
      const uint64_t N = g->d.N;
      Buf k0(ctx, size_t(V) * 8, s), k1(ctx, size_t(V) * 8, s), v0(ctx, size_t(V) * 4, s), v1(ctx, size_t(V) * 4, s);
      Buf rs(ctx, gt::radix_scratch_bytes(V, true, 4), s);
      count_keys_kernel<<<gt::grid_for(V, threads, cap), threads, 0, s>>>(wc.as<uint64_t>(), V, N, k0.as<uint64_t>(),
                                                                          v0.as<uint32_t>());
      GT_LAUNCH_CHECK();
      gt::radix_sort_u64(k0.as<uint64_t>(), k1.as<uint64_t>(), v0.p, v1.p, 4, V, 0, bits_for(N), rs.p, s);
      count_unkey_kernel<<<gt::grid_for(V, threads, cap), threads, 0, s>>>(k1.as<uint64_t>(), v1.as<uint32_t>(), V, N,
                                                                           words, counts, nlen);
      GT_LAUNCH_CHECK();
    }
    rb.field_dyn("word", words, nlen);
    rb.field_dyn("count", counts, nlen);
    GT_CUDA(cudaMemcpyAsync(rb.status(), ctx->d_status, 4, cudaMemcpyDeviceToDevice, s));
    *out = rb.finish();
  });
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
  if (r->done) {
    cudaEventSynchronize(r->done);
    cudaEventDestroy(r->done);
  }
  for (void* p : r->owned) cudaFreeAsync(p, nullptr);
  if (r->h_lens) cudaFreeHost(r->h_lens);
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

GT_API gt_status gt_set_param(gt_ctx* ctx, const char* name, int64_t value) {
  if (!ctx || !name) return GT_EINVAL;
  static const char* known[] = {"wc_aggregate"};
  for (const char* k : known)
    if (std::strcmp(k, name) == 0) {
      ctx->params[name] = value;
      return GT_OK;
    }
  ctx->last_error = std::string("unknown parameter: ") + name;
  return GT_ENOTFOUND;
}
