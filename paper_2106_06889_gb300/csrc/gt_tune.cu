// Autotuner: per grammar, time the candidate launch configurations of the
// word count and the per-file analytics on the grammar itself and keep the
// fastest (the schedule choice of the batched form; the paper fixes its
// parameters by hand and picks top-down or bottom-up by the number of files,
// Section V-C).
//
// Tuned: "wc_aggregate" (warp-merged or per-lane histogram updates),
// "wc_slices" (histogram CTAs per 16k-word bucket) and "file_strategy"
// (top-down or bottom-up per-file traversal).  Choices are stored on the
// grammar and override the context's gt_set_param values for it; every later
// call on the grammar (direct, gt_run_batch, the server) uses them.
#include <algorithm>
#include <vector>

#include "gt_device.cuh"

namespace gt {

int64_t gparam(const gt_grammar* g, const char* name, int64_t dflt) {
  {
    std::lock_guard<std::mutex> lk(g->tune_mu);
    auto it = g->tuned.find(name);
    if (it != g->tuned.end()) return it->second;
  }
  return g->ctx->param(name, dflt);
}

}  // namespace gt

namespace {

void set_tuned(gt_grammar* g, const char* name, int64_t v) {
  std::lock_guard<std::mutex> lk(g->tune_mu);
  g->tuned[name] = v;
}

// Captured word-count graphs bake in launch shapes: drop them when a shape
// parameter changes (the caller has synchronised the device).
void drop_graphs(gt_grammar* g) {
  std::lock_guard<std::mutex> lk(g->graph_mu);
  for (auto& e : g->wc_graphs)
    if (e.exec) cudaGraphExecDestroy(e.exec);
  g->wc_graphs.clear();
}

// Median device time (ms) of `reps` runs of fn on stream s, after one
// untimed run; +inf if a run fails (e.g. out of memory for that candidate).
// cleanup() runs after each run, outside the timed region.
template <class Fn, class Cleanup>
double time_median(cudaStream_t s, int reps, Fn&& fn, Cleanup&& cleanup) {
  cudaEvent_t a = nullptr, b = nullptr;
  GT_CUDA(cudaEventCreate(&a));
  if (cudaEventCreate(&b) != cudaSuccess) {
    cudaEventDestroy(a);
    gt::fail(GT_ECUDA, "event creation failed");
  }
  std::vector<double> t;
  bool ok = true;
  try {
    fn();
    GT_CUDA(cudaStreamSynchronize(s));
    cleanup();
    for (int r = 0; r < reps; ++r) {
      GT_CUDA(cudaEventRecord(a, s));
      fn();
      GT_CUDA(cudaEventRecord(b, s));
      GT_CUDA(cudaEventSynchronize(b));
      cleanup();
      float ms = 0;
      GT_CUDA(cudaEventElapsedTime(&ms, a, b));
      t.push_back(ms);
    }
  } catch (const gt::Error& e) {
    cudaStreamSynchronize(s);
    cleanup();
    if (e.code != GT_ENOMEM && e.code != GT_EOVERFLOW) {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
      throw;
    }
    cudaGetLastError();
    ok = false;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (!ok || t.empty()) return 1e30;
  std::sort(t.begin(), t.end());
  return t[t.size() / 2];
}

}  // namespace

GT_API gt_status gt_autotune(gt_grammar* g, uint32_t kinds, int reps, void* stream, gt_tune_result* out) {
  if (!g || reps < 1 || reps > 1000) return GT_EINVAL;
  gt_ctx* ctx = g->ctx;
  try {
    GT_CUDA(cudaSetDevice(ctx->device));
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    GT_CUDA(cudaStreamSynchronize(s));
    GT_CUDA(cudaDeviceSynchronize());
    drop_graphs(g);
    {
      std::lock_guard<std::mutex> lk(g->tune_mu);
      g->tuned.clear();
    }
    gt_tune_result res{};
    const gt::DevGrammar& d = g->d;
    if (kinds & ((1u << GT_Q_WORD_COUNT) | (1u << GT_Q_SORT))) {
      const int nb = int((int64_t(d.V) + 16383) / 16384);
      const int kd = std::max(1, (3 * ctx->num_sms + nb - 1) / nb);
      std::vector<int> ks{std::max(1, kd / 2), kd, std::min(64, 2 * kd)};
      ks.erase(std::unique(ks.begin(), ks.end()), ks.end());
      gt::Buf counts(ctx, size_t(d.V) * 8 + 8, s);
      double best = 1e30;
      int best_agg = 0, best_k = kd;
      for (int agg = 0; agg < 2; ++agg)
        for (int k : ks) {
          set_tuned(g, "wc_aggregate", agg);
          set_tuned(g, "wc_slices", k);
          const double ms = time_median(
              s, reps,
              [&] {
                gt::Buf wt(ctx, size_t(d.R) * 8, s);
                gt::run_rule_weights(g, wt.as<uint64_t>(), s);
                gt::run_word_count(g, wt.as<uint64_t>(), counts.as<uint64_t>(), s);
              },
              [] {});
          ++res.candidates;
          if (ms < best) {
            best = ms;
            best_agg = agg;
            best_k = k;
          }
        }
      set_tuned(g, "wc_aggregate", best_agg);
      set_tuned(g, "wc_slices", best_k);
      res.wc_aggregate = best_agg;
      res.wc_slices = best_k;
      res.wc_ms = best < 1e29 ? best : -1.0;
    }
    const uint32_t per_file = (1u << GT_Q_INVERTED_INDEX) | (1u << GT_Q_TERM_VECTOR) |
                              (1u << GT_Q_SEQUENCE_COUNT) | (1u << GT_Q_RANKED_INDEX);
    if ((kinds & per_file) && d.F > 0) {
      double best = 1e30;
      int best_st = d.F <= 64 ? 1 : 2;
      for (int st = 1; st <= 2; ++st) {
        if (st == 1 && d.F > 64) continue;  // top-down file masks hold 64 files
        set_tuned(g, "file_strategy", st);
        gt_result* tv = nullptr;
        gt_result* ii = nullptr;
        const double ms = time_median(
            s, reps,
            [&] {
              const int topk = 0;
              gt::run_file_batch(g, &topk, 1, &tv, &ii, s);
            },
            [&] {
              if (tv) gt_free_result(tv);
              if (ii) gt_free_result(ii);
              tv = ii = nullptr;
            });
        ++res.candidates;
        if (ms < best) {
          best = ms;
          best_st = st;
        }
      }
      set_tuned(g, "file_strategy", best_st);
      res.file_strategy = best_st;
      res.file_ms = best < 1e29 ? best : -1.0;
    }
    GT_CUDA(cudaStreamSynchronize(s));
    if (out) *out = res;
    ctx->last_error.clear();
    return GT_OK;
  } catch (const gt::Error& e) {
    ctx->last_error = e.msg;
    return e.code;
  } catch (const std::bad_alloc&) {
    ctx->last_error = "host allocation failed";
    return GT_ENOMEM;
  } catch (...) {
    ctx->last_error = "unexpected failure";
    return GT_ECUDA;
  }
}
