// Word count that allocates no device memory (gt_word_count_noalloc).
//
// For callers that cannot allocate device memory at the time of the call: no
// cudaMalloc/cudaFree, no stream-ordered pool allocation and no allocating
// library routine runs here.  The only scratch the computation needs is the
// top-down rule weights (one uint64 per rule, Algorithm 1); they live in a
// file-scope __device__ array of fixed size instead of pool memory, so the
// grammar may have at most kNoAllocMaxRules rules.
//
// The steps are the same top-down traversal as gt_word_count - weights level
// by level, then every word occurrence of a rule body adds the rule's weight -
// but with one plain global atomic per edge and per occurrence instead of the
// partition / shared-memory histogram pipeline, whose buffers scale with the
// grammar and would have to be allocated.
//
// The scratch array is shared by every call on a device: calls whose work may
// overlap on the device (different streams without ordering between them)
// race on it and give wrong counts.  Calls on one stream, or ordered by events,
// are safe.
#include <mutex>

#include "gt_device.cuh"

namespace {

constexpr int64_t kNoAllocMaxRules = int64_t(1) << 22;  // 4,194,304 rules: 32 MiB of weights
constexpr int kNoAllocMaxDevices = 64;

// Starts at zero by the language rules, but the first R entries are cleared by
// every call anyway (a previous call leaves its weights behind).
__device__ __align__(256) unsigned long long g_noalloc_wt[kNoAllocMaxRules];

std::mutex g_noalloc_mu;
unsigned long long* g_noalloc_ptr[kNoAllocMaxDevices] = {};

// Address of the scratch array on the current device (looked up once per
// device; the lookup may load the module, so make the first call on a device
// outside any stream capture).
unsigned long long* noalloc_scratch(int device) {
  if (device < 0 || device >= kNoAllocMaxDevices) gt::fail(GT_EINVAL, "device index out of range");
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_wt);
    if (e != cudaSuccess || !p)
      gt::fail(GT_ECUDA, std::string("cudaGetSymbolAddress(weights scratch): ") + cudaGetErrorString(e));
    g_noalloc_ptr[device] = static_cast<unsigned long long*>(p);
  }
  return g_noalloc_ptr[device];
}

__global__ void noalloc_root_kernel(unsigned long long* __restrict__ wt) { wt[0] = 1ull; }

// One level of children: wt[child] += mult * wt[parent]; parents lie on lower
// levels, finished by the previous launches.
__global__ void noalloc_weights_kernel(const int32_t* __restrict__ lchild, const int32_t* __restrict__ lpar,
                                       const uint32_t* __restrict__ lmult, int64_t a, int64_t b,
                                       unsigned long long* __restrict__ wt) {
  for (int64_t i = a + blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < b; i += int64_t(gridDim.x) * blockDim.x)
    atomicAdd(&wt[lchild[i]], (unsigned long long)lmult[i] * wt[lpar[i]]);
}

// Every word symbol of every body adds the weight of the rule holding it (the
// root's weight is 1).
__global__ void noalloc_count_kernel(const gt::DevGrammar d, const unsigned long long* __restrict__ wt,
                                     unsigned long long* __restrict__ counts) {
  for (int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; j < d.G; j += int64_t(gridDim.x) * blockDim.x) {
    const int32_t s = d.sym[j];
    if (s >= d.V) continue;
    const int64_t r = gt::upper_bound_dev(d.rule_off, int64_t(d.R) + 1, j) - 1;
    const unsigned long long w = wt[r];
    if (w) atomicAdd(&counts[s], w);
  }
}

}  // namespace

GT_API gt_status gt_word_count_noalloc(gt_grammar* g, uint64_t* d_counts, void* stream) {
  if (!g || !d_counts) return GT_EINVAL;
  gt_ctx* ctx = g->ctx;
  try {
    const gt::DevGrammar& d = g->d;
    if (int64_t(d.R) > kNoAllocMaxRules)
      gt::fail(GT_EOVERFLOW, "gt_word_count_noalloc holds the weights of at most 4194304 rules; this grammar has " +
                                 std::to_string(d.R) + " (use gt_word_count)");
    GT_CUDA(cudaSetDevice(ctx->device));
    unsigned long long* wt = noalloc_scratch(ctx->device);
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int threads = 256, cap = ctx->num_sms * 16;
    // both the output and the weights accumulate with atomics: clear them
    GT_CUDA(cudaMemsetAsync(d_counts, 0, size_t(d.V) * 8, s));
    GT_CUDA(cudaMemsetAsync(wt, 0, size_t(d.R) * 8, s));
    noalloc_root_kernel<<<1, 1, 0, s>>>(wt);
    GT_LAUNCH_CHECK();
    for (int lv = 1; lv < d.depth; ++lv) {
      const int64_t a = g->ledge_off[lv], b = g->ledge_off[lv + 1];
      if (b <= a) continue;
      noalloc_weights_kernel<<<gt::grid_for(b - a, threads, cap), threads, 0, s>>>(d.ledge_child, d.ledge_par,
                                                                                   d.ledge_mult, a, b, wt);
      GT_LAUNCH_CHECK();
    }
    if (d.G > 0) {
      noalloc_count_kernel<<<gt::grid_for(d.G, threads, cap), threads, 0, s>>>(
          d, wt, reinterpret_cast<unsigned long long*>(d_counts));
      GT_LAUNCH_CHECK();
    }
    ctx->last_error.clear();
    return GT_OK;
  } catch (const gt::Error& e) {
    ctx->last_error = e.msg;
    return e.code;
  } catch (...) {
    ctx->last_error = "unexpected failure";
    return GT_ECUDA;
  }
}
