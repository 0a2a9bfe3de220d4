// Internal definitions shared by the translation units of libgtadoc.so.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "gtadoc.h"

#define GT_API extern "C" __attribute__((visibility("default")))

namespace gt {

struct Error {
  gt_status code;
  std::string msg;
};

[[noreturn]] inline void fail(gt_status code, std::string msg) { throw Error{code, std::move(msg)}; }

#define GT_CUDA(call)                                                                          \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess)                                                                     \
      ::gt::fail(e_ == cudaErrorMemoryAllocation ? GT_ENOMEM : GT_ECUDA,                       \
                 std::string(#call) + ": " + cudaGetErrorString(e_));                         \
  } while (0)

// Every kernel launch site is followed by this check; it also counts launches.
#define GT_LAUNCH_CHECK()                                            \
  do {                                                               \
    ::gt::g_launches.fetch_add(1, std::memory_order_relaxed);        \
    GT_CUDA(cudaGetLastError());                                     \
  } while (0)

extern std::atomic<long long> g_launches;

// Bits of the device status word.
enum : uint32_t {
  ST_TABLE_FULL = 1u,
  ST_TIMEOUT = 2u,
  ST_OVERFLOW = 4u,
  ST_INVALID = 8u,
};

constexpr int kTile = 2048;  // symbols per streaming tile (512 threads x int4)

// Device-resident grammar and the DAG built from it at load time.  All
// arrays are library-owned device memory.
struct DevGrammar {
  int32_t V, R, F;
  int64_t G;         // total body symbols
  int64_t root_len;  // symbols in the root body (the root body is sym[0, root_len))
  int64_t ntiles;    // ceil(G / kTile)
  const int32_t* sym;       // [G]
  const int64_t* rule_off;  // [R+1]
  const int64_t* file_off;  // [F+1], positions inside the root body
  const int32_t* tile_rule; // [ntiles+1]: rule holding the first symbol of each tile
  // rule of every symbol, from the tile holding the root's end onwards (the
  // root's own symbols there read 0); symbol i maps to sym_rule[i - first_rule_tile * kTile]
  int64_t first_rule_tile;
  const int32_t* sym_rule;
  // child lists (Algorithm 1's subRules): distinct (child, multiplicity) per rule
  int64_t E;
  const int64_t* cedge_off;  // [R+1]
  const int32_t* cedge_child;
  const uint32_t* cedge_mult;
  // parent lists (Algorithm 2's parentIds), multiplicity of the child in the parent
  const int64_t* pedge_off;  // [R+1]
  const int32_t* pedge_par;
  const uint32_t* pedge_mult;
  // parent edges grouped by the level of the child, children ascending within a
  // level: the top-down weight pass reads level l's slice
  const int32_t* ledge_child;
  const int32_t* ledge_par;
  const uint32_t* ledge_mult;
  // root edges per file: distinct (file, child, multiplicity)
  int64_t ER;
  const int64_t* redge_off;  // [F+1]
  const int32_t* redge_child;
  const uint32_t* redge_mult;
  // DAG levels: level(r) = longest path from a source; parents have lower levels
  int32_t depth;
  const int32_t* level;      // [R]
  const int32_t* lvl_order;  // [R] rules sorted by level
  // per-rule facts
  const int32_t* nwords;   // [R] W_r: words in the body
  const int32_t* nrefs;    // [R] S_r: rule references in the body
  const uint64_t* exp_len; // [R] L_r: words in the expansion
  const uint64_t* file_len;// [F] words in each file's expansion
  uint64_t N;              // tokens in the expanded corpus
};

}  // namespace gt

// ---- host-side objects behind the opaque C handles -------------------------

struct gt_ctx {
  int device = 0;
  int num_sms = 0;
  cudaMemPool_t pool = nullptr;
  uint32_t* d_status = nullptr;  // device status word (ST_* bits)
  std::string last_error;
  // phase timing: CUDA events recorded around each phase's launches
  bool prof_on = false;
  struct Span {
    cudaEvent_t a, b;
    int launches;
  };
  std::map<std::string, std::vector<Span>> prof;
  // tunable parameters (Section IV-A, parameter selection); see gt_set_param
  std::map<std::string, int64_t> params;
  int64_t param(const char* name, int64_t dflt) const {
    auto it = params.find(name);
    return it == params.end() ? dflt : it->second;
  }
};

struct gt_grammar {
  gt_ctx* ctx = nullptr;
  gt::DevGrammar d{};
  gt_grammar_info info{};
  std::vector<int64_t> lvl_off;  // host copy: rules of level l are lvl_order[lvl_off[l] .. lvl_off[l+1])
  std::vector<int64_t> ledge_off; // host copy: parent edges of level-l children are ledge_*[ledge_off[l] ..)
  std::vector<void*> owned;      // device allocations to free with the grammar
};

struct gt_result {
  gt_ctx* ctx = nullptr;
  struct Field {
    std::string name;
    void* ptr;
    int64_t len;        // valid once `ready` is set
    int64_t* len_src;   // pinned host slot receiving the length, or null if len is fixed
  };
  std::vector<Field> fields;
  std::vector<void*> owned;  // device buffers to release
  int64_t* h_lens = nullptr; // pinned host array holding data-dependent lengths
  cudaEvent_t done = nullptr;
  bool ready = false;
};

namespace gt {

// Stream-ordered device buffer from the context pool, released on the same
// stream when it goes out of scope (safe: later work on the stream is
// ordered after every kernel that used it).
struct Buf {
  void* p = nullptr;
  cudaStream_t s = nullptr;
  Buf() = default;
  Buf(gt_ctx* ctx, size_t bytes, cudaStream_t st) : s(st) {
    if (bytes == 0) bytes = 16;
    GT_CUDA(cudaMallocFromPoolAsync(&p, bytes, ctx->pool, st));
  }
  Buf(const Buf&) = delete;
  Buf& operator=(const Buf&) = delete;
  Buf(Buf&& o) noexcept : p(o.p), s(o.s) { o.p = nullptr; }
  Buf& operator=(Buf&& o) noexcept {
    release();
    p = o.p;
    s = o.s;
    o.p = nullptr;
    return *this;
  }
  ~Buf() { release(); }
  void release() {
    if (p) cudaFreeAsync(p, s);
    p = nullptr;
  }
  void* detach() {
    void* q = p;
    p = nullptr;
    return q;
  }
  template <class T>
  T* as() const {
    return static_cast<T*>(p);
  }
};

// Records CUDA events on `s` around a phase when profiling is on.
struct Phase {
  gt_ctx* ctx;
  const char* name;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  long long l0 = 0;
  Phase(gt_ctx* c, const char* n, cudaStream_t st) : ctx(c), name(n), s(st) {
    if (!ctx->prof_on) return;
    GT_CUDA(cudaEventCreate(&a));
    GT_CUDA(cudaEventRecord(a, s));
    l0 = g_launches.load();
  }
  ~Phase() {
    if (!a) return;
    cudaEvent_t b;
    if (cudaEventCreate(&b) != cudaSuccess) return;
    cudaEventRecord(b, s);
    ctx->prof[name].push_back({a, b, int(g_launches.load() - l0)});
  }
};

inline int grid_for(int64_t n, int threads, int cap) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return int(b);
}

// ---- launchers implemented in the kernel translation units -----------------

// gt_load.cu
void load_build_dag(gt_grammar* g, cudaStream_t s);

// gt_wc.cu
void run_rule_weights(gt_grammar* g, uint64_t* d_wt, cudaStream_t s);
void run_word_count(gt_grammar* g, const uint64_t* d_wt, uint64_t* d_counts, cudaStream_t s);
void run_head_tail(gt_grammar* g, int32_t* d_head, int32_t* d_tail, cudaStream_t s);

// gt_sort.cu: device primitives
size_t scan_scratch_bytes(int64_t n);
void exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, void* scratch, cudaStream_t s);
size_t radix_scratch_bytes(int64_t n, bool with_values, int value_bytes);
// Stable LSD radix sort of n uint64 keys on bits [begin_bit, end_bit); values
// (optional, value_bytes 4 or 8) move with their keys.  Results land in
// keys_out / vals_out.  keys_in / vals_in are clobbered.
void radix_sort_u64(uint64_t* keys_in, uint64_t* keys_out, void* vals_in, void* vals_out, int value_bytes,
                    int64_t n, int begin_bit, int end_bit, void* scratch, cudaStream_t s);

}  // namespace gt
