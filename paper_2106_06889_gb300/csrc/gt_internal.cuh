// Internal definitions shared by the translation units of libgtadoc.so.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <mutex>
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

// The context of the API call running on this thread (set on entry), for
// phase timers in primitives that take no context.
extern thread_local gt_ctx* t_call_ctx;

// Bits of the device status word.
enum : uint32_t {
  ST_TABLE_FULL = 1u,
  ST_TIMEOUT = 2u,
  ST_OVERFLOW = 4u,
  ST_INVALID = 8u,
};

constexpr int kTile = 2048;        // symbols per streaming tile (512 threads x int4)
constexpr int kFileChunk = 8192;   // items of a root chunk's window (per-file analytics)
// root symbols per file-pure chunk: the chunk's 16-byte-aligned window (it
// may start up to 3 symbols early) fits kFileChunk
constexpr int kRootChunk = kFileChunk - 4;

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
  // the root edges child-major: files referencing each rule from the root
  const int64_t* rfile_off;  // [R+1]
  const int32_t* rfile_f;
  const uint32_t* rfile_m;
  // DAG levels: level(r) = longest path from a source; parents have lower levels
  int32_t depth;
  const int32_t* level;      // [R]
  const int32_t* lvl_order;  // [R] rules sorted by level
  // per-rule facts
  const int32_t* nwords;   // [R] W_r: words in the body
  const int32_t* nrefs;    // [R] S_r: rule references in the body
  const uint64_t* exp_len; // [R] L_r: words in the expansion
  const uint64_t* file_len;// [F] words in each file's expansion
  // the root cut into chunks of at most kFileChunk symbols that never cross a
  // file: chunk c = [rch_start[c], + rch_len[c]); file f's are [rch_foff[f], rch_foff[f+1])
  const int64_t* rch_start;
  const int32_t* rch_len;
  const int64_t* rch_foff;
  const int64_t* rch_count;
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
  // recycled pinned length blocks and events of released results
  std::mutex res_mu;
  std::vector<int64_t*> free_lens;
  std::vector<cudaEvent_t> free_events;
  std::vector<void*> pinned_chunks;
  int64_t* take_lens(int slots) {
    std::lock_guard<std::mutex> lk(res_mu);
    if (free_lens.empty()) {
      const int per = 256;
      void* p = nullptr;
      if (cudaMallocHost(&p, size_t(per) * slots * sizeof(int64_t)) != cudaSuccess) return nullptr;
      pinned_chunks.push_back(p);
      for (int i = 0; i < per; ++i) free_lens.push_back(static_cast<int64_t*>(p) + size_t(i) * slots);
    }
    int64_t* q = free_lens.back();
    free_lens.pop_back();
    return q;
  }
  cudaEvent_t take_event() {
    std::lock_guard<std::mutex> lk(res_mu);
    if (free_events.empty()) {
      cudaEvent_t e = nullptr;
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return nullptr;
      return e;
    }
    cudaEvent_t e = free_events.back();
    free_events.pop_back();
    return e;
  }
  void give_back(int64_t* lens, cudaEvent_t e) {
    std::lock_guard<std::mutex> lk(res_mu);
    if (lens) free_lens.push_back(lens);
    if (e) free_events.push_back(e);
  }
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
  int64_t root_chunks = 0;        // host copy of *rch_count
  int64_t fentry_bound = 0;       // (rule, file) pairs with a nonzero per-file weight (<= 64 files)
  int64_t fword_bound = 0;        // rule words emitted once per such pair
  int64_t fsym_bound = 0;         // rule body symbols visited once per such pair
  // top-down per-file layout (<= 64 files), built at load: the set of files
  // holding each rule (64-bit mask) and each rule's first (rule, file) slot;
  // slots are laid out level by level (rules in level order, files ascending),
  // light rules (few parents) first: level l's light slots are
  // [lvl_slot[l], lvl_slot[l+1]), its heavy ones [lvl_heavy[l], lvl_heavy[l+1])
  const unsigned long long* fmask = nullptr;
  const int64_t* foff = nullptr;
  const int64_t* fnnz = nullptr;
  std::vector<int64_t> lvl_slot;
  std::vector<int64_t> lvl_heavy;
  int64_t light_slots = 0;
  // per-file weights of a query are kept in pair order (file-major):
  // slot_pair[slot] = its pair, root_pairs[pair] = the root's references.
  // Slot i's row row_entries[row_off[i], row_off[i+1]) lists (parent's pair,
  // mult) over the rule's non-root parents holding the slot's file; heavy
  // rows are cut into pieces (pair, first entry, end entry), level l's
  // [lvl_piece[l], lvl_piece[l+1])
  const uint32_t* slot_pair = nullptr;
  const uint32_t* root_pairs = nullptr;
  const uint32_t* row_off = nullptr;
  const uint2* row_entries = nullptr;
  int64_t row_entries_n = 0;
  const uint4* row_pieces = nullptr;
  int64_t row_pieces_n = 0;
  std::vector<int64_t> lvl_piece;
  // the rule words (file-major) cut into chunks of at most 4096 words inside
  // each file: chunk c = words [xch_start[c], + xch_len[c]), overlapped by the
  // pairs [xch_p0[c], xch_p1[c]); file f's chunks are [xch_foff[f], xch_foff[f+1])
  int64_t rule_chunks = 0;  // host copy of *xch_count
  // the rule words of each file sorted by 16k-word bucket per rule-word chunk:
  // entry = (pair - chunk's first pair) << 14 | index in bucket, runs per (chunk, bucket)
  const uint32_t* xent = nullptr;
  const int64_t* xrun_start = nullptr;
  const int32_t* xrun_len = nullptr;
  const int64_t* xch_start = nullptr;
  const int32_t* xch_len = nullptr;
  const int64_t* xch_foff = nullptr;
  const int64_t* xch_count = nullptr;
  const int64_t* xch_p0 = nullptr;
  const int64_t* xch_p1 = nullptr;
  const int32_t* file_order = nullptr;  // files by length, longest first
  int64_t bu_words = 0;           // sum over distinct (file, root child) pairs of the child's length
  int64_t bu_windows = 0;         // ... and of the child's 3-word windows
  int64_t max_file_len = 0;       // tokens of the longest file
  // owned 3-word windows of every tile of symbols, exclusive scan [ntiles + 1]:
  // structure only (no weights), built by the first global sequence count
  // and kept; seq_tile_ev marks its completion for other streams
  const int64_t* seq_tile_off = nullptr;
  cudaEvent_t seq_tile_ev = nullptr;
  std::mutex seq_mu;
  std::vector<void*> owned;      // device allocations to free with the grammar
  // word-count launch sequences captured as CUDA graphs, keyed by output
  // buffer; at most kMaxWcGraphs per grammar, the least recently used evicted
  struct WcGraph {
    uint64_t* out;
    cudaGraphExec_t exec;  // null until the second call with this buffer
    uint64_t last_use;     // value of graph_tick at the last call
    int kernels;           // kernels one replay launches
  };
  static constexpr size_t kMaxWcGraphs = 8;
  std::vector<WcGraph> wc_graphs;
  uint64_t graph_tick = 0;
  std::mutex graph_mu;
  // per-grammar parameter choices of gt_autotune; they take precedence over
  // the context's gt_set_param values
  std::map<std::string, int64_t> tuned;
  mutable std::mutex tune_mu;
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
  int64_t* d_lens = nullptr; // their device copies (slot 0: status word), written by the kernels
  std::vector<gt_result*> deps;  // results whose buffers this one reads; freed with it
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
    if (!ctx || !ctx->prof_on) return;
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
    r->h_lens = ctx->take_lens(kMaxSlots);
    if (!r->h_lens) fail(GT_ENOMEM, "pinned host allocation failed");
    void* p = nullptr;
    GT_CUDA(cudaMallocFromPoolAsync(&p, kMaxSlots * sizeof(int64_t), ctx->pool, s));
    r->owned.push_back(p);
    d_lens = static_cast<int64_t*>(p);
    r->d_lens = d_lens;
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
    r->done = r->ctx->take_event();
    if (!r->done) fail(GT_ECUDA, "event creation failed");
    GT_CUDA(cudaEventRecord(r->done, s));
    gt_result* out = r;
    r = nullptr;
    return out;
  }
  ~ResultBuilder() {
    if (r) gt_free_result(r);
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
// off[h] = first index of the sorted keys whose high 32 bits are >= h, h in [0, nh]
void csr_offsets_hi(const uint64_t* keys, int64_t n, int64_t nh, int64_t* off, cudaStream_t s);

// gt_wc.cu
void run_rule_weights(gt_grammar* g, uint64_t* d_wt, cudaStream_t s);
// Device-detected failures of a word count (ST_* bits) go to *status, or to
// the context's status word (read by gt_sync) when status is null.
void run_word_count(gt_grammar* g, const uint64_t* d_wt, uint64_t* d_counts, cudaStream_t s,
                    uint32_t* status = nullptr);
// word counts of up to 64 grammars (one context) in one fused launch sequence
void run_word_count_multi(gt_grammar* const* gs, uint64_t* const* counts, int n, cudaStream_t s,
                          uint32_t* status = nullptr);
void run_head_tail(gt_grammar* g, int32_t* d_head, int32_t* d_tail, cudaStream_t s);

// Sorted 3-word window rows: compact keys (kb bits per word, key_pad above
// every real key), optional file keys, weights; n rows including pads.
struct Windows {
  Buf keys, fkeys, vals;
  int64_t n = 0;
  int kb = 1;
  uint64_t key_pad = 0;
  // already one row per distinct (file, key): keys[0, *total) with rfile
  // (int32) and rcnt (uint64) instead of fkeys / vals
  bool reduced = false;
  Buf rfile, rcnt, total;
};

// per-file strategy: 1 top-down (file masks, <= 64 files), 2 bottom-up
// (expansion of each distinct (file, root child) pair); "file_strategy" 0 = auto
int file_strategy(const gt_grammar* g);

// gt_seq.cu
void sort_by_file_key(gt_ctx* ctx, Buf& k0, Buf& f0, Buf& v0, int64_t bound, int key_bits, int file_bits,
                      cudaStream_t s, Windows& out);

// gt_bu.cu: bottom-up per-file rows
void bu_window_rows(gt_grammar* g, Buf& head, Buf& tail, int kb, uint64_t key_pad, cudaStream_t s, Windows& out);
void run_file_batch_bu(gt_grammar* g, const int* tv_topk, int n_tv, gt_result** tv_out, gt_result** ii_out,
                       cudaStream_t s);
gt_result* run_ranked_words_bu(gt_grammar* g, cudaStream_t s);
// A device allocation that lives as long as the grammar: taken from the
// context's stream-ordered pool (which keeps freed memory for reuse, so
// loading and freeing grammars does not go back to the driver).
inline void* grammar_alloc(gt_grammar* g, size_t bytes, cudaStream_t s) {
  void* p = nullptr;
  GT_CUDA(cudaMallocFromPoolAsync(&p, bytes ? bytes : 16, g->ctx->pool, s));
  g->owned.push_back(p);
  g->info.device_bytes += int64_t(bytes);
  return p;
}

// gt_tune.cu: a parameter of this grammar (autotuned value, else the context's)
int64_t gparam(const gt_grammar* g, const char* name, int64_t dflt);
// gt_file.cu: term-vector result from (word, count) rows in (file, word) order
// top_k == kTfIdf: the term vector with a "tfidf" field (float64) instead of top-k selection
constexpr int kTfIdf = -1;
gt_result* tv_from_arrays(gt_ctx* ctx, const int32_t* word, const uint64_t* cnt, const int64_t* tv_off_in,
                          const int64_t* total, int64_t bound, int32_t F, int top_k, cudaStream_t s,
                          int32_t V = 0);
// Device pointer of a result field and the device slot holding its length
// (valid on the result's stream before the result completes).
void result_device_field(gt_result* r, const char* field, void** ptr, const int64_t** d_len);

// gt_seq.cu: sequence count (l = 3) and ranked inverted index
gt_result* run_sequence_count(gt_grammar* g, int per_file, cudaStream_t s);
// gt_adv.cu: TF-IDF (term vector with idf weights) and word co-occurrence
gt_result* run_tfidf(gt_grammar* g, cudaStream_t s);
gt_result* run_cooccurrence(gt_grammar* g, cudaStream_t s);
// gt_seq.cu: rows (key, weight) -> one row per distinct key with the weights
// summed, ascending key; n rows (host bound), rows past *n_dev hold key_pad
gt_result* reduce_key_rows(gt_ctx* ctx, Buf& keys, Buf& vals, int64_t n, int key_bits, uint64_t key_pad,
                           cudaStream_t s, const uint32_t* status_in = nullptr);
// gt_seqg.cu: the global count (per_file == 0) by sample-sort buckets
gt_result* run_sequence_count_global(gt_grammar* g, cudaStream_t s);
// owned windows of every tile of kTile symbols, exclusive scan [ntiles + 1]:
// structure, built by the first call and kept with the grammar (outside
// stream capture; GT_EINVAL if the first call is captured)
const int64_t* seq_tile_offsets(gt_grammar* g, const int32_t* head, const int32_t* tail, int kb, cudaStream_t s);
gt_result* run_ranked_windows(gt_grammar* g, cudaStream_t s);
// rows (key, file, count) -> ranked index; keys are compact 3-word keys
// (windows = true, kb bits per word) or word ids (windows = false)
gt_result* ranked_from_rows(gt_ctx* ctx, Buf& rkey, Buf& rfile, Buf& rcnt, const int64_t* n_dev, int64_t bound,
                            int kb, bool windows, uint64_t key_pad, uint64_t max_count, cudaStream_t s);
// gt_file.cu: ranked index over words (rows from the term vector)
gt_result* run_ranked_words(gt_grammar* g, cudaStream_t s);

// gt_file.cu: per-file analytics (top-down strategy, up to 64 files)
gt_result* run_term_vector(gt_grammar* g, int top_k, cudaStream_t s);
// Top-down per-file weights (<= 64 files): rule r's files are the set bits of
// mask[r]; its weight in its k-th file (ascending) is w[slot_pair[off[r] + k]]
// (weights are kept in file-major pair order).
struct FileWeights {
  const unsigned long long* mask = nullptr;  // [R] files holding each rule (the grammar's, from load)
  const int64_t* off = nullptr;              // [R] first (rule, file) slot of each rule (from load)
  const int64_t* nnz = nullptr;              // number of (rule, file) pairs (from load)
  const uint32_t* slot_pair = nullptr;       // [pairs] the pair of each slot (from load)
  Buf w;                                     // uint32 [pairs]: per-file weights of this query, by pair
};
void file_weights(gt_grammar* g, cudaStream_t s, FileWeights& fw);
// at load: exact sizes of the per-file buffers (<= 64 files)
void file_sizes(gt_grammar* g, cudaStream_t s);
// One shared traversal for several per-file queries on one grammar: n_tv term
// vectors (top_k each) and, if ii_out is set, the inverted index.
// Term vectors / inverted index of one grammar from one traversal.  With
// wc_out (top-down strategy only) the word counts are written too, as the sum
// of the per-file counts; returns whether they were.
bool run_file_batch(gt_grammar* g, const int* tv_topk, int n_tv, gt_result** tv_out, gt_result** ii_out,
                    cudaStream_t s, uint64_t* wc_out = nullptr);
gt_result* run_inverted_index(gt_grammar* g, cudaStream_t s);

// gt_sort.cu: device primitives
size_t scan_scratch_bytes(int64_t n);
void exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, void* scratch, cudaStream_t s);
size_t radix_scratch_bytes(int64_t n, bool with_values, int value_bytes);
// Stable LSD radix sort of n uint64 keys on bits [begin_bit, end_bit); values
// (optional, value_bytes 4 or 8) move with their keys.  Results land in
// keys_out / vals_out.  keys_in / vals_in are clobbered.
void radix_sort_u64(uint64_t* keys_in, uint64_t* keys_out, void* vals_in, void* vals_out, int value_bytes,
                    int64_t n, int begin_bit, int end_bit, void* scratch, cudaStream_t s);
// The same on bits [begin_a, end_a) then [begin_b, end_b) (keys whose other
// bits are all equal, e.g. hi << 32 | lo with narrow hi and lo).
void radix_sort_u64_split(uint64_t* keys_in, uint64_t* keys_out, void* vals_in, void* vals_out, int value_bytes,
                          int64_t n, int begin_a, int end_a, int begin_b, int end_b, void* scratch, cudaStream_t s);

}  // namespace gt
