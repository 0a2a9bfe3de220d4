/*
 * gtadoc.h - C ABI of libgtadoc.so: text analytics run directly on
 * Sequitur grammar-compressed corpora (G-TADOC, arXiv 2106.06889) on one
 * NVIDIA GB300 GPU (sm_103a).
 *
 * Input model (Section II-A and Fig. 1 of the paper): words are dictionary-
 * converted to integer IDs; a context-free grammar of rules R0..Rn encodes
 * every file; the root R0 holds the files one after another, separated by
 * unique splitter symbols; every other rule stands for a repeated phrase.
 * Here the splitters are removed from the root body and their positions are
 * given as file offsets instead.
 *
 * Conventions shared by every call:
 *   - A `stream` argument is a cudaStream_t passed as void*; NULL means the
 *     legacy default stream.  Calls that take a stream only enqueue work on it
 *     and return without waiting for the GPU, unless stated otherwise.
 *   - Pointers named d_* are device pointers on the context's device;
 *     everything else is a host pointer.
 *   - Inputs stay owned by the caller.  The grammar is copied into library-
 *     owned device memory at load time.  Results (gt_result) are library-owned
 *     device buffers released with gt_free_result.
 *   - Every output is canonical (sorted as each call states), so equal inputs
 *     give byte-identical outputs whatever the grammar that encodes them.
 *   - Counts are exact unsigned 64-bit integers.
 *   - Errors: a call returns a gt_status; GT_OK is 0.  A human-readable
 *     message for the last failure on a context is available from
 *     gt_last_error.  Failures that only the GPU can detect (a full overflow
 *     list, a row count past its bound, an invalid symbol) are recorded in a
 *     device status word and reported by gt_sync / gt_result_view.  The
 *     only waits inside kernels are decoupled look-backs (the global
 *     sequence count's bucket path and the inverted index: a CTA polls the
 *     published totals of the items taken before its own); each gives up
 *     after a bounded number of polls with GT_ETIMEOUT.
 *   - There is no CPU fallback: if no usable sm_103a device is present,
 *     gt_create fails with GT_ECUDA.
 */
#ifndef GTADOC_H
#define GTADOC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int gt_status;
#define GT_OK 0
#define GT_EINVAL 1       /* malformed argument or grammar                      */
#define GT_ENOMEM 2       /* device or pool allocation failed                   */
#define GT_ECUDA 3        /* a CUDA runtime call failed                         */
#define GT_ETIMEOUT 4     /* a bounded device-side wait gave up (a decoupled look-back) */
#define GT_ETABLE_FULL 5  /* a device overflow list ran out of room             */
#define GT_EOVERFLOW 6    /* a size exceeds what the encoding supports          */
#define GT_EBUSY 7        /* admission refused: not enough free memory / slots  */
#define GT_ENOTFOUND 8    /* unknown result field or ticket                     */

typedef struct gt_ctx gt_ctx;
typedef struct gt_grammar gt_grammar;
typedef struct gt_result gt_result;

/* Grammar description (Section II-A).  num_rules counts the root.
 *   rule_off [num_rules+1] int64: body of rule r is sym[rule_off[r] .. rule_off[r+1]).
 *                          rule_off[0] must be 0; rule 0 is the root.
 *   sym      [rule_off[num_rules]] int32: s < num_words is a word ID,
 *                          s >= num_words references rule s - num_words (never 0).
 *   file_off [num_files+1] int64: file f is root body positions
 *                          file_off[f] .. file_off[f+1]; file_off[0] = 0 and
 *                          file_off[num_files] = root body length.
 *   on_device: 0 if the three arrays are host memory, 1 if device memory.
 * Every non-root body must be non-empty and the rule graph must be acyclic. */
typedef struct {
  int32_t num_words;
  int32_t num_rules;
  int32_t num_files;
  const int64_t* rule_off;
  const int32_t* sym;
  const int64_t* file_off;
  int32_t on_device;
} gt_grammar_desc;

/* Facts about a loaded grammar, filled by gt_grammar_info_get. */
typedef struct {
  int64_t num_words, num_rules, num_files;
  int64_t num_syms;        /* G: total body symbols                              */
  int64_t num_edges;       /* E: distinct (parent, child) rule pairs             */
  int64_t num_root_edges;  /* distinct (file, child) pairs in the root           */
  int64_t depth;           /* number of DAG levels (root = level 0)              */
  int64_t num_tokens;      /* N: length of the fully expanded corpus             */
  int64_t owned_windows;   /* sum over rules of the owned 3-word windows (Eq. 1) */
  int64_t device_bytes;    /* device memory held by the loaded grammar           */
  int64_t root_words;      /* words (not rule references) in the root body       */
  int64_t file_pairs;      /* (rule, file) pairs with a nonzero per-file weight (<= 64 files, else 0) */
  int64_t file_words;      /* sum over those pairs of the rule's own words       */
} gt_grammar_info;

/* ---- context ---------------------------------------------------------- */

/* Create a context on CUDA device `device`.  pool_bytes > 0 reserves that
 * much device memory for the stream-ordered pool that backs per-query scratch
 * and results (0 = grow on demand).  Fails with GT_ECUDA when the device is
 * absent or is not compute capability 10.3. */
gt_status gt_create(gt_ctx** ctx, int device, size_t pool_bytes);
gt_status gt_destroy(gt_ctx* ctx);
/* Message for the last failure on ctx (never NULL; "" when none, "null
 * context" when ctx is NULL). */
const char* gt_last_error(const gt_ctx* ctx);
/* Wait for `stream`, then return and clear the device status word. */
gt_status gt_sync(gt_ctx* ctx, void* stream);

/* ---- grammar ---------------------------------------------------------- */

/* Load a grammar (the initialisation phase of Section IV-A): copy it to the
 * device and build the rule DAG used by every traversal - deduplicated child
 * lists with multiplicities (the subRules of Algorithm 1), the parent lists
 * (genRuleParentsKernel, Algorithm 2), per-file root edges, the DAG levels
 * that order top-down and bottom-up passes, per-rule word/rule counts and
 * expansion lengths; for at most 64 files also the top-down per-file layout
 * (each rule's set of files and its (rule, file) slots in file-major order),
 * which depends only on the DAG.  Host arrays are read in place and uploaded
 * directly (pinned memory gives asynchronous DMA).  Synchronises `stream`
 * before returning (it validates the grammar on the device).  GT_EINVAL for a
 * malformed or cyclic grammar; GT_EOVERFLOW when num_words + num_rules >= 2^31,
 * the grammar holds 2^40 symbols or more, or one body (the root included)
 * holds 2^32 or more. */
gt_status gt_load_grammar(gt_ctx* ctx, const gt_grammar_desc* desc, void* stream, gt_grammar** out);
gt_status gt_free_grammar(gt_grammar* g);
gt_status gt_grammar_info_get(const gt_grammar* g, gt_grammar_info* info);

/* ---- analytics (Section VI: the six CompressDirect applications) ------- */

/* Top-down rule weights (Algorithm 1): d_weights[r] = number of times rule r
 * occurs in the full expansion of the corpus; d_weights[0] = 1.
 * d_weights: device uint64[num_rules], written entirely. */
gt_status gt_rule_weights(gt_grammar* g, uint64_t* d_weights, void* stream);

/* Word count (Fig. 2): d_counts[w] = occurrences of word w in all files.
 * d_counts: device uint64[num_words], written entirely.  Replayed from a CUDA
 * graph once the same buffer has been used before (see "use_graphs"). */
gt_status gt_word_count(gt_grammar* g, uint64_t* d_counts, void* stream);

/* Word counts of n grammars of one context in one fused launch sequence
 * (the batched form: one launch per DAG level covers every grammar, then one
 * partition, one histogram and one reduce launch for all of them, up to 64
 * grammars per sequence).  d_counts[i]: device uint64[num_words of gs[i]],
 * written entirely.  Same results as n calls of gt_word_count. */
gt_status gt_word_count_batch(gt_grammar* const* gs, uint64_t* const* d_counts, int n, void* stream);

/* Word count that allocates no device memory: same result as gt_word_count
 * (bit-identical counts), for callers that cannot allocate at the time of the
 * call.  The paper has no counterpart.  Its only scratch, one uint64 weight
 * per rule, is a fixed library-owned device array of 4,194,304 entries
 * (32 MiB); a grammar with more rules is rejected with GT_EOVERFLOW (use
 * gt_word_count).  The call clears d_counts and the scratch itself.
 * d_counts: device uint64[num_words], written entirely.
 * The scratch array's address is looked up on the first call on a device;
 * make that first call outside any stream capture.  Every call on a device
 * shares the one scratch array: calls that may overlap on the device
 * (different streams with no ordering between them) race and give wrong
 * counts; calls on one stream, or ordered by events, are safe.  Slower than
 * gt_word_count (global atomics instead of shared-memory histograms). */
gt_status gt_word_count_noalloc(gt_grammar* g, uint64_t* d_counts, void* stream);

/* Sort: the distinct words with their counts.  order 0: ascending word ID;
 * order 1: descending count, ties by ascending word ID.
 * Result fields: "word" int32[n], "count" uint64[n]. */
gt_status gt_sort(gt_grammar* g, int order, void* stream, gt_result** out);

/* Inverted index: for each word, the ascending list of files containing it.
 * Result fields: "offsets" int64[num_words+1], "file" int32[offsets[V]].
 * Top-down strategy (Section IV-A) for at most 64 files, bottom-up beyond
 * (see "file_strategy"). */
gt_status gt_inverted_index(gt_grammar* g, void* stream, gt_result** out);

/* Term vector: for each file, its distinct words with their in-file counts.
 * top_k == 0: all words, ascending word ID.  top_k > 0: the top_k largest
 * counts of each file, by descending count then ascending word ID.
 * Result fields: "offsets" int64[num_files+1], "word" int32[], "count" uint64[].
 * Same strategy selection as gt_inverted_index. */
gt_status gt_term_vector(gt_grammar* g, int top_k, void* stream, gt_result** out);

/* Sequence count for l = 3 (Section IV-D): every window of three consecutive
 * words inside one file (windows never cross a file boundary), keyed as
 * key = w1 << 42 | w2 << 21 | w3 (requires num_words <= 2^21).
 * per_file == 0: fields "key" uint64[n], "count" uint64[n], ascending key.
 * per_file == 1: fields "file" int32[n], "key" uint64[n], "count" uint64[n],
 *                ascending (file, key); strategy as for gt_inverted_index.
 * Each window is counted once, by the lowest rule whose body it crosses, with
 * that rule's weight; the windows a rule owns are built from its body, a
 * two-symbol look-ahead and its children's head/tail buffers. */
gt_status gt_sequence_count(gt_grammar* g, int per_file, void* stream, gt_result** out);

/* Ranked inverted index.  n == 3: keys are 3-word windows as in
 * gt_sequence_count; n == 1: keys are words.  For each key (ascending), the
 * files containing it with the in-file count, by descending count then
 * ascending file.  Fields: "offsets" int64[nkeys+1], "key" uint64[nkeys],
 * "file" int32[m], "count" uint64[m].  Strategy as for gt_inverted_index. */
gt_status gt_ranked_index(gt_grammar* g, int n, void* stream, gt_result** out);

/* TF-IDF (the Introduction lists it among the analytics that build on the
 * six of Section VI): the term vector of every file with, per entry,
 * tfidf = count * ln(F / df(word)), df(word) = the number of files holding
 * the word, F = num_files.  Fields "offsets" int64[num_files+1], "word"
 * int32[], "count" uint64[], "tfidf" float64[] (ascending word per file).
 * One traversal serves the term vector and the document frequencies;
 * strategy as for gt_inverted_index.  float64 arithmetic: ln is CUDA's
 * double-precision log (at most 1 ulp off), the quotient and the product
 * are correctly rounded. */
gt_status gt_tfidf(gt_grammar* g, void* stream, gt_result** out);

/* Word co-occurrence within a window of three words: every ordered pair of
 * words (a, b) with b one or two positions after a inside one file, counted.
 * Fields "key" uint64[n] = a << 21 | b (ascending), "count" uint64[n]
 * (requires num_words <= 2^21).  Derived from the 3-word counts of
 * gt_sequence_count: the (first, second) and (first, third) pairs of every
 * window, plus the last pair of every file. */
gt_status gt_cooccurrence(gt_grammar* g, void* stream, gt_result** out);

/* Head and tail buffers (Section IV-C): for every rule, the first two and
 * the last two words of its expansion (word IDs; -1 pads a rule whose
 * expansion has a single word).  d_head, d_tail: device int32[2*num_rules]. */
gt_status gt_head_tail(gt_grammar* g, int32_t* d_head, int32_t* d_tail, void* stream);

/* ---- batches ------------------------------------------------------------
 * Several analytics over one or more grammars in one call.  Queries on the
 * same grammar share one traversal: word count and sort share the rule
 * weights and the counts; term vectors and the inverted index share the
 * per-file weights and (file, word) histograms, and a word count of a grammar
 * that also has such queries is summed from the per-file counts (top-down).
 * The word counts of different grammars run as one fused launch sequence (as
 * gt_word_count_batch).  out[i] receives query i's result (NULL for a word
 * count, which writes into its d_counts).  On failure no result is returned.
 * (Not in the paper: it serves one query at a time.) */
typedef enum {
  GT_Q_WORD_COUNT = 0,     /* d_counts: device uint64[num_words]                */
  GT_Q_SORT = 1,           /* param: order (0 or 1)                             */
  GT_Q_INVERTED_INDEX = 2,
  GT_Q_TERM_VECTOR = 3,    /* param: top_k (0 = all)                            */
  GT_Q_SEQUENCE_COUNT = 4, /* param: per_file (0 or 1)                          */
  GT_Q_RANKED_INDEX = 5,   /* param: n (1 or 3)                                 */
  GT_Q_TFIDF = 6,          /* shares the term vector's traversal                */
  GT_Q_COOCCURRENCE = 7
} gt_query_kind;

typedef struct {
  gt_grammar* grammar;
  int32_t kind;       /* gt_query_kind */
  int32_t param;
  uint64_t* d_counts; /* word count only */
} gt_query;

gt_status gt_run_batch(gt_ctx* ctx, const gt_query* q, int nq, void* stream, gt_result** out);

/* Plans (the batched form as one launch; not in the paper).  gt_plan_create
 * runs the batch once on `stream` (and waits for it), then captures the same
 * batch - every launch, scratch allocation and result copy - into a CUDA
 * graph.  gt_plan_launch replays that graph on a stream: one graph launch per
 * step.  Each launch rewrites the plan's results in place; gt_plan_result
 * gives query i's field (as gt_result_view, waiting for the launch) and is
 * valid until the next launch; GT_EBUSY before the first launch, GT_ENOTFOUND
 * for a word count (it writes into its d_counts, rewritten by every launch).
 * The queries' grammars and word-count buffers must stay valid while the plan
 * exists.  Launches of one plan must be ordered (one stream, or events).
 * GT_EINVAL while profiling is enabled. */
typedef struct gt_plan gt_plan;
gt_status gt_plan_create(gt_ctx* ctx, const gt_query* q, int nq, void* stream, gt_plan** out);
gt_status gt_plan_launch(gt_plan* p, void* stream);
gt_status gt_plan_result(gt_plan* p, int i, const char* field, const void** d_ptr, int64_t* len);
gt_status gt_plan_destroy(gt_plan* p);

/* ---- serving (not in the paper) ------------------------------------------
 * A server keeps the context's grammars resident and runs submitted requests
 * (each a list of gt_query, like one gt_run_batch call) with continuous
 * batching: a worker thread owns `slots` CUDA streams; whenever a slot is free
 * it admits waiting requests in arrival order while their estimated device
 * footprint fits `mem_budget` bytes (0 = unlimited), groups the admitted
 * queries by grammar so that they share one traversal, and launches each
 * group on a free stream, so that groups overlap on the device.  Results of a
 * request are the same as those of gt_run_batch on the same queries.  The
 * budget covers requests in flight; a completed request's results belong to
 * the caller and stay allocated, outside the budget, until they are polled
 * and freed, so a caller that submits much faster than it collects can still
 * exhaust device memory.
 *   gt_submit: enqueue; *ticket identifies the request.  GT_EBUSY if the
 *     request's footprint alone exceeds the budget.  Word-count buffers must
 *     stay valid until the request completes.
 *   gt_poll: wait != 0 blocks until the request completes; otherwise
 *     GT_EBUSY while it runs.  On completion, out (room for the request's nq
 *     results, or NULL to discard them) receives the results, *latency_ns the
 *     time from submission to completion, and the ticket is released; the
 *     return value is the request's status.
 *   gt_server_destroy: finishes every submitted request, then frees the
 *     results nobody polled.
 * Profiling (gt_profile_enable) must be off while a server runs. */
typedef struct gt_server gt_server;
gt_status gt_server_create(gt_ctx* ctx, int slots, size_t mem_budget, gt_server** out);
gt_status gt_submit(gt_server* sv, const gt_query* q, int nq, uint64_t* ticket);
gt_status gt_poll(gt_server* sv, uint64_t ticket, int wait, gt_result** out, int64_t* latency_ns);
gt_status gt_server_stats(gt_server* sv, int64_t* waiting, int64_t* inflight, int64_t* max_inflight,
                          uint64_t* mem_in_use);
gt_status gt_server_destroy(gt_server* sv);

/* ---- results ---------------------------------------------------------- */

/* Device pointer and element count of one field of a result.  Waits for the
 * work that produced the result; returns the device status if that work
 * failed (e.g. GT_ETABLE_FULL) and GT_ENOTFOUND for an unknown field. */
gt_status gt_result_view(gt_result* r, const char* field, const void** d_ptr, int64_t* len);
gt_status gt_free_result(gt_result* r);

/* ---- profiling (not in the paper; the paper reports phase times only) ----
 * When enabled, the library records CUDA events on the caller's stream around
 * each phase it runs ("weights", "wc_partition", "wc_hist", "file_weights",
 * "expand_words", "tv_hist", "chunk_sort_root", "chunk_sort_rules",
 * "tv_hist_kernel", "tv_out", "ii_out", "wc_from_files",
 * "seq_emit", "seq_sort", "seq_reduce", "bu_local", "bu_rows", "ranked", ...).
 * gt_profile_read waits for those events and returns, for one phase, the
 * summed device time in ms, the number of timed spans, and the number of
 * kernels launched inside them.  gt_kernel_launches returns how many kernels
 * this process has launched through the library so far. */
gt_status gt_profile_enable(gt_ctx* ctx, int on);
gt_status gt_profile_reset(gt_ctx* ctx);
gt_status gt_profile_read(gt_ctx* ctx, const char* phase, double* total_ms, int64_t* spans, int64_t* launches);
int64_t gt_kernel_launches(void);

/* Self-check of the bounded waits (the decoupled look-backs of the global
 * sequence count's bucket path and of the inverted index): one warp plays an
 * item whose predecessor either publishes its prefix (publish != 0: returns
 * GT_OK, *prefix = 7) or never does (publish == 0: the wait gives up after
 * `polls` polls, 1..2^24, and the call returns GT_ETIMEOUT with *prefix = -1;
 * the context stays usable).  No kernel faults or hangs either way. */
gt_status gt_check_bounded_wait(gt_ctx* ctx, int publish, int64_t polls, int64_t* prefix);

/* Tunable parameters (Section IV-A, parameter selection: results never depend
 * on them, only speed does).  Known names:
 *   "wc_aggregate"  1: merge equal words inside a warp (__match_any_sync)
 *                   before the shared-memory histogram update; 0 (default):
 *                   update per lane.
 *   "use_graphs"    1 (default): word counts (gt_word_count, and word-count
 *                   queries of gt_run_batch / the server) capture a grammar's
 *                   launch sequence into a CUDA graph on the second call that
 *                   writes into a given output buffer, and replay it from then
 *                   on (that call should happen outside any stream capture);
 *                   not while profiling is enabled.  0: launch kernel by kernel.
 *   "wc_slices"     histogram CTAs per 16k-word bucket in the word count
 *                   (1..64); 0 (default): about 3 x SMs / buckets.
 *   "bu_local"      1 (default): bottom-up word rows of grammars whose files
 *                   all have at most 8192 tokens are built per file in shared
 *                   memory; 0: always by the global (file, word) sort.
 *   "seq_path"      global sequence count: 1 (default) one row per owned window,
 *                   LSD radix sort by key, segmented sum; 2 sample-sort
 *                   buckets reduced in shared memory (gt_seqg.cu).  Same
 *                   results; bench.py times both.
 *   "seq_table_cap" distinct keys a bucket may hold in shared memory on the
 *                   bucket path (2..3072, default 3072); fuller buckets are
 *                   sorted in global memory.
 *   "radix_items"   keys per thread of the LSD radix sort's scatter passes:
 *                   8 (default, tiles of 2048 keys) or 16 (tiles of 4096:
 *                   longer runs per digit in each tile's writes); GT_EINVAL
 *                   otherwise.  Same results.
 *   "radix_prefetch" 1: the radix sort's scatter passes (2048-key tiles) run
 *                   as a persistent kernel that copies the next tile into
 *                   shared memory asynchronously while it ranks the current
 *                   one; 0 (default): one CTA per tile.  Same results.
 *   "file_strategy" per-file analytics (term vector, inverted index, per-file
 *                   sequence count, ranked index): 0 (default) picks top-down
 *                   for at most 64 files and bottom-up otherwise (the paper's
 *                   strategy selection, Section V-C); 1 forces top-down, 2
 *                   forces bottom-up.
 * GT_ENOTFOUND for an unknown name. */
gt_status gt_set_param(gt_ctx* ctx, const char* name, int64_t value);

/* Autotuner (the schedule choice of the batched form, Section V-C's
 * top-down/bottom-up selection made by measurement).  Times, on g itself,
 * the candidates of the analytics in `kinds` (a bit mask of 1 << gt_query_kind):
 *   word count / sort: "wc_aggregate" in {0, 1} x "wc_slices" in {k/2, k, 2k}
 *                      (k = the default number of histogram CTAs per bucket);
 *   per-file kinds:    "file_strategy" top-down (when F <= 64) vs bottom-up,
 *                      timed on a term vector + inverted index batch.
 * Each candidate runs once untimed, then `reps` times (1..1000) on `stream`;
 * the median device time decides.  The choices are stored on g and take
 * precedence over gt_set_param values for every later call on g (direct,
 * gt_run_batch, server).  kinds = 0 clears g's choices.  Synchronises the
 * device; must not run while other work on g is in flight.  A candidate that
 * runs out of memory is skipped.  `out` (may be null) receives the choices
 * and the best median times (ms; 0 for analytics not tuned). */
typedef struct {
  int32_t wc_aggregate;
  int32_t wc_slices;
  int32_t file_strategy; /* 1 top-down, 2 bottom-up; 0 if not tuned */
  int32_t candidates;    /* configurations timed */
  double wc_ms;          /* best word-count time */
  double file_ms;        /* best per-file batch time */
} gt_tune_result;
gt_status gt_autotune(gt_grammar* g, uint32_t kinds, int reps, void* stream, gt_tune_result* out);

#ifdef __cplusplus
}
#endif
#endif /* GTADOC_H */
