// Serving loop: continuous batching of analytics requests over grammars kept
// resident on the device (not in the paper, which runs one query at a time).
//
// A worker thread owns `slots` CUDA streams.  Requests wait in a FIFO queue.
// Whenever a slot is free it admits waiting requests in arrival order while
// their estimated footprints fit the memory budget (the first one that does
// not fit stops admission until memory is released: no overtaking), groups
// the admitted queries by grammar so that analytics on the same grammar share
// one traversal (gt_run_batch's sharing), and launches each group on a free
// slot.  Groups in flight overlap on the
// device.  Completion is observed with events; the slot and the memory are
// released and the next arrivals are admitted right away.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <thread>
#include <unordered_map>

#include "gt_device.cuh"

extern "C" gt_status gt_run_batch(gt_ctx* ctx, const gt_query* q, int nq, void* stream, gt_result** out);

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t ticket = 0;
  std::vector<gt_query> q;
  std::vector<gt_result*> out;
  size_t footprint = 0;
  Clock::time_point submitted, finished;
  gt_status status = GT_OK;
  bool done = false;
};

struct Group {
  std::vector<Request*> reqs;
  int slot = -1;
  cudaEvent_t ev = nullptr;
  size_t footprint = 0;
};

}  // namespace

struct gt_server {
  gt_ctx* ctx = nullptr;
  int nslots = 0;
  size_t budget = 0;
  std::vector<cudaStream_t> streams;
  std::vector<bool> busy;
  std::mutex mu;
  std::condition_variable cv;       // wakes the worker
  std::condition_variable done_cv;  // wakes pollers
  std::deque<Request*> waiting;
  std::unordered_map<uint64_t, Request*> all;
  std::vector<Group> inflight;
  size_t in_use = 0;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::thread worker;
  int64_t admitted_rounds = 0, max_inflight = 0;
};

namespace gt {

// Upper estimate of the device scratch one query needs (bytes).
size_t query_footprint(const gt_grammar* g, int kind) {
  const DevGrammar& d = g->d;
  const double Gp = double((d.G + kTile - 1) / kTile + 1) * kTile;
  const double R = d.R, V = d.V, F = d.F, N = double(d.N);
  const double nb = std::ceil(V / 16384.0);
  double b = 0;
  if (file_strategy(g) == 2 && kind >= GT_Q_INVERTED_INDEX) {  // bottom-up rows: keys, sort, reduce
    const double rows = std::max(double(d.root_len + g->bu_words), 2.0 * double(d.root_len) + double(g->bu_windows));
    return size_t(128 * rows + 24 * V) + (size_t(64) << 20);
  }
  switch (kind) {
    case GT_Q_WORD_COUNT:
    case GT_Q_SORT:
      b = 20 * Gp + 16 * R + 64 * V + 4.0 * g->ctx->num_sms * nb * 16384 * 3;
      break;
    case GT_Q_INVERTED_INDEX:
    case GT_Q_TERM_VECTOR:
    case GT_Q_TFIDF:
      b = 8 * F * nb * 16384 + 2400 * F * nb + 64 * double(g->fentry_bound) + 40 * double(g->fword_bound) +
          2 * double(d.root_len) + 40 * R + 24 * std::min(N, F * nb * 16384) + 16 * V;
      break;
    case GT_Q_COOCCURRENCE:  // the 3-word count, then two rows per distinct 3-gram sorted again
      b = 2 * (160 * Gp + 32 * R);
      break;
    default:
      b = 160 * Gp + 32 * R;
  }
  return size_t(b) + (size_t(64) << 20);
}

}  // namespace gt

namespace {

void worker_loop(gt_server* sv) {
  cudaSetDevice(sv->ctx->device);
  std::unique_lock<std::mutex> lk(sv->mu);
  while (true) {
    // ---- retire finished groups ----
    for (size_t i = 0; i < sv->inflight.size();) {
      Group& gr = sv->inflight[i];
      // anything but "not ready" ends the group: a failed query (a sticky
      // context error included) must not stay in flight forever
      const cudaError_t q = cudaEventQuery(gr.ev);
      if (q != cudaErrorNotReady) {
        const auto now = Clock::now();
        for (Request* r : gr.reqs) {
          r->finished = now;
          r->done = true;
          if (q != cudaSuccess && r->status == GT_OK) r->status = GT_ECUDA;
        }
        sv->busy[gr.slot] = false;
        sv->in_use -= gr.footprint;
        sv->ctx->give_back(nullptr, gr.ev);
        sv->inflight.erase(sv->inflight.begin() + long(i));
        sv->done_cv.notify_all();
      } else {
        ++i;
      }
    }
    if (sv->stop && sv->waiting.empty() && sv->inflight.empty()) break;
    // ---- admit: free slot + memory budget, arrival order ----
    std::vector<Request*> adm;
    size_t adm_mem = 0;
    int free_slots = 0;
    for (bool b : sv->busy) free_slots += !b;
    if (free_slots > 0) {
      for (auto it = sv->waiting.begin(); it != sv->waiting.end();) {
        Request* r = *it;
        if (sv->in_use + adm_mem + r->footprint <= sv->budget || (sv->inflight.empty() && adm.empty())) {
          adm.push_back(r);
          adm_mem += r->footprint;
          it = sv->waiting.erase(it);
        } else {
          break;  // keep arrival order: the first request that does not fit blocks the rest
        }
      }
    }
    if (!adm.empty()) {
      // group the admitted requests by grammar of their first query, one group
      // per free slot; the rest of the admitted requests share the last slot
      std::vector<std::vector<Request*>> groups;
      std::unordered_map<const gt_grammar*, size_t> gi;
      for (Request* r : adm) {
        const gt_grammar* key = r->q.empty() ? nullptr : r->q[0].grammar;
        auto f = gi.find(key);
        if (f == gi.end() && int(groups.size()) < free_slots) {
          gi[key] = groups.size();
          groups.push_back({r});
        } else if (f != gi.end()) {
          groups[f->second].push_back(r);
        } else {
          groups.back().push_back(r);
        }
      }
      ++sv->admitted_rounds;
      for (auto& reqs : groups) {
        int slot = 0;
        while (sv->busy[slot]) ++slot;
        Group gr;
        gr.reqs = reqs;
        gr.slot = slot;
        for (Request* r : reqs) gr.footprint += r->footprint;
        std::vector<gt_query> qs;
        for (Request* r : reqs) qs.insert(qs.end(), r->q.begin(), r->q.end());
        std::vector<gt_result*> outs(qs.size(), nullptr);
        sv->busy[slot] = true;
        sv->in_use += gr.footprint;
        lk.unlock();
        const gt_status st = gt_run_batch(sv->ctx, qs.data(), int(qs.size()), sv->streams[slot], outs.data());
        gr.ev = sv->ctx->take_event();
        if (gr.ev) cudaEventRecord(gr.ev, sv->streams[slot]);
        lk.lock();
        size_t k = 0;
        for (Request* r : reqs) {
          r->status = st;
          for (size_t j = 0; j < r->q.size(); ++j) r->out[j] = outs[k++];
        }
        if (!gr.ev) {  // could not track completion: finish synchronously
          cudaStreamSynchronize(sv->streams[slot]);
          for (Request* r : reqs) {
            r->finished = Clock::now();
            r->done = true;
            if (r->status == GT_OK) r->status = GT_ECUDA;
          }
          sv->busy[slot] = false;
          sv->in_use -= gr.footprint;
          sv->done_cv.notify_all();
        } else {
          sv->inflight.push_back(gr);
          if (int64_t(sv->inflight.size()) > sv->max_inflight) sv->max_inflight = int64_t(sv->inflight.size());
        }
      }
      continue;
    }
    if (sv->inflight.empty()) {
      sv->cv.wait(lk, [&] { return sv->stop || !sv->waiting.empty(); });
    } else {
      // poll completions: short waits keep latency low without spinning a core
      sv->cv.wait_for(lk, std::chrono::microseconds(20));
    }
  }
}

}  // namespace

GT_API gt_status gt_server_create(gt_ctx* ctx, int slots, size_t mem_budget, gt_server** out) {
  if (!ctx || !out || slots < 1 || slots > 64) return GT_EINVAL;
  *out = nullptr;
  gt_server* sv = new (std::nothrow) gt_server();
  if (!sv) return GT_ENOMEM;
  sv->ctx = ctx;
  sv->nslots = slots;
  sv->budget = mem_budget ? mem_budget : ~size_t(0);
  if (cudaSetDevice(ctx->device) != cudaSuccess) {
    delete sv;
    return GT_ECUDA;
  }
  for (int i = 0; i < slots; ++i) {
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      for (cudaStream_t x : sv->streams) cudaStreamDestroy(x);
      delete sv;
      return GT_ECUDA;
    }
    sv->streams.push_back(st);
  }
  sv->busy.assign(size_t(slots), false);
  sv->worker = std::thread(worker_loop, sv);
  *out = sv;
  return GT_OK;
}

GT_API gt_status gt_submit(gt_server* sv, const gt_query* q, int nq, uint64_t* ticket) {
  if (!sv || !q || nq < 1 || !ticket) return GT_EINVAL;
  for (int i = 0; i < nq; ++i)
    if (!q[i].grammar || q[i].grammar->ctx != sv->ctx || q[i].kind < GT_Q_WORD_COUNT || q[i].kind > GT_Q_COOCCURRENCE)
      return GT_EINVAL;
  Request* r = new (std::nothrow) Request();
  if (!r) return GT_ENOMEM;
  r->q.assign(q, q + nq);
  r->out.assign(size_t(nq), nullptr);
  for (int i = 0; i < nq; ++i) r->footprint += gt::query_footprint(q[i].grammar, q[i].kind);
  if (r->footprint > sv->budget) {
    delete r;
    return GT_EBUSY;  // can never be admitted under this budget
  }
  r->submitted = Clock::now();
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    r->ticket = sv->next_ticket++;
    sv->waiting.push_back(r);
    sv->all[r->ticket] = r;
  }
  sv->cv.notify_one();
  *ticket = r->ticket;
  return GT_OK;
}

GT_API gt_status gt_poll(gt_server* sv, uint64_t ticket, int wait, gt_result** out, int64_t* latency_ns) {
  if (!sv) return GT_EINVAL;
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->all.find(ticket);
  if (it == sv->all.end()) return GT_ENOTFOUND;
  Request* r = it->second;
  if (!r->done) {
    if (!wait) return GT_EBUSY;
    sv->done_cv.wait(lk, [&] { return r->done; });
  }
  const gt_status st = r->status;
  if (out)
    for (size_t i = 0; i < r->out.size(); ++i) out[i] = r->out[i];
  else
    for (gt_result* x : r->out)
      if (x) gt_free_result(x);
  if (latency_ns)
    *latency_ns = int64_t(std::chrono::duration_cast<std::chrono::nanoseconds>(r->finished - r->submitted).count());
  sv->all.erase(it);
  delete r;
  return st;
}

GT_API gt_status gt_server_stats(gt_server* sv, int64_t* waiting, int64_t* inflight, int64_t* max_inflight,
                                 uint64_t* mem_in_use) {
  if (!sv) return GT_EINVAL;
  std::lock_guard<std::mutex> lk(sv->mu);
  if (waiting) *waiting = int64_t(sv->waiting.size());
  if (inflight) *inflight = int64_t(sv->inflight.size());
  if (max_inflight) *max_inflight = sv->max_inflight;
  if (mem_in_use) *mem_in_use = uint64_t(sv->in_use);
  return GT_OK;
}

GT_API gt_status gt_server_destroy(gt_server* sv) {
  if (!sv) return GT_EINVAL;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv.notify_all();
  if (sv->worker.joinable()) sv->worker.join();
  cudaSetDevice(sv->ctx->device);
  for (auto& kv : sv->all) {
    for (gt_result* x : kv.second->out)
      if (x) gt_free_result(x);
    delete kv.second;
  }
  for (cudaStream_t st : sv->streams) cudaStreamDestroy(st);
  delete sv;
  return GT_OK;
}
