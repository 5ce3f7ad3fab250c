// Serving loop of lrep.h: continuous batching of concurrent BOSP solves.
//
//  * Admission: when a slot is free, the queued request with the smallest
//    device footprint (the solver workspace, plus the bf16 operator split
//    in mixed mode) that fits the HBM budget next to the solves already
//    running starts; a request that has been passed over kMaxOvertakes
//    times goes first once it fits (nothing starves), and while it does not
//    fit nothing overtakes it.  Slots free up as solves finish, so requests
//    that arrive while others run are admitted as soon as they fit, and a
//    large request waiting for memory does not hold up small ones behind
//    it.
//  * Overlap: every slot is a host thread with its own CUDA stream; the
//    solve of an admitted request runs on its slot's stream, so the work of
//    concurrent requests overlaps on the device.
//  * Shared launches: the small projected problems (eq. small_eigen) of
//    order < 40 of all running solves meet at a rendezvous and are solved by
//    one batched launch, one CTA per request; larger ones run in their
//    multi-CTA form on the requester's stream (concurrent requests fill the
//    GPU).  Neither form's arithmetic depends on the batch, so a request's
//    result is the same alone, in a mix, or through a direct lrep_solve.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/lrep.h"
#include "problem.h"

using namespace lrep;

namespace {

constexpr int kMaxBatch = 16;
constexpr int kMaxOvertakes = 64;  // admissions a queued request lets pass

// Rendezvous of the small LREPs of concurrently running solves.
struct Batcher : SmallBatcher {
  std::mutex mu;
  std::condition_variable cv;
  cudaStream_t bstream = nullptr;
  int running = 0;  // solves in progress (maintained by the server)
  struct Waiter {
    SmallJob job;
    cudaStream_t st;
    cudaEvent_t ready;
    bool finished = false;
    cudaError_t err = cudaSuccess;
  };
  std::vector<Waiter*> waiting;
  SmallJob* dev_jobs = nullptr;  // device copy of one batch (leader-owned)
  std::mutex launch_mu;
  int64_t batches = 0, jobs_total = 0, max_batch = 0;

  cudaError_t init() {
    cudaError_t e = cudaStreamCreateWithFlags(&bstream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&dev_jobs, sizeof(SmallJob) * kMaxBatch);
    return e;
  }
  ~Batcher() {
    if (dev_jobs) cudaFree(dev_jobs);
    if (bstream) cudaStreamDestroy(bstream);
  }

  cudaError_t launch(std::vector<Waiter*>& batch) {
    std::lock_guard<std::mutex> g(launch_mu);
    cudaError_t e = cudaSuccess;
    for (Waiter* w : batch)
      if (e == cudaSuccess) e = cudaStreamWaitEvent(bstream, w->ready, 0);
    for (size_t b0 = 0; b0 < batch.size() && e == cudaSuccess; b0 += kMaxBatch) {
      SmallJob h[kMaxBatch];
      const int nb = (int)std::min<size_t>(kMaxBatch, batch.size() - b0);
      for (int i = 0; i < nb; ++i) h[i] = batch[b0 + i]->job;
      e = cudaMemcpyAsync(dev_jobs, h, sizeof(SmallJob) * nb, cudaMemcpyHostToDevice, bstream);
      if (e == cudaSuccess) e = small_lrep_batched(dev_jobs, nb, bstream);
      // the pageable copy above completes before the call returns, but the
      // device array is reused by the next launch: order it on bstream
    }
    cudaEvent_t done;
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&done, cudaEventDisableTiming);
    if (e == cudaSuccess) {
      e = cudaEventRecord(done, bstream);
      for (Waiter* w : batch)
        if (e == cudaSuccess) e = cudaStreamWaitEvent(w->st, done, 0);
      cudaEventDestroy(done);
    }
    batches++;
    jobs_total += (int64_t)batch.size();
    max_batch = std::max<int64_t>(max_batch, (int64_t)batch.size());
    return e;
  }

  cudaError_t run(const SmallJob& job, cudaStream_t st) override {
    // orders that the grid-wide form serves better are not batched: they
    // run on the requester's stream, with the arithmetic of a direct solve
    if (job.d >= small_wide_min()) return small_lrep_one(job, st);
    Waiter me;
    me.job = job;
    me.st = st;
    cudaError_t e = cudaEventCreateWithFlags(&me.ready, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
    e = cudaEventRecord(me.ready, st);
    if (e != cudaSuccess) {
      cudaEventDestroy(me.ready);
      return e;
    }
    std::unique_lock<std::mutex> lk(mu);
    waiting.push_back(&me);
    cv.notify_all();
    if (waiting.size() == 1) {
      // leader: wait briefly for the other running solves to arrive
      cv.wait_for(lk, std::chrono::microseconds(300),
                  [&] { return (int)waiting.size() >= running; });
      std::vector<Waiter*> batch;
      batch.swap(waiting);
      lk.unlock();
      const cudaError_t le = launch(batch);
      lk.lock();
      for (Waiter* w : batch) {
        w->err = le;
        w->finished = true;
      }
      cv.notify_all();
    } else {
      cv.wait(lk, [&] { return me.finished; });
    }
    lk.unlock();
    cudaEventDestroy(me.ready);
    return me.err;
  }
};

struct Req {
  uint64_t ticket;
  lrep_problem p;
  int nev, block;
  double tol;
  size_t footprint;
  int overtaken = 0;  // later arrivals admitted before this one
};

}  // namespace

struct lrep_server_s {
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Req> queue;
  std::map<uint64_t, lrep_status> done;
  uint64_t next = 1;
  bool stop = false;
  int64_t budget = 0;
  int64_t in_use = 0;
  int max_slots = 1;
  int idle = 0;
  int device = 0;
  std::vector<std::thread> workers;
  Batcher batcher;

  bool fits(const Req& r) const { return (int64_t)r.footprint + in_use <= budget; }

  // index in the queue of the request to start now, or -1: the oldest
  // request passed over kMaxOvertakes times if any (when it fits), else the
  // smallest footprint that fits (ties: arrival order)
  int pick() const {
    if (queue.empty() || idle <= 0) return -1;
    for (size_t i = 0; i < queue.size(); ++i)
      if (queue[i].overtaken >= kMaxOvertakes) return fits(queue[i]) ? (int)i : -1;
    int best = -1;
    for (size_t i = 0; i < queue.size(); ++i)
      if (fits(queue[i]) && (best < 0 || queue[i].footprint < queue[best].footprint))
        best = (int)i;
    return best;
  }
  bool admissible() const { return pick() >= 0; }

  void worker() {
    cudaSetDevice(device);
    cudaStream_t st = nullptr;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    for (;;) {
      Req r;
      {
        std::unique_lock<std::mutex> g(mu);
        idle++;
        cv_work.notify_all();
        cv_work.wait(g, [&] { return stop || admissible(); });
        // decide while this worker still counts as idle
        const int k = pick();
        idle--;
        if (stop && queue.empty()) break;
        if (k < 0) continue;
        r = queue[k];
        for (int i = 0; i < k; ++i) queue[i].overtaken++;
        queue.erase(queue.begin() + k);
        in_use += (int64_t)r.footprint;
        std::lock_guard<std::mutex> bg(batcher.mu);
        batcher.running++;
      }
      cudaStream_t own = r.p->stream;
      r.p->stream = st;
      lrep_status s = LREP_OK;
      if (!split_ready(r.p)) s = build_split(r.p);
      if (s == LREP_OK) {
        r.p->err.clear();
        s = bosp_solve(r.p, r.nev, r.block, r.tol, &batcher);
      }
      cudaStreamSynchronize(st);
      r.p->stream = own;
      {
        std::lock_guard<std::mutex> bg(batcher.mu);
        batcher.running--;
        batcher.cv.notify_all();
      }
      {
        std::lock_guard<std::mutex> g(mu);
        in_use -= (int64_t)r.footprint;
        done[r.ticket] = s;
      }
      cv_done.notify_all();
      cv_work.notify_all();
    }
    if (st) cudaStreamDestroy(st);
  }
};

extern "C" {

lrep_status lrep_server_create(lrep_server* out, int64_t hbm_budget_bytes, int32_t max_slots,
                               void* stream) {
  (void)stream;
  if (!out || hbm_budget_bytes <= 0 || max_slots < 1 || max_slots > 64) return LREP_ERR_ARG;
  lrep_server s = new lrep_server_s();
  s->budget = hbm_budget_bytes;
  s->max_slots = max_slots;
  cudaGetDevice(&s->device);
  if (s->batcher.init() != cudaSuccess) {
    delete s;
    return LREP_ERR_CUDA;
  }
  for (int i = 0; i < max_slots; ++i) s->workers.emplace_back([s] { s->worker(); });
  *out = s;
  return LREP_OK;
}

lrep_status lrep_footprint(lrep_problem p, int32_t nev, int32_t block, int64_t* bytes) {
  if (!p || !bytes || nev < 1 || block < 1) return LREP_ERR_ARG;
  size_t fp = bosp_footprint(p, nev, block);
  if (!split_ready(p)) fp += split_bytes(p);
  *bytes = (int64_t)fp;
  return LREP_OK;
}

lrep_status lrep_server_submit(lrep_server s, lrep_problem p, int32_t nev, int32_t block,
                               double tol, uint64_t* ticket) {
  if (!s || !p || !ticket || nev < 1 || block < 1 || !(tol > 0.0)) return LREP_ERR_ARG;
  int64_t fpb = 0;
  lrep_footprint(p, nev, block, &fpb);
  const size_t fp = (size_t)fpb;
  if ((int64_t)fp > s->budget) return p->fail(LREP_ERR_NOMEM, "request exceeds the HBM budget");
  std::lock_guard<std::mutex> g(s->mu);
  const uint64_t t = s->next++;
  s->queue.push_back(Req{t, p, nev, block, tol, fp});
  *ticket = t;
  s->cv_work.notify_all();
  return LREP_OK;
}

lrep_status lrep_server_wait(lrep_server s, uint64_t ticket, int32_t timeout_ms) {
  if (!s) return LREP_ERR_ARG;
  std::unique_lock<std::mutex> g(s->mu);
  auto ready = [&] { return s->done.count(ticket) > 0; };
  if (timeout_ms < 0) {
    s->cv_done.wait(g, ready);
  } else if (!s->cv_done.wait_for(g, std::chrono::milliseconds(timeout_ms), ready)) {
    return LREP_ERR_TIMEOUT;
  }
  const lrep_status st = s->done[ticket];
  s->done.erase(ticket);
  return st;
}

lrep_status lrep_server_destroy(lrep_server s) {
  if (!s) return LREP_ERR_ARG;
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers)
    if (t.joinable()) t.join();
  delete s;
  return LREP_OK;
}

lrep_status lrep_server_stats(lrep_server s, int64_t* out3) {
  if (!s || !out3) return LREP_ERR_ARG;
  std::lock_guard<std::mutex> g(s->batcher.mu);
  out3[0] = s->batcher.batches;
  out3[1] = s->batcher.jobs_total;
  out3[2] = s->batcher.max_batch;
  return LREP_OK;
}

}  // extern "C"
