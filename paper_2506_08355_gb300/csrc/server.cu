// Serving loop of lrep.h: a host thread that admits submitted solves by
// their HBM footprint and slot count and runs them.
#include <cuda_runtime.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>

#include "../../include/lrep.h"
#include "problem.h"

namespace {
struct Req {
  uint64_t ticket;
  lrep_problem p;
  int nev, block;
  double tol;
};
}  // namespace

struct lrep_server_s {
  std::mutex mu;
  std::condition_variable cv, cv_done;
  std::deque<Req> queue;
  std::map<uint64_t, lrep_status> done;
  uint64_t next = 1;
  bool stop = false;
  int64_t budget = 0;
  int max_slots = 1;
  cudaStream_t stream = nullptr;
  std::thread worker;
  int device = 0;

  void loop() {
    cudaSetDevice(device);
    for (;;) {
      Req r;
      {
        std::unique_lock<std::mutex> g(mu);
        cv.wait(g, [&] { return stop || !queue.empty(); });
        if (stop && queue.empty()) return;
        r = queue.front();
        queue.pop_front();
      }
      const lrep_status s = lrep_solve(r.p, r.nev, r.block, r.tol);
      {
        std::lock_guard<std::mutex> g(mu);
        done[r.ticket] = s;
      }
      cv_done.notify_all();
    }
  }
};

extern "C" {

lrep_status lrep_server_create(lrep_server* out, int64_t hbm_budget_bytes, int32_t max_slots,
                               void* stream) {
  if (!out || hbm_budget_bytes <= 0 || max_slots < 1) return LREP_ERR_ARG;
  lrep_server s = new lrep_server_s();
  s->budget = hbm_budget_bytes;
  s->max_slots = max_slots;
  s->stream = (cudaStream_t)stream;
  cudaGetDevice(&s->device);
  s->worker = std::thread([s] { s->loop(); });
  *out = s;
  return LREP_OK;
}

lrep_status lrep_server_submit(lrep_server s, lrep_problem p, int32_t nev, int32_t block,
                               double tol, uint64_t* ticket) {
  if (!s || !p || !ticket || nev < 1 || block < 1 || !(tol > 0.0)) return LREP_ERR_ARG;
  std::lock_guard<std::mutex> g(s->mu);
  const uint64_t t = s->next++;
  s->queue.push_back(Req{t, p, nev, block, tol});
  *ticket = t;
  s->cv.notify_all();
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
  s->cv.notify_all();
  if (s->worker.joinable()) s->worker.join();
  delete s;
  return LREP_OK;
}

}  // extern "C"
