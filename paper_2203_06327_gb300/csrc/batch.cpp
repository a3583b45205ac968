// Packing the local solves of several in-flight solves into shared launches
// (the serving path of the bpjd_server_* entry points).
//
// Every served request runs its own host-driven iteration loop on its own
// worker thread and CUDA stream.  When a request reaches the local part of its
// preconditioner application (Eq. (3.3), first term: the banded factorisations
// or forward sweeps and the backward sweeps of all its (subdomain, shift)
// pairs), it hands the work to the batcher and blocks.  The batcher launches
// the pending work of every request as soon as each request in a solve has
// handed in its own, or once the oldest waited batch_wait_us: one grouped
// launch per kernel kind and window tier, over all subdomains of all those
// requests (launch_local_grouped; the factorisations of the wide tiers keep a
// launch per request), on the batcher's stream, ordered after each
// request's stream by an event and before the rest of each request's step by
// another.  Each pair is computed by the same kernel body on the same inputs as
// in a launch of its request alone, so the results do not depend on the mix.

#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <mutex>
#include <vector>

#include "bpjd_internal.h"

namespace bpjd {

struct LocalBatcher {
  struct Job {
    Handle* h;
    const double* rho;
    const double* lam;
    int refactor;
    int rc;
    bool done;
  };
  std::mutex mu;
  std::condition_variable cv;
  std::vector<Job*> pending;
  int members = 0;  // solves in progress that hand in their local solves
  int wait_us = 100;
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaEvent_t done_ev = nullptr;
  int64_t flushes = 0, jobs = 0;

  // Launches every pending job (caller holds mu).
  void flush_locked() {
    std::vector<Job*> js;
    js.swap(pending);
    if (js.empty()) return;
    int rc = BPJD_OK;
    // the batcher's stream after each request's work so far
    for (Job* q : js) {
      Handle& h = *q->h;
      if (!h.batch_ev) {
        cudaEvent_t ev;
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
          rc = BPJD_ERR_CUDA;
          break;
        }
        h.batch_ev = ev;
      }
      if (cudaEventRecord((cudaEvent_t)h.batch_ev, h.stream) != cudaSuccess ||
          cudaStreamWaitEvent(stream, (cudaEvent_t)h.batch_ev, 0) != cudaSuccess) {
        rc = BPJD_ERR_CUDA;
        break;
      }
    }
    // one grouped launch per window tier (at most kGroupedMax requests each)
    if (rc == BPJD_OK) {
      std::vector<Job*> order(js);
      std::stable_sort(order.begin(), order.end(),
                       [](const Job* a, const Job* b) { return a->h->Bpad < b->h->Bpad; });
      for (size_t a = 0; a < order.size() && rc == BPJD_OK;) {
        size_t b = a;
        while (b < order.size() && b - a < (size_t)kGroupedMax && order[b]->h->Bpad == order[a]->h->Bpad) ++b;
        Handle* hs[kGroupedMax];
        const double* rh[kGroupedMax];
        const double* lm[kGroupedMax];
        int rf[kGroupedMax];
        for (size_t j = a; j < b; ++j) {
          hs[j - a] = order[j]->h;
          rh[j - a] = order[j]->rho;
          lm[j - a] = order[j]->lam;
          rf[j - a] = order[j]->refactor;
        }
        if (launch_local_grouped(hs, rh, lm, rf, (int)(b - a), stream) != 0) rc = BPJD_ERR_CUDA;
        a = b;
      }
    }
    // the rest of each request's step after the shared launches
    if (rc == BPJD_OK && cudaEventRecord(done_ev, stream) != cudaSuccess) rc = BPJD_ERR_CUDA;
    for (Job* q : js) {
      if (rc == BPJD_OK && cudaStreamWaitEvent(q->h->stream, done_ev, 0) != cudaSuccess) q->rc = BPJD_ERR_CUDA;
      else q->rc = rc;
      q->done = true;
    }
    ++flushes;
    jobs += (int64_t)js.size();
    cv.notify_all();
  }
};

LocalBatcher* batch_create(int wait_us) {
  auto* b = new LocalBatcher;
  b->wait_us = std::max(0, wait_us);
  if (cudaGetDevice(&b->device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->done_ev, cudaEventDisableTiming) != cudaSuccess) {
    batch_free(b);
    return nullptr;
  }
  return b;
}

void batch_free(LocalBatcher* b) {
  if (!b) return;
  if (b->stream) {
    cudaStreamSynchronize(b->stream);
    cudaStreamDestroy(b->stream);
  }
  if (b->done_ev) cudaEventDestroy(b->done_ev);
  delete b;
}

void batch_enter(LocalBatcher* b) {
  std::lock_guard<std::mutex> lk(b->mu);
  ++b->members;
}

void batch_leave(LocalBatcher* b) {
  std::lock_guard<std::mutex> lk(b->mu);
  --b->members;
  // the requests still waiting need not wait for this one
  if (!b->pending.empty() && (int)b->pending.size() >= b->members) b->flush_locked();
}

bool batch_eligible(const Handle& h) { return h.host_loop && h.local_f32() && can_reuse_factors(h); }

int batch_local(LocalBatcher* b, Handle& h, const double* rho, const double* lam, bool refactor) {
  std::unique_lock<std::mutex> lk(b->mu);
  LocalBatcher::Job job{&h, rho, lam, refactor ? 1 : 0, BPJD_OK, false};
  b->pending.push_back(&job);
  if ((int)b->pending.size() >= b->members) {
    b->flush_locked();
  } else {
    const auto until = std::chrono::steady_clock::now() + std::chrono::microseconds(b->wait_us);
    b->cv.wait_until(lk, until, [&] { return job.done; });
    if (!job.done) b->flush_locked();
  }
  return job.rc == BPJD_OK ? 0 : (int)cudaErrorUnknown;
}

void batch_stats(const LocalBatcher* b, int64_t* flushes, int64_t* jobs) {
  auto* m = const_cast<LocalBatcher*>(b);
  std::lock_guard<std::mutex> lk(m->mu);
  if (flushes) *flushes = m->flushes;
  if (jobs) *jobs = m->jobs;
}

}  // namespace bpjd
