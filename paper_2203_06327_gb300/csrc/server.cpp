// Serving many independent eigenproblems on one GPU (the bpjd_server_* entry
// points of bpjd.h).  Worker threads, each with its own CUDA stream, run
// bpjd_setup + bpjd_solve on requests taken from a queue (smallest estimated
// work first with aging, or first-in first-out); a request starts when its
// estimated device footprint fits in the memory budget beside the requests in
// flight.  With batch_local the local solves of the requests in flight share
// grouped launches (batch.cpp).

#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "bpjd.h"
#include "bpjd_internal.h"

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct CsrCopy {
  int32_t nr = 0, nc = 0;
  std::vector<int64_t> rp;
  std::vector<int32_t> ci;
  std::vector<double> v;
  bool take(const bpjd_csr* c) {
    if (!c || c->n_rows < 1 || c->n_cols < 1 || c->nnz < 0 || !c->row_ptr || (c->nnz > 0 && (!c->col_idx || !c->val)))
      return false;
    nr = c->n_rows;
    nc = c->n_cols;
    rp.assign(c->row_ptr, c->row_ptr + nr + 1);
    ci.assign(c->col_idx, c->col_idx + c->nnz);
    v.assign(c->val, c->val + c->nnz);
    if (rp[0] != 0 || rp[nr] != c->nnz) return false;
    for (int32_t r = 0; r < nr; ++r)
      if (rp[r + 1] < rp[r]) return false;
    for (int32_t x : ci)
      if (x < 0 || x >= nc) return false;
    return true;
  }
  bpjd_csr view() const { return bpjd_csr{nr, nc, (int64_t)ci.size(), rp.data(), ci.data(), v.data()}; }
};

struct Request {
  uint64_t id = 0;
  int32_t k = 0;
  CsrCopy A, M, P, P0;
  bool has_p0 = false;
  std::vector<int64_t> sub_ptr;
  std::vector<int32_t> sub_dofs, sub_color;
  int32_t n_sub = 0, n_colors = 0;
  size_t est_bytes = 0;
  double est_work = 0;      // dofs x k: the admission order of BPJD_ADMIT_SMALLEST
  double t_submit = 0, t_start = 0, t_end = 0;
  bool done = false;
  int status = BPJD_OK;
  std::vector<double> lam, X;
  bpjd_stats st{};
};

// Band width (max |i - j| + 1 over the principal submatrix, local numbering) of
// the widest subdomain: what the local factorisations will hold per row.
int band_width(const Request& r) {
  const int n = r.A.nr;
  std::vector<int32_t> pos(n, -1);
  int band = 0;
  for (int l = 0; l < r.n_sub; ++l) {
    const int64_t b = r.sub_ptr[l], e = r.sub_ptr[l + 1];
    for (int64_t t = b; t < e; ++t) pos[r.sub_dofs[t]] = (int32_t)(t - b);
    for (int64_t t = b; t < e; ++t) {
      const int32_t d = r.sub_dofs[t];
      for (int64_t q = r.A.rp[d]; q < r.A.rp[d + 1]; ++q) {
        const int32_t j = pos[r.A.ci[q]];
        if (j >= 0) band = std::max(band, (int)std::abs((int64_t)(t - b) - j));
      }
    }
    for (int64_t t = b; t < e; ++t) pos[r.sub_dofs[t]] = -1;
  }
  return band + 1;
}

// Device bytes of one solver instance (matrices, bands, band factors, block
// vectors, coarse basis, reduction scratch), with a margin.
size_t estimate_bytes(const Request& r) {
  const size_t n = (size_t)r.A.nr, k = (size_t)r.k;
  const size_t nnz = r.A.ci.size() + r.M.ci.size();
  const size_t nH = (size_t)r.P.nc;
  const size_t sum_nl = (size_t)r.sub_ptr[r.n_sub];
  const int B = band_width(r);
  int Bpad = B;
  for (int t : {16, 24, 32, 40, 48, 64, 96, 128})
    if (B <= t) {
      Bpad = t;
      break;
    }
  size_t b = 0;
  b += 2 * (n + 1) * 8 + nnz * (4 + 8 + 8);                 // K, M and their split values
  b += 2 * (r.P.ci.size() * 12 + (n + nH + 2) * 8);        // P and P^T
  b += sum_nl * std::max((size_t)B * 8, (size_t)Bpad * 4) * 2;  // bands of K_l and M_l (FP64, or FP32 padded)
  {
    // band factors (FP64 worst case), solved in chunks of subdomains within the
    // default 2 GiB scratch bound (at least one subdomain per chunk)
    size_t max_nl = 0;
    for (int l = 0; l < r.n_sub; ++l) max_nl = std::max<size_t>(max_nl, (size_t)(r.sub_ptr[l + 1] - r.sub_ptr[l]));
    b += std::min(sum_nl * k * (size_t)Bpad * 8, ((size_t)2 << 30) + max_nl * k * (size_t)Bpad * 8);
  }
  b += sum_nl * k * 8 + sum_nl * 12;                       // local solutions, maps
  b += n * k * 8 * 20;                                     // block vectors
  b += nH * nH * 8 * 2;                                    // coarse eigenbasis
  b += (size_t)456 * 96 * 96 * 8 + (size_t)6 * 96 * 96 * 8;  // reduction scratch, small matrices
  return b + b / 5 + ((size_t)8 << 20);
}

}  // namespace

struct bpjd_server {
  bpjd_server_opts o{};
  int device = 0;
  size_t budget = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Request>> queue;
  std::unordered_map<uint64_t, std::shared_ptr<Request>> all;
  size_t in_use = 0;
  int running = 0;
  uint64_t next_id = 1;
  bool stop = false;
  std::vector<std::thread> threads;
  bpjd::LocalBatcher* batch = nullptr;  // shared launches of the local solves (batch_local)
};

namespace {

void run_request(bpjd_server* s, Request& r, cudaStream_t stream) {
  bpjd_opts o;
  bpjd_default_opts(&o);
  o.k = r.k;
  o.precision = s->o.precision;
  o.subspace = s->o.subspace;
  o.stop_rule = s->o.stop_rule;
  o.tol = s->o.tol;
  o.max_iter = s->o.max_iter;
  o.inputs_on_device = 0;
  o.stream = stream;
  o.host_loop = s->o.host_loop;
  const bpjd_csr A = r.A.view(), M = r.M.view(), P = r.P.view();
  bpjd_csr P0;
  if (r.has_p0) P0 = r.P0.view();
  bpjd_partition part{r.n_sub, r.sub_ptr.data(), r.sub_dofs.data(),
                      r.sub_color.empty() ? nullptr : r.sub_color.data(), r.n_colors};
  bpjd_handle* h = nullptr;
  int rc = bpjd_setup(&A, &M, &P, r.has_p0 ? &P0 : nullptr, &part, &o, &h);
  if (rc == BPJD_OK) {
    reinterpret_cast<bpjd::Handle*>(h)->batch = s->batch;
    r.lam.resize((size_t)r.k);
    r.X.resize((size_t)r.A.nr * r.k);
    rc = bpjd_solve(h, r.lam.data(), r.X.data(), 0, &r.st);
    bpjd_free(h);
  }
  r.status = rc;
}

// Index of the queued request to start next, or -1 when none fits the budget
// (a request always fits when nothing runs).  FIFO: the head only.  Smallest
// first: any request older than the aging limit goes first (oldest of those),
// otherwise the smallest estimated work among those that fit, ties by arrival.
int pick_request(const bpjd_server* s, double now) {
  auto fits = [&](const Request& r) { return s->in_use + r.est_bytes <= s->budget || s->running == 0; };
  if (s->queue.empty()) return -1;
  if (s->o.admission == BPJD_ADMIT_FIFO) return fits(*s->queue.front()) ? 0 : -1;
  const double limit = s->o.starvation_s > 0 ? s->o.starvation_s : 1.0;
  if (now - s->queue.front()->t_submit > limit) return fits(*s->queue.front()) ? 0 : -1;
  int best = -1;
  for (int i = 0; i < (int)s->queue.size(); ++i) {
    const Request& r = *s->queue[i];
    if (!fits(r)) continue;
    if (best < 0 || r.est_work < s->queue[best]->est_work) best = i;
  }
  return best;
}

void worker(bpjd_server* s) {
  cudaSetDevice(s->device);
  cudaStream_t stream = nullptr;
  // without a stream the worker's requests fail with BPJD_ERR_CUDA
  if (cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess) stream = nullptr;
  for (;;) {
    std::shared_ptr<Request> r;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      int pick = -1;
      s->cv_work.wait(lk, [&] {
        if (s->queue.empty()) return s->stop;
        pick = pick_request(s, now_s());
        return pick >= 0;
      });
      if (s->queue.empty()) break;
      r = s->queue[pick];
      s->queue.erase(s->queue.begin() + pick);
      s->in_use += r->est_bytes;
      ++s->running;
      r->t_start = now_s();
    }
    if (stream)
      run_request(s, *r, stream);
    else
      r->status = BPJD_ERR_CUDA;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->in_use -= r->est_bytes;
      --s->running;
      r->t_end = now_s();
      r->done = true;
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();
  }
  if (stream) cudaStreamDestroy(stream);
}

}  // namespace

extern "C" void bpjd_server_default_opts(bpjd_server_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->hbm_budget_bytes = 0;
  o->workers = 8;
  o->precision = BPJD_MIXED;
  o->subspace = BPJD_W_3K;
  o->stop_rule = BPJD_STOP_RESIDUAL;
  o->tol = 1e-8;
  o->max_iter = 500;
  o->admission = BPJD_ADMIT_SMALLEST;
  o->starvation_s = 1.0;
  o->host_loop = 1;
  o->batch_local = 1;
  o->batch_wait_us = 100;
}

extern "C" int bpjd_server_create(const bpjd_server_opts* opts, bpjd_server** out) {
  if (!opts || !out) return BPJD_ERR_BAD_ARG;
  *out = nullptr;
  if (opts->workers < 1 || opts->workers > 32) return BPJD_ERR_BAD_ARG;
  if (opts->admission != BPJD_ADMIT_SMALLEST && opts->admission != BPJD_ADMIT_FIFO) return BPJD_ERR_BAD_ARG;
  if (opts->batch_local < 0 || opts->batch_local > 1 || opts->batch_wait_us < 0 ||
      (opts->batch_local && !opts->host_loop))
    return BPJD_ERR_BAD_ARG;
  auto* s = new bpjd_server;
  s->o = *opts;
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    return BPJD_ERR_CUDA;
  }
  if (opts->batch_local) {
    s->batch = bpjd::batch_create(opts->batch_wait_us);
    if (!s->batch) {
      delete s;
      return BPJD_ERR_CUDA;
    }
  }
  s->budget = opts->hbm_budget_bytes;
  if (s->budget == 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      delete s;
      return BPJD_ERR_CUDA;
    }
    s->budget = fr / 10 * 8;
  }
  for (int w = 0; w < opts->workers; ++w) s->threads.emplace_back(worker, s);
  *out = s;
  return BPJD_OK;
}

extern "C" int bpjd_server_submit(bpjd_server* s, const bpjd_csr* A, const bpjd_csr* M, const bpjd_csr* P,
                                  const bpjd_csr* P0, const bpjd_partition* part, int32_t k, uint64_t* ticket) {
  if (!s || !part || !ticket || k < 1 || k > 32) return BPJD_ERR_BAD_ARG;
  auto r = std::make_shared<Request>();
  r->k = k;
  if (!r->A.take(A) || !r->M.take(M) || !r->P.take(P)) return BPJD_ERR_CSR_INVALID;
  if (P0) {
    if (!r->P0.take(P0)) return BPJD_ERR_CSR_INVALID;
    r->has_p0 = true;
  }
  const int32_t n = r->A.nr;
  if (r->A.nc != n || r->M.nr != n || r->M.nc != n || r->P.nr != n || (r->has_p0 && r->P0.nr != n))
    return BPJD_ERR_BAD_ARG;
  if (part->n_sub < 1 || !part->sub_ptr || !part->sub_dofs) return BPJD_ERR_MAP_INVALID;
  r->n_sub = part->n_sub;
  r->n_colors = part->n_colors;
  r->sub_ptr.assign(part->sub_ptr, part->sub_ptr + part->n_sub + 1);
  if (r->sub_ptr[0] != 0) return BPJD_ERR_MAP_INVALID;
  for (int l = 0; l < r->n_sub; ++l)
    if (r->sub_ptr[l + 1] <= r->sub_ptr[l]) return BPJD_ERR_MAP_INVALID;
  r->sub_dofs.assign(part->sub_dofs, part->sub_dofs + r->sub_ptr[r->n_sub]);
  for (int l = 0; l < r->n_sub; ++l)
    for (int64_t t = r->sub_ptr[l]; t < r->sub_ptr[l + 1]; ++t) {
      const int32_t d = r->sub_dofs[t];
      if (d < 0 || d >= n || (t > r->sub_ptr[l] && d <= r->sub_dofs[t - 1])) return BPJD_ERR_MAP_INVALID;
    }
  if (part->sub_color) r->sub_color.assign(part->sub_color, part->sub_color + r->n_sub);
  r->est_bytes = estimate_bytes(*r);
  r->est_work = (double)n * (double)k;
  if (r->est_bytes > s->budget) return BPJD_ERR_TOO_LARGE;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    r->id = s->next_id++;
    r->t_submit = now_s();
    s->all[r->id] = r;
    s->queue.push_back(r);
    *ticket = r->id;
  }
  s->cv_work.notify_one();
  return BPJD_OK;
}

extern "C" int bpjd_server_poll(bpjd_server* s, uint64_t ticket, int32_t wait, double* eigvals, double* eigvecs,
                                bpjd_stats* st, double* times) {
  if (!s) return BPJD_ERR_BAD_ARG;
  std::shared_ptr<Request> r;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return BPJD_ERR_BAD_ARG;
    r = it->second;
    if (!r->done) {
      if (!wait) return BPJD_PENDING;
      s->cv_done.wait(lk, [&] { return r->done; });
    }
    s->all.erase(ticket);
  }
  if (r->status == BPJD_OK) {
    if (eigvals) std::memcpy(eigvals, r->lam.data(), sizeof(double) * r->lam.size());
    if (eigvecs) std::memcpy(eigvecs, r->X.data(), sizeof(double) * r->X.size());
  }
  if (st) {
    *st = r->st;
    st->status = r->status;
  }
  if (times) {
    times[0] = r->t_start - r->t_submit;
    times[1] = r->t_end - r->t_start;
    times[2] = r->t_end - r->t_submit;
  }
  return r->status;
}

extern "C" void bpjd_server_free(bpjd_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->threads) t.join();
  bpjd::batch_free(s->batch);
  delete s;
}

extern "C" int bpjd_server_batch_stats(const bpjd_server* s, int64_t* launches, int64_t* solves) {
  if (!s) return BPJD_ERR_BAD_ARG;
  if (launches) *launches = 0;
  if (solves) *solves = 0;
  if (s->batch) bpjd::batch_stats(s->batch, launches, solves);
  return BPJD_OK;
}
