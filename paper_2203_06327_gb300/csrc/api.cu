// C ABI of the BPJD library: setup (Algorithm 3.1 Step 1 and the device
// data of Eq. (3.3)), the iteration driver (Steps 2-4) and the step-level
// entry points.  See include/bpjd.h for the contract of every function.

#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <future>
#include <new>
#include <thread>
#include <vector>

#include "bpjd_internal.h"

using namespace bpjd;

namespace {

#define CK(call)                          \
  do {                                    \
    cudaError_t e_ = (call);              \
    if (e_ != cudaSuccess) {              \
      rc = (e_ == cudaErrorMemoryAllocation) ? BPJD_ERR_OOM : BPJD_ERR_CUDA; \
      goto fail;                          \
    }                                     \
  } while (0)

#define CKI(call)                         \
  do {                                    \
    int e_ = (call);                      \
    if (e_ != 0) {                        \
      rc = BPJD_ERR_CUDA;                 \
      goto fail;                          \
    }                                     \
  } while (0)

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// BPJD_TRACE=1 in the environment: JSON lines on stderr for setup phases and
// iterations.
bool trace_on() {
  static const bool on = [] {
    const char* e = std::getenv("BPJD_TRACE");
    return e && e[0] && e[0] != '0';
  }();
  return on;
}

struct PhaseTimer {
  double t;
  std::string buf;
  PhaseTimer() : t(now_s()) {}
  void mark(const char* name, cudaStream_t s) {
    if (!trace_on()) return;
    cudaStreamSynchronize(s);
    const double u = now_s();
    char tmp[96];
    std::snprintf(tmp, sizeof(tmp), "%s\"%s\": %.3f", buf.empty() ? "" : ", ", name, 1e3 * (u - t));
    buf += tmp;
    t = u;
  }
  void emit() {
    if (trace_on()) std::fprintf(stderr, "{\"bpjd_setup_ms\": {%s}}\n", buf.c_str());
  }
};

template <typename T>
cudaError_t dalloc(Handle& h, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e == cudaSuccess) {
    h.allocs.push_back((void*)*p);
    h.bytes += count * sizeof(T);
  }
  return e;
}

// Host view of a CSR (copied from the device when the inputs live there).
struct HostCsr {
  int32_t n_rows = 0, n_cols = 0;
  int64_t nnz = 0;
  std::vector<int64_t> rp_buf;
  std::vector<int32_t> ci_buf;
  std::vector<double> v_buf;
  const int64_t* rp = nullptr;
  const int32_t* ci = nullptr;
  const double* v = nullptr;
};

int host_view(const bpjd_csr* c, bool on_dev, bool need_vals, HostCsr& out) {
  out.n_rows = c->n_rows;
  out.n_cols = c->n_cols;
  out.nnz = c->nnz;
  if (!on_dev) {
    out.rp = c->row_ptr;
    out.ci = c->col_idx;
    out.v = c->val;
    return BPJD_OK;
  }
  out.rp_buf.resize((size_t)c->n_rows + 1);
  out.ci_buf.resize((size_t)std::max<int64_t>(c->nnz, 1));
  if (cudaMemcpy(out.rp_buf.data(), c->row_ptr, sizeof(int64_t) * (c->n_rows + 1), cudaMemcpyDeviceToHost) !=
      cudaSuccess)
    return BPJD_ERR_CUDA;
  if (c->nnz > 0 &&
      cudaMemcpy(out.ci_buf.data(), c->col_idx, sizeof(int32_t) * c->nnz, cudaMemcpyDeviceToHost) != cudaSuccess)
    return BPJD_ERR_CUDA;
  if (need_vals) {
    out.v_buf.resize((size_t)std::max<int64_t>(c->nnz, 1));
    if (c->nnz > 0 && cudaMemcpy(out.v_buf.data(), c->val, sizeof(double) * c->nnz, cudaMemcpyDeviceToHost) !=
                          cudaSuccess)
      return BPJD_ERR_CUDA;
    out.v = out.v_buf.data();
  }
  out.rp = out.rp_buf.data();
  out.ci = out.ci_buf.data();
  return BPJD_OK;
}

// Row pointers start at 0, end at nnz and never decrease; every row's columns
// ascend strictly within [0, n_cols).  The matrices are checked together, in
// row ranges on up to 16 host threads (a row range only reads its own rows).
int validate_csrs(const std::vector<const HostCsr*>& cs) {
  int64_t nnz = 0;
  for (const HostCsr* c : cs) {
    if (c->n_rows < 0 || c->n_cols < 0 || c->nnz < 0) return BPJD_ERR_BAD_ARG;
    if (c->rp[0] != 0 || c->rp[c->n_rows] != c->nnz) return BPJD_ERR_CSR_INVALID;
    // the row pointers first: every row range then indexes inside [0, nnz)
    for (int64_t r = 0; r < c->n_rows; ++r)
      if (c->rp[r + 1] < c->rp[r] || c->rp[r + 1] > c->nnz) return BPJD_ERR_CSR_INVALID;
    nnz += c->nnz;
  }
  auto rows = [](const HostCsr& c, int64_t r0, int64_t r1) -> bool {
    for (int64_t r = r0; r < r1; ++r)
      for (int64_t e = c.rp[r]; e < c.rp[r + 1]; ++e) {
        if (c.ci[e] < 0 || c.ci[e] >= c.n_cols) return false;
        if (e > c.rp[r] && c.ci[e] <= c.ci[e - 1]) return false;
      }
    return true;
  };
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const int T = (int)std::max<int64_t>(1, std::min<int64_t>(std::min<unsigned>(16, hw), nnz / 400000));
  std::vector<char> ok((size_t)T, 1);
  auto part = [&](int t) {
    for (const HostCsr* c : cs) {
      const int64_t per = (c->n_rows + T - 1) / T;
      const int64_t r0 = std::min<int64_t>(c->n_rows, t * per), r1 = std::min<int64_t>(c->n_rows, r0 + per);
      if (!rows(*c, r0, r1)) ok[t] = 0;
    }
  };
  std::vector<std::thread> th;
  for (int t = 1; t < T; ++t) th.emplace_back(part, t);
  part(0);
  for (auto& x : th) x.join();
  for (char v : ok)
    if (!v) return BPJD_ERR_CSR_INVALID;
  return BPJD_OK;
}

// Copies a CSR (host or device source) into handle-owned device memory.
cudaError_t upload_csr(Handle& h, const bpjd_csr* c, bool on_dev, CsrDev& d, bool vals = true) {
  d.n_rows = c->n_rows;
  d.n_cols = c->n_cols;
  d.nnz = c->nnz;
  cudaMemcpyKind kind = on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  cudaError_t e;
  if ((e = dalloc(h, &d.row_ptr, (size_t)c->n_rows + 1)) != cudaSuccess) return e;
  if ((e = dalloc(h, &d.col, (size_t)c->nnz)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(d.row_ptr, c->row_ptr, sizeof(int64_t) * (c->n_rows + 1), kind, h.stream)) != cudaSuccess)
    return e;
  if (c->nnz && (e = cudaMemcpyAsync(d.col, c->col_idx, sizeof(int32_t) * c->nnz, kind, h.stream)) != cudaSuccess)
    return e;
  if (vals) {
    if ((e = dalloc(h, &d.val, (size_t)c->nnz)) != cudaSuccess) return e;
    if (c->nnz && (e = cudaMemcpyAsync(d.val, c->val, sizeof(double) * c->nnz, kind, h.stream)) != cudaSuccess)
      return e;
  }
  return cudaSuccess;
}

// Subdomain lists: sub_ptr starts at 0 and grows strictly, every list ascending
// within [0, n).
int validate_partition(int nsub, int n, const int64_t* sptr, const int32_t* sdofs) {
  if (sptr[0] != 0) return BPJD_ERR_MAP_INVALID;
  for (int l = 0; l < nsub; ++l) {
    if (sptr[l + 1] <= sptr[l]) return BPJD_ERR_MAP_INVALID;
    for (int64_t e = sptr[l]; e < sptr[l + 1]; ++e)
      if (sdofs[e] < 0 || sdofs[e] >= n || (e > sptr[l] && sdofs[e] <= sdofs[e - 1])) return BPJD_ERR_MAP_INVALID;
  }
  return BPJD_OK;
}

// Galerkin products K_H = P^T K P and M_H = P^T M P on the device, copied to
// the host (symmetrised) for the dense coarse eigensolve.
int galerkin_host(Handle& h, const CsrDev& P, const CsrDev& PT, std::vector<double>& KH, std::vector<double>& MH) {
  int rc = BPJD_OK;
  const int nH = P.n_cols;
  double *dKH = nullptr, *dMH = nullptr;
  KH.assign((size_t)nH * nH, 0.0);
  MH.assign((size_t)nH * nH, 0.0);
  CK(cudaMalloc(&dKH, sizeof(double) * nH * nH));
  CK(cudaMalloc(&dMH, sizeof(double) * nH * nH));
  CKI(launch_galerkin(h.A, h.same_pattern ? CsrDev{h.A.n_rows, h.A.n_cols, h.A.nnz, h.A.row_ptr, h.A.col, h.M.val}
                                          : h.M,
                      P, PT, dKH, dMH, h.stream));
  CK(cudaMemcpyAsync(KH.data(), dKH, sizeof(double) * nH * nH, cudaMemcpyDeviceToHost, h.stream));
  CK(cudaMemcpyAsync(MH.data(), dMH, sizeof(double) * nH * nH, cudaMemcpyDeviceToHost, h.stream));
  CK(cudaStreamSynchronize(h.stream));
  for (int i = 0; i < nH; ++i)
    for (int j = i + 1; j < nH; ++j) {
      double a = 0.5 * (KH[(size_t)i * nH + j] + KH[(size_t)j * nH + i]);
      KH[(size_t)i * nH + j] = KH[(size_t)j * nH + i] = a;
      double b = 0.5 * (MH[(size_t)i * nH + j] + MH[(size_t)j * nH + i]);
      MH[(size_t)i * nH + j] = MH[(size_t)j * nH + i] = b;
    }
fail:
  cudaFree(dKH);
  cudaFree(dMH);
  return rc;
}

struct EigResult {
  int rc = BPJD_OK;
  std::vector<double> lam, Phi;
};

}  // namespace

// ===========================================================================

extern "C" void bpjd_default_opts(bpjd_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->k = 1;
  o->precision = BPJD_FP64;
  o->subspace = BPJD_W_2K;
  o->stop_rule = BPJD_STOP_RESIDUAL;
  o->tol = 1e-8;
  o->max_iter = 500;
  o->drop_tol = 1e-10;
}

extern "C" const char* bpjd_status_string(int c) {
  switch (c) {
    case BPJD_OK: return "ok";
    case BPJD_ERR_BAD_ARG: return "bad argument";
    case BPJD_ERR_CSR_INVALID: return "invalid CSR matrix";
    case BPJD_ERR_MAP_INVALID: return "invalid subdomain map";
    case BPJD_ERR_K_TOO_LARGE: return "k must be smaller than the coarse space dimension";
    case BPJD_ERR_GAP: return "coarse eigenvalues k and k+1 coincide (Assumption 1)";
    case BPJD_ERR_LOCAL_INDEFINITE: return "shifted local matrix not positive definite (Eq. (3.1))";
    case BPJD_ERR_BREAKDOWN: return "Rayleigh-Ritz basis lost rank";
    case BPJD_ERR_NOCONV: return "no convergence within max_iter";
    case BPJD_ERR_OOM: return "device out of memory";
    case BPJD_ERR_CUDA: return "CUDA error";
    case BPJD_ERR_UNSUPPORTED: return "unsupported option";
    case BPJD_ERR_TOO_LARGE: return "request exceeds the fixed scratch capacity of the allocation-free entry point";
    case BPJD_ERR_TIMEOUT: return "a bounded device-side wait ran out (bulk copy not completed in time)";
    default: return "unknown status";
  }
}

extern "C" void bpjd_free(bpjd_handle* hh) {
  if (!hh) return;
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->gexec) cudaGraphExecDestroy((cudaGraphExec_t)h->gexec);
  for (void* st : h->gside)
    if (st) cudaStreamDestroy((cudaStream_t)st);
  for (void* p : h->allocs) cudaFree(p);
  for (void* e : h->ev_pool) cudaEventDestroy((cudaEvent_t)e);
  if (h->batch_ev) cudaEventDestroy((cudaEvent_t)h->batch_ev);
  if (h->hstat) cudaFreeHost(h->hstat);
  delete h;
}

extern "C" int bpjd_setup(const bpjd_csr* A, const bpjd_csr* M, const bpjd_csr* P, const bpjd_csr* P0,
                          const bpjd_partition* part, const bpjd_opts* opts, bpjd_handle** out) {
  if (!out) return BPJD_ERR_BAD_ARG;
  *out = nullptr;
  if (!A || !M || !P || !part || !opts) return BPJD_ERR_BAD_ARG;
  if (!A->row_ptr || !A->col_idx || !A->val || !M->row_ptr || !M->col_idx || !M->val || !P->row_ptr ||
      !P->col_idx || !P->val || !part->sub_ptr || !part->sub_dofs)
    return BPJD_ERR_BAD_ARG;
  const int k = opts->k;
  const int n = A->n_rows;
  if (k < 1 || k > 32 || n < 1 || A->n_cols != n || M->n_rows != n || M->n_cols != n || P->n_rows != n ||
      part->n_sub < 1)
    return BPJD_ERR_BAD_ARG;
  if (P0 && (P0->n_rows != n || !P0->row_ptr || !P0->col_idx || !P0->val)) return BPJD_ERR_BAD_ARG;
  if (opts->precision != BPJD_FP64 && opts->precision != BPJD_MIXED && opts->precision != BPJD_MIXED_LOCAL)
    return BPJD_ERR_UNSUPPORTED;
  if (opts->subspace != BPJD_W_2K && opts->subspace != BPJD_W_3K) return BPJD_ERR_UNSUPPORTED;
  const int mmax = (opts->subspace == BPJD_W_3K) ? 3 * k : 2 * k;
  if (mmax > 64) return BPJD_ERR_UNSUPPORTED;
  const bool on_dev = opts->inputs_on_device != 0;
  const double t0 = now_s();

  Handle* h = new (std::nothrow) Handle();
  if (!h) return BPJD_ERR_OOM;
  int rc = BPJD_OK;
  h->n = n;
  h->k = k;
  h->nsub = part->n_sub;
  h->precision = opts->precision;
  h->subspace = opts->subspace;
  h->stop_rule = opts->stop_rule;
  h->tol = opts->tol > 0 ? opts->tol : 1e-8;
  h->max_iter = opts->max_iter > 0 ? opts->max_iter : 500;
  h->drop_tol = opts->drop_tol > 0 ? opts->drop_tol : 1e-10;
  // reuse of the local factors while the shifts stay within a relative tolerance
  // (default 3e-4 with FP32 local solves; exact shifts for BPJD_FP64 or a negative value)
  h->refactor_tol = opts->local_refactor_tol > 0
                        ? opts->local_refactor_tol
                        : ((opts->local_refactor_tol == 0 && opts->precision != BPJD_FP64) ? 3e-4 : 0.0);
  h->stream = (cudaStream_t)opts->stream;
  h->host_loop = opts->host_loop != 0;

  {
    std::vector<int64_t> sub_ptr_buf;
    std::vector<int32_t> sub_dofs_buf;
    const int64_t* sptr = nullptr;
    const int32_t* sdofs = nullptr;
    const int nsub = part->n_sub;
    std::vector<double> lamH, Phi, lam0H, Phi0;
    int64_t sum_nl;
    int bw = 0;
    std::vector<int32_t> rtp, rtpos;
    CsrDev dP0, dP0T;
    double* dPhi0 = nullptr;
    PhaseTimer pt;
    Handle tmp0;  // device copies of P0 and its transpose (released at the end of setup)
    std::future<EigResult> eigP, eigP0;

    if (!on_dev) {
      // host inputs are validated before any device work (device inputs on the device below)
      HostCsr vA, vM, vP, vP0;
      host_view(A, false, false, vA);
      host_view(M, false, false, vM);
      host_view(P, false, false, vP);
      std::vector<const HostCsr*> cs{&vA, &vM, &vP};
      if (P0) {
        host_view(P0, false, false, vP0);
        cs.push_back(&vP0);
      }
      if ((rc = validate_csrs(cs)) != BPJD_OK) goto fail;
      if ((rc = validate_partition(nsub, n, part->sub_ptr, part->sub_dofs)) != BPJD_OK) goto fail;
    }
    h->nH = P->n_cols;
    h->nH0 = P0 ? P0->n_cols : P->n_cols;
    if (!(k < h->nH) || !(k < h->nH0)) {
      rc = BPJD_ERR_K_TOO_LARGE;
      goto fail;
    }
    if (h->nH > kTransposeMaxCols || h->nH0 > kTransposeMaxCols) {
      rc = BPJD_ERR_TOO_LARGE;
      goto fail;
    }
    pt.mark("host_validate", h->stream);
    // device copies of the matrices and interpolations, validated on the device
    // before any kernel indexes with them
    CK(upload_csr(*h, A, on_dev, h->A));
    CK(upload_csr(*h, M, on_dev, h->M));
    CK(upload_csr(*h, P, on_dev, h->P));
    tmp0.stream = h->stream;
    if (P0) CK(upload_csr(tmp0, P0, on_dev, dP0));
    CK(dalloc(*h, &h->derr, 4));
    CK(cudaMemsetAsync(h->derr, 0, 4 * sizeof(int32_t), h->stream));
    CKI(launch_validate_csr(h->A, h->derr, h->stream));
    CKI(launch_validate_csr(h->M, h->derr, h->stream));
    CKI(launch_validate_csr(h->P, h->derr, h->stream));
    if (P0) CKI(launch_validate_csr(dP0, h->derr, h->stream));
    if (A->nnz == M->nnz) CKI(launch_same_pattern(h->A, h->M, h->derr, h->stream));
    {
      int32_t flags = 0;
      CK(cudaMemcpyAsync(&flags, h->derr, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
      CK(cudaStreamSynchronize(h->stream));
      if (flags & 1) {
        rc = BPJD_ERR_CSR_INVALID;
        goto fail;
      }
      h->same_pattern = (A->nnz == M->nnz) && !(flags & 2);
    }
    if (h->dword()) {
      CK(dalloc(*h, &h->Asplit, (size_t)A->nnz));
      CK(dalloc(*h, &h->Msplit, (size_t)M->nnz));
      CK(dalloc(*h, &h->xsplit, (size_t)n * k));
      CKI(launch_split_values(h->A.val, A->nnz, h->Asplit, h->stream));
      CKI(launch_split_values(h->M.val, M->nnz, h->Msplit, h->stream));
    }
    // P^T on the device (rows in ascending fine index)
    h->PT.n_rows = h->nH;
    h->PT.n_cols = n;
    h->PT.nnz = P->nnz;
    CK(dalloc(*h, &h->PT.row_ptr, (size_t)h->nH + 1));
    CK(dalloc(*h, &h->PT.col, (size_t)P->nnz));
    CK(dalloc(*h, &h->PT.val, (size_t)P->nnz));
    CKI(launch_csr_transpose(h->P, h->PT.row_ptr, h->PT.col, h->PT.val, h->stream));
    if (h->local_f32()) {
      // FP32 preconditioners take the prolongation-add in FP32
      CK(dalloc(*h, &h->Psplit, (size_t)std::max<int64_t>(P->nnz, 1)));
      CKI(launch_split_values(h->P.val, P->nnz, h->Psplit, h->stream));
    }
    // coarse pencils: Galerkin products on the device now, dense eigensolves on
    // host threads while the device-side setup below proceeds
    {
      std::vector<double> KH, MH;
      if ((rc = galerkin_host(*h, h->P, h->PT, KH, MH)) != BPJD_OK) goto fail;
      const int nH = h->nH;
      eigP = std::async(std::launch::async, [nH, KH = std::move(KH), MH = std::move(MH)]() {
        EigResult r;
        r.rc = gen_eig_host(nH, KH, MH, r.lam, r.Phi);
        return r;
      });
      if (P0) {
        dP0T.n_rows = h->nH0;
        dP0T.n_cols = n;
        dP0T.nnz = P0->nnz;
        CK(dalloc(tmp0, &dP0T.row_ptr, (size_t)h->nH0 + 1));
        CK(dalloc(tmp0, &dP0T.col, (size_t)P0->nnz));
        CK(dalloc(tmp0, &dP0T.val, (size_t)P0->nnz));
        CKI(launch_csr_transpose(dP0, dP0T.row_ptr, dP0T.col, dP0T.val, h->stream));
        tmp0.A = h->A;
        tmp0.M = h->M;
        tmp0.same_pattern = h->same_pattern;
        std::vector<double> K0, M0;
        if ((rc = galerkin_host(tmp0, dP0, dP0T, K0, M0)) != BPJD_OK) goto fail;
        const int nH0 = h->nH0;
        eigP0 = std::async(std::launch::async, [nH0, k, K0 = std::move(K0), M0 = std::move(M0)]() {
          EigResult r;
          // the initial guess needs the lowest k eigenvectors of the grid H/2^tau only
          r.rc = gen_eig_host(nH0, K0, M0, r.lam, r.Phi, k);
          return r;
        });
      }
    }
    pt.mark("validate_upload_galerkin", h->stream);
    // partition (validated on the host while the coarse eigensolves run)
    if (on_dev) {
      sub_ptr_buf.resize(nsub + 1);
      CK(cudaMemcpy(sub_ptr_buf.data(), part->sub_ptr, sizeof(int64_t) * (nsub + 1), cudaMemcpyDeviceToHost));
      sub_dofs_buf.resize((size_t)std::max<int64_t>(sub_ptr_buf[nsub], 1));
      if (sub_ptr_buf[nsub] > 0)
        CK(cudaMemcpy(sub_dofs_buf.data(), part->sub_dofs, sizeof(int32_t) * sub_ptr_buf[nsub],
                      cudaMemcpyDeviceToHost));
      sptr = sub_ptr_buf.data();
      sdofs = sub_dofs_buf.data();
    } else {
      sptr = part->sub_ptr;
      sdofs = part->sub_dofs;
    }
    if (on_dev && (rc = validate_partition(nsub, n, sptr, sdofs)) != BPJD_OK) goto fail;
    for (int l = 0; l < nsub; ++l) h->max_nl = std::max<int32_t>(h->max_nl, (int32_t)(sptr[l + 1] - sptr[l]));
    sum_nl = sptr[nsub];
    h->sum_nl = sum_nl;
    CK(dalloc(*h, &h->sub_ptr, (size_t)nsub + 1));
    CK(dalloc(*h, &h->sub_dofs, (size_t)sum_nl));
    CK(cudaMemcpyAsync(h->sub_ptr, sptr, sizeof(int64_t) * (nsub + 1), cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(h->sub_dofs, sdofs, sizeof(int32_t) * sum_nl, cudaMemcpyHostToDevice, h->stream));

    pt.mark("partition", h->stream);
    // band structure of every local matrix (principal submatrix on the subdomain
    // dofs), found on the device by binary search of the CSR columns in the
    // ascending dof lists
    {
      int32_t* dbw = h->derr + 1;
      CK(cudaMemsetAsync(dbw, 0, sizeof(int32_t), h->stream));
      CKI(launch_band_width(*h, h->A, dbw));
      if (!h->same_pattern) CKI(launch_band_width(*h, h->M, dbw));
      CK(cudaMemcpyAsync(&bw, dbw, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
      CK(cudaStreamSynchronize(h->stream));
    }
    h->B = bw + 1;
    if (h->local_f32()) {
      static const int tiers[] = {16, 24, 32, 40, 48, 64, 96, 128, 152};
      for (int t : tiers)
        if (h->B <= t) {
          h->Bpad = t;
          break;
        }
    }
    if (h->Bpad == 0) {
      // windows above every tier run in the shared-memory kernel, one (B x B) window per warp
      int dev = 0, optin = 0;
      CK(cudaGetDevice(&dev));
      CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
      const size_t esz = h->local_f32() ? sizeof(float) : sizeof(double);
      if ((size_t)(h->B * h->B + 3 * h->B) * esz > (size_t)optin) {
        rc = BPJD_ERR_UNSUPPORTED;
        goto fail;
      }
    }
    // band rows of the local matrices: FP32 (padded to the kernel tier) for FP32
    // local solves, FP64 otherwise
    if (h->local_f32()) {
      const size_t W = (size_t)std::max(h->B, h->Bpad);
      CK(dalloc(*h, &h->bandKf, (size_t)sum_nl * W));
      CK(dalloc(*h, &h->bandMf, (size_t)sum_nl * W));
      if (h->same_pattern) {
        CKI(launch_band_fill(*h, h->A, h->M.val, nullptr, nullptr, h->bandKf, h->bandMf));
      } else {
        CKI(launch_band_fill(*h, h->A, nullptr, nullptr, nullptr, h->bandKf, nullptr));
        CKI(launch_band_fill(*h, h->M, nullptr, nullptr, nullptr, h->bandMf, nullptr));
      }
    } else {
      CK(dalloc(*h, &h->bandK, (size_t)sum_nl * h->B));
      CK(dalloc(*h, &h->bandM, (size_t)sum_nl * h->B));
      if (h->same_pattern) {
        CKI(launch_band_fill(*h, h->A, h->M.val, h->bandK, h->bandM, nullptr, nullptr));
      } else {
        CKI(launch_band_fill(*h, h->A, nullptr, h->bandK, nullptr, nullptr, nullptr));
        CKI(launch_band_fill(*h, h->M, nullptr, h->bandM, nullptr, nullptr, nullptr));
      }
    }
    pt.mark("bands", h->stream);
    // inverse map dof -> packed local positions, ascending subdomain order
    rtp.assign((size_t)n + 1, 0);
    for (int64_t e = 0; e < sum_nl; ++e) rtp[sdofs[e] + 1]++;
    for (int g = 0; g < n; ++g) rtp[g + 1] += rtp[g];
    rtpos.resize((size_t)sum_nl);
    {
      std::vector<int32_t> fill(rtp.begin(), rtp.end() - 1);
      for (int64_t e = 0; e < sum_nl; ++e) rtpos[fill[sdofs[e]]++] = (int32_t)e;
    }
    CK(dalloc(*h, &h->rt_ptr, (size_t)n + 1));
    CK(dalloc(*h, &h->rt_pos, (size_t)sum_nl));
    CK(cudaMemcpyAsync(h->rt_ptr, rtp.data(), sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(h->rt_pos, rtpos.data(), sizeof(int32_t) * sum_nl, cudaMemcpyHostToDevice, h->stream));

    pt.mark("inverse_map", h->stream);
    // scratch and iteration vectors (allocated while the host threads finish the
    // coarse eigensolves)
    {
      // the band factors of every (subdomain, shift) pair are written by the
      // factorisation and read back by the backward sweep; subdomains are taken in
      // chunks whose factors fit the scratch bound
      const size_t esz = h->local_f32() ? sizeof(float) : sizeof(double);
      const size_t lw = (size_t)std::max(h->B, h->Bpad);
      const size_t bound = opts->local_scratch_bytes ? opts->local_scratch_bytes : ((size_t)2 << 30);
      h->chunk_l0.assign(1, 0);
      h->chunk_off.assign(1, 0);
      size_t cur = 0, most = 0;
      for (int l = 0; l < nsub; ++l) {
        const size_t need = esz * (size_t)(sptr[l + 1] - sptr[l]) * k * lw;
        if (cur > 0 && cur + need > bound) {
          h->chunk_l0.push_back(l);
          h->chunk_off.push_back(sptr[l]);
          cur = 0;
        }
        cur += need;
        most = std::max(most, cur);
      }
      h->chunk_l0.push_back(nsub);
      void* p;
      CK(cudaMalloc(&p, most));
      h->allocs.push_back(p);
      h->bytes += most;
      h->Lbuf = p;
      CK(cudaMalloc(&p, esz * (size_t)sum_nl * k));
      h->allocs.push_back(p);
      h->bytes += esz * (size_t)sum_nl * k;
      h->wpk = p;
    }
    CK(dalloc(*h, &h->cH, (size_t)h->nH * k));
    CK(dalloc(*h, &h->aH, (size_t)h->nH * k));
    CK(dalloc(*h, &h->w0, (size_t)h->nH * k));
    {
      double** vecs[] = {&h->X, &h->AX, &h->MX, &h->Xn, &h->AXn, &h->MXn,
                         &h->T, &h->AT, &h->MT, &h->Pd, &h->APd, &h->MPd, &h->rho, &h->Z,
                         &h->Pd2, &h->APd2, &h->MPd2};
      for (double** v : vecs) CK(dalloc(*h, v, (size_t)n * k));
    }
    CK(dalloc(*h, &h->lam, (size_t)2 * k));
    h->partial_cap = (size_t)456 * 96 * 96;
    CK(dalloc(*h, &h->partial, h->partial_cap));
    CK(dalloc(*h, &h->small, (size_t)5 * 96 * 96));
    h->hist_rows = h->max_iter + 1;
    CK(dalloc(*h, &h->hist, (size_t)h->hist_rows * k));
    CK(dalloc(*h, &h->dstat, 1));
    CK(cudaMallocHost(&h->hstat, sizeof(DevStatus)));
    CK(dalloc(*h, &h->dctl, 4));
    CK(dalloc(*h, &h->dlam_fact, (size_t)k));
    {
      double* cb[12] = {h->X, h->AX, h->MX, h->Xn, h->AXn, h->MXn, h->Pd, h->APd, h->MPd, h->Pd2, h->APd2, h->MPd2};
      for (int q = 0; q < 12; ++q) h->canon[q] = cb[q];
    }
    pt.mark("alloc", h->stream);
    // coarse eigenbases (host threads started above)
    {
      EigResult r = eigP.get();
      if ((rc = r.rc) != BPJD_OK) goto fail;
      lamH = std::move(r.lam);
      Phi = std::move(r.Phi);
      if (P0) {
        EigResult r0 = eigP0.get();
        if ((rc = r0.rc) != BPJD_OK) goto fail;
        lam0H = std::move(r0.lam);
        Phi0 = std::move(r0.Phi);
      }
    }
    if ((lamH[k] - lamH[k - 1]) <= 1e-8 * std::fabs(lamH[k]) ||
        (P0 && (lam0H[k] - lam0H[k - 1]) <= 1e-8 * std::fabs(lam0H[k]))) {
      rc = BPJD_ERR_GAP;
      goto fail;
    }
    CK(dalloc(*h, &h->Phi, (size_t)h->nH * h->nH));
    CK(dalloc(*h, &h->lamH, (size_t)h->nH));
    CK(cudaMemcpyAsync(h->Phi, Phi.data(), sizeof(double) * h->nH * h->nH, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(h->lamH, lamH.data(), sizeof(double) * h->nH, cudaMemcpyHostToDevice, h->stream));
    pt.mark("coarse_eig_join", h->stream);
    // initial guess X0 = P0 Phi0[:, :k] (Step 1)
    CK(dalloc(*h, &h->X0, (size_t)n * k));
    CK(dalloc(*h, &h->lam0, (size_t)k));
    if (P0) {
      CK(dalloc(tmp0, &dPhi0, (size_t)h->nH0 * h->nH0));
      CK(cudaMemcpyAsync(dPhi0, Phi0.data(), sizeof(double) * h->nH0 * h->nH0, cudaMemcpyHostToDevice, h->stream));
      CKI(launch_csr_times_dense(dP0, dPhi0, h->nH0, k, h->X0, k, h->stream));
    } else {
      CKI(launch_csr_times_dense(h->P, h->Phi, h->nH, k, h->X0, k, h->stream));
    }
    pt.mark("initial_guess", h->stream);
    CK(cudaStreamSynchronize(h->stream));
    for (void* p : tmp0.allocs) cudaFree(p);
    tmp0.allocs.clear();
    pt.mark("release", h->stream);
    pt.emit();
    h->t_setup = now_s() - t0;
    *out = reinterpret_cast<bpjd_handle*>(h);
    return BPJD_OK;
  fail:
    if (eigP.valid()) eigP.wait();
    if (eigP0.valid()) eigP0.wait();
    cudaStreamSynchronize(h->stream);
    for (void* p : tmp0.allocs) cudaFree(p);
  }
  bpjd_free(reinterpret_cast<bpjd_handle*>(h));
  return rc;
}

namespace {

// sign normalisation: flip each column so its largest-magnitude entry is
// positive (lowest row index wins ties).  Three passes: per-block column
// maxima over contiguous row ranges, one thread per column over the blocks,
// then the flip.  The result does not depend on the order of the comparisons.
constexpr int kSignBlocks = 304;

__device__ __forceinline__ bool sign_better(double a, int ia, double b, int ib) {
  return a > b || (a == b && ia < ib);
}

__global__ void __launch_bounds__(256) k_colmax_partial(int n, int k, const double* __restrict__ X,
                                                        double* __restrict__ partial) {
  __shared__ double bv[256];
  __shared__ int bi[256];
  const int bs = k * (256 / k);  // threads in use; thread t serves column t % k
  const int rows = (n + gridDim.x - 1) / gridDim.x;
  const int r0 = blockIdx.x * rows, r1 = min(n, r0 + rows);
  const int tid = threadIdx.x;
  double best = -1;
  int bidx = n;
  if (tid < bs) {
    const int col = tid % k;
    for (int64_t e = (int64_t)r0 * k + tid; e < (int64_t)r1 * k; e += bs) {
      const double a = fabs(X[e]);
      const int r = (int)(e / k);
      if (sign_better(a, r, best, bidx)) {
        best = a;
        bidx = r;
      }
    }
    (void)col;
  }
  bv[tid] = best;
  bi[tid] = bidx;
  __syncthreads();
  if (tid < k) {
    for (int t = tid + k; t < bs; t += k)
      if (sign_better(bv[t], bi[t], best, bidx)) {
        best = bv[t];
        bidx = bi[t];
      }
    partial[((int64_t)blockIdx.x * k + tid) * 2] = best;
    partial[((int64_t)blockIdx.x * k + tid) * 2 + 1] = (double)bidx;
  }
}

__global__ void k_colmax_final(int nblk, int n, int k, const double* __restrict__ X, const double* partial,
                               double* sign) {
  const int col = threadIdx.x;
  if (col >= k) return;
  double best = -1;
  int bidx = n;
  for (int b = 0; b < nblk; ++b) {
    const double a = partial[((int64_t)b * k + col) * 2];
    const int r = (int)partial[((int64_t)b * k + col) * 2 + 1];
    if (sign_better(a, r, best, bidx)) {
      best = a;
      bidx = r;
    }
  }
  sign[col] = (bidx < n && X[(int64_t)bidx * k + col] < 0) ? -1.0 : 1.0;
}

__global__ void k_col_flip(int64_t nk, int k, const double* __restrict__ sign, double* __restrict__ X) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nk; e += (int64_t)gridDim.x * blockDim.x)
    if (sign[e % k] < 0) X[e] = -X[e];
}

}  // namespace

namespace {

// ---------------------------------------------------------------------------
// The iteration loop captured as one CUDA graph.  A WHILE node repeats a body of
// two BPJD steps (the buffers of the iterate and of the previous update swap
// roles from one step to the next, so the body holds one step of each parity;
// the second sits in an IF node).  Kernels set the conditions on the device:
// after every step k_step_done evaluates the stop test of the new iterate (and
// any local error flag) exactly as the host loop does, and ahead of every
// preconditioner application k_factor_decide chooses between forming the local
// factors anew and reusing them (an IF/ELSE node: factorisation or forward sweep,
// then the shared backward sweep), with the host loop's rule.  No host round
// trip happens until the loop ends.
// ---------------------------------------------------------------------------

// ctl[0]: stored factors valid, ctl[1]: factorisations, ctl[2]: reuses
__global__ void k_factor_decide(int k, const double* __restrict__ lam, double* lam_fact, int32_t* ctl, double tol,
                                cudaGraphConditionalHandle hfac) {
  if (threadIdx.x != 0) return;
  bool reuse = ctl[0] != 0;
  for (int i = 0; reuse && i < k; ++i)
    if (!(fabs(lam[i] - lam_fact[i]) <= tol * fabs(lam[i]))) reuse = false;
  if (!reuse) {
    for (int i = 0; i < k; ++i) lam_fact[i] = lam[i];
    ctl[0] = 1;
    ++ctl[1];
  } else {
    ++ctl[2];
  }
  cudaGraphSetConditional(hfac, reuse ? 0u : 1u);
}

// ctl[3]: steps taken; continue while no stop rule, error or step limit holds
__global__ void k_step_done(const DevStatus* st, const int32_t* derr, int32_t* ctl, int max_iter,
                            cudaGraphConditionalHandle h1, cudaGraphConditionalHandle h2, int set2) {
  if (threadIdx.x != 0) return;
  const int it = ++ctl[3];
  const unsigned go = (!st->converged && derr[0] == 0 && !st->err_breakdown && it < max_iter) ? 1u : 0u;
  cudaGraphSetConditional(h1, go);
  if (set2) cudaGraphSetConditional(h2, go);
}

struct StepBufs {
  double *X, *AX, *MX, *Xn, *AXn, *MXn, *Pc, *APc, *MPc, *Pn, *APn, *MPn, *lam_cur, *lam_nxt;
  void advance(bool p_block) {
    if (p_block) {
      std::swap(Pc, Pn);
      std::swap(APc, APn);
      std::swap(MPc, MPn);
    }
    std::swap(X, Xn);
    std::swap(AX, AXn);
    std::swap(MX, MXn);
    std::swap(lam_cur, lam_nxt);
  }
};

struct CaptureCtx {
  cudaGraphConditionalHandle hfac;  // IF/ELSE of the local factorisation
  cudaStream_t side;                // stream that captures the two branches
  bool decide;                      // the handle can reuse factors: device decision
};

// One BPJD step after the stop test: Algorithm 3.1 Step 2 (preconditioner and
// projection) and Step 3 (Rayleigh-Ritz), the new iterate and, for the 3k space,
// the previous-update block; the buffers advance.  Eager: the host decides factor
// reuse (reuse) and numbers the history row (it); captured (cap): the device does.
int run_step(Handle& h, StepBufs& b, int nb, int it, bool reuse, const CaptureCtx* cap) {
  int rc = BPJD_OK;
  const int k = h.k;
  const int mixed = h.dword() ? 1 : 0;
  double* C1 = h.small;                 // k x k
  double* G = h.small + 2 * 96 * 96;    // m x m
  double* Hm = h.small + 3 * 96 * 96;   // m x m
  double* Crr = h.small + 4 * 96 * 96;  // m x k
  // Step 2: t_i = (I - X X^T M) (B_i)^{-1} r_i.  The local factors of an earlier
  // application are reused while every shift lies within refactor_tol of the
  // one they were formed at (the local solves then differ from exact-shift
  // solves by about that relative amount, far below their FP32 rounding)
  if (cap && cap->decide) {
    k_factor_decide<<<1, 32, 0, h.stream>>>(k, b.lam_cur, h.dlam_fact, h.dctl, h.refactor_tol, cap->hfac);
    h.launches += 1;
    CK(cudaGetLastError());
    {
      cudaStreamCaptureStatus cs;
      cudaGraph_t cg;
      const cudaGraphNode_t* deps = nullptr;
      size_t nd = 0;
      CK(cudaStreamGetCaptureInfo(h.stream, &cs, nullptr, &cg, &deps, nullptr, &nd));
      cudaGraphNodeParams np{};
      np.type = cudaGraphNodeTypeConditional;
      np.conditional.handle = cap->hfac;
      np.conditional.type = cudaGraphCondTypeIf;
      np.conditional.size = 2;
      cudaGraphNode_t node;
      CK(cudaGraphAddNode(&node, cg, deps, nullptr, nd, &np));
      cudaGraph_t branch[2] = {np.conditional.phGraph_out[0], np.conditional.phGraph_out[1]};
      cudaStream_t main = h.stream;
      h.stream = cap->side;
      for (int q = 0; q < 2 && rc == BPJD_OK; ++q) {
        CK(cudaStreamBeginCaptureToGraph(cap->side, branch[q], nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
        const int e = launch_local(h, h.rho, b.lam_cur, q == 0 ? kLocalFactorOnly : kLocalForwardOnly);
        cudaGraph_t done;
        const cudaError_t ee = cudaStreamEndCapture(cap->side, &done);
        if (e != 0 || ee != cudaSuccess) rc = BPJD_ERR_CUDA;
      }
      h.stream = main;
      if (rc != BPJD_OK) goto fail;
      CK(cudaStreamUpdateCaptureDependencies(h.stream, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    }
    CKI(launch_local(h, h.rho, b.lam_cur, kLocalBackwardOnly));
    CKI(launch_coarse_prolong(h, h.rho, b.lam_cur, h.Z));
  } else {
    CKI(launch_precond(h, h.rho, b.lam_cur, h.Z, reuse ? 1 : 0));
  }
  {
    const double* U[1] = {b.MX};
    const double* V[1] = {h.Z};
    if (h.dword())
      CKI(launch_gram(h, 1, U, 1, 1, V, nullptr, 0, C1, nullptr));
    else
      CKI(launch_inner(h, 1, U, 1, V, C1));
    const double* Win[1] = {b.X};
    // double-word: the preconditioned residual is dominated by its component
    // along the iterate, so t is a small difference of large terms
    CKI(launch_combine_rows(h, 1, Win, C1, k, k, h.Z, h.T, -1.0, 0, h.xsplit));
  }
  CKI(launch_spmm(h, h.T, h.AT, h.MT, k, h.xsplit));
  {
    // Step 3: Rayleigh-Ritz in W = U^k + span{t} (+ U^{k-1})
    const double *W[3], *AW[3], *MW[3];
    auto put = [&](int q, const double* w, const double* aw, const double* mw) {
      W[q] = w;
      AW[q] = aw;
      MW[q] = mw;
    };
    // span{X, P} = U^k + U^{k-1}: P is the part of the previous update outside X.
    // Mixed precision: the iterate goes last, so that the upper Gram tiles (the
    // ones formed) pair the correction and P blocks with the exact products of
    // the iterate, never the FP32 products of t or P with the iterate.
    const int bx = mixed ? nb - 1 : 0;  // block of the iterate
    put(bx, b.X, b.AX, b.MX);
    if (nb == 3) {
      put(1, b.Pc, b.APc, b.MPc);
      put(mixed ? 0 : 2, h.T, h.AT, h.MT);
    } else {
      put(mixed ? 0 : 1, h.T, h.AT, h.MT);
    }
    const int m = nb * k;
    if (h.dword()) {
      CKI(launch_gram(h, nb, W, nb, 2, MW, AW, 1, G, Hm));
    } else {
      CKI(launch_inner(h, nb, W, nb, MW, G));
      CKI(launch_inner(h, nb, W, nb, AW, Hm));
    }
    CKI(launch_rr(h, m, G, Hm, b.lam_cur, Crr, b.lam_nxt, it + 1, cap ? h.dctl + 3 : nullptr));
    CKI(launch_combine_rows(h, nb, W, Crr, k, k, nullptr, b.Xn, 1.0, 0, h.xsplit));
    CKI(launch_spmm(h, b.Xn, b.AXn, b.MXn, k, h.xsplit));
    if (h.subspace == BPJD_W_3K) {
      // P_new = the non-iterate blocks of W times their rows of C, with K P_new and
      // M P_new by SpMM (no cancellation)
      if (mixed)
        CKI(launch_combine_rows(h, nb - 1, W, Crr, k, k, nullptr, b.Pn, 1.0, 1, h.xsplit));
      else
        CKI(launch_combine_rows(h, nb - 1, W + 1, Crr + (size_t)k * k, k, k, nullptr, b.Pn, 1.0, 0, h.xsplit));
      CKI(launch_spmm(h, b.Pn, b.APn, b.MPn, k, h.xsplit));
    }
  }
  b.advance(h.subspace == BPJD_W_3K);
  return BPJD_OK;
fail:
  return rc;
}

// Captures the loop (from the buffer state b, steps of nb blocks) into h.gexec.
int build_loop_graph(Handle& h, const StepBufs& b0, int nb) {
  int rc = BPJD_OK;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  cudaStream_t main = h.stream;
  bool capturing = false;
  cudaStream_t cap_stream = nullptr;
  const int64_t launches0 = h.launches;
  const bool decide = h.refactor_tol > 0 && can_reuse_factors(h);
  StepBufs b = b0;
  cudaGraphConditionalHandle hw, hodd, hfa, hfb;
  CKI(prime_kernel_attributes(h));
  for (int q = 0; q < 3; ++q)
    if (!h.gside[q]) {
      cudaStream_t st;
      CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
      h.gside[q] = st;
    }
  CK(cudaGraphCreate(&g, 0));
  CK(cudaGraphConditionalHandleCreate(&hw, g, 1, cudaGraphCondAssignDefault));
  CK(cudaGraphConditionalHandleCreate(&hodd, g, 0, cudaGraphCondAssignDefault));
  CK(cudaGraphConditionalHandleCreate(&hfa, g, 1, cudaGraphCondAssignDefault));
  CK(cudaGraphConditionalHandleCreate(&hfb, g, 1, cudaGraphCondAssignDefault));
  {
    cudaGraphNodeParams wp{};
    wp.type = cudaGraphNodeTypeConditional;
    wp.conditional.handle = hw;
    wp.conditional.type = cudaGraphCondTypeWhile;
    wp.conditional.size = 1;
    cudaGraphNode_t wn;
    CK(cudaGraphAddNode(&wn, g, nullptr, nullptr, 0, &wp));
    cudaGraph_t body = wp.conditional.phGraph_out[0];
    cudaStream_t s1 = (cudaStream_t)h.gside[0], s2 = (cudaStream_t)h.gside[1], s3 = (cudaStream_t)h.gside[2];
    h.stream = s1;
    CK(cudaStreamBeginCaptureToGraph(s1, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    capturing = true;
    cap_stream = s1;
    {
      const CaptureCtx ca{hfa, s2, decide};
      if ((rc = run_step(h, b, nb, 0, false, &ca)) != BPJD_OK) goto fail;
      CKI(launch_residual(h, b.AX, b.MX, b.lam_cur, h.rho));
      k_step_done<<<1, 32, 0, s1>>>(h.dstat, h.derr, h.dctl, h.max_iter, hw, hodd, 1);
      CK(cudaGetLastError());
      // the second step of the body, in an IF node on the first one's verdict
      cudaStreamCaptureStatus cs;
      cudaGraph_t cg;
      const cudaGraphNode_t* deps = nullptr;
      size_t nd = 0;
      CK(cudaStreamGetCaptureInfo(s1, &cs, nullptr, &cg, &deps, nullptr, &nd));
      cudaGraphNodeParams ip{};
      ip.type = cudaGraphNodeTypeConditional;
      ip.conditional.handle = hodd;
      ip.conditional.type = cudaGraphCondTypeIf;
      ip.conditional.size = 1;
      cudaGraphNode_t in;
      CK(cudaGraphAddNode(&in, cg, deps, nullptr, nd, &ip));
      cudaGraph_t second = ip.conditional.phGraph_out[0];
      h.stream = s2;
      CK(cudaStreamBeginCaptureToGraph(s2, second, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
      cap_stream = s2;
      const CaptureCtx cb{hfb, s3, decide};
      if ((rc = run_step(h, b, nb, 0, false, &cb)) != BPJD_OK) goto fail;
      CKI(launch_residual(h, b.AX, b.MX, b.lam_cur, h.rho));
      k_step_done<<<1, 32, 0, s2>>>(h.dstat, h.derr, h.dctl, h.max_iter, hw, hw, 0);
      CK(cudaGetLastError());
      {
        cudaGraph_t done;
        CK(cudaStreamEndCapture(s2, &done));
      }
      cap_stream = s1;
      h.stream = s1;
      CK(cudaStreamUpdateCaptureDependencies(s1, &in, nullptr, 1, cudaStreamSetCaptureDependencies));
    }
    {
      cudaGraph_t done;
      CK(cudaStreamEndCapture(s1, &done));
    }
    capturing = false;
  }
  h.stream = main;
  CK(cudaGraphInstantiate(&ge, g, 0));
  cudaGraphDestroy(g);
  g = nullptr;
  h.gexec = ge;
  // kernels per step: the launches of the two captured steps (with both branches
  // of each factorisation decision, of which one runs), plus the two stop tests
  h.graph_step_launches = (h.launches - launches0 + 2) / 2 - (decide ? 1 : 0);
  h.launches = launches0;
  return BPJD_OK;
fail:
  if (capturing && cap_stream) {
    cudaGraph_t junk = nullptr;
    if (cap_stream != (cudaStream_t)h.gside[0] && cudaStreamEndCapture(cap_stream, &junk) == cudaSuccess && junk)
      cudaGraphDestroy(junk);
    junk = nullptr;
    if (cudaStreamEndCapture((cudaStream_t)h.gside[0], &junk) == cudaSuccess && junk) cudaGraphDestroy(junk);
  }
  cudaGetLastError();
  h.stream = main;
  h.launches = launches0;
  if (g) cudaGraphDestroy(g);
  return rc == BPJD_OK ? BPJD_ERR_CUDA : rc;
}

bool graphs_enabled() {
  const char* e = std::getenv("BPJD_GRAPH");
  return !(e && e[0] == '0');
}

}  // namespace

extern "C" int bpjd_solve(bpjd_handle* hh, double* eigvals, double* eigvecs, int32_t eigvecs_on_device,
                          bpjd_stats* st) {
  if (!hh) return BPJD_ERR_BAD_ARG;
  Handle& h = *reinterpret_cast<Handle*>(hh);
  const int n = h.n, k = h.k;
  const size_t vbytes = sizeof(double) * (size_t)n * k;
  int rc = BPJD_OK;
  const double t0 = now_s();
  // a served solve whose local solves share launches with other requests'
  // takes part in the batching for its whole duration
  struct BatchMember {
    LocalBatcher* b;
    explicit BatchMember(LocalBatcher* bb) : b(bb) {
      if (b) batch_enter(b);
    }
    ~BatchMember() {
      if (b) batch_leave(b);
    }
  } member(h.batch && batch_eligible(h) ? h.batch : nullptr);
  int it = 0;
  bool converged = false;
  // every solve starts from the same buffer assignment (a captured loop refers to it)
  StepBufs b{h.canon[0], h.canon[1], h.canon[2], h.canon[3], h.canon[4], h.canon[5], h.canon[6],
             h.canon[7], h.canon[8], h.canon[9], h.canon[10], h.canon[11], h.lam, h.lam + k};
  double *&X = b.X, *&AX = b.AX, *&MX = b.MX;
  double*& lam_cur = b.lam_cur;
  bool have_prev = false;
  // the loop runs as one CUDA graph once every step has the same shape (eager
  // when profiling or tracing, which need the host between kernels)
  bool graph = !h.host_loop && graphs_enabled() && !h.profile && !trace_on();

  std::vector<double> lam_h((size_t)k);
  h.factors_valid = false;
  h.refactorisations = h.reuses = 0;
  CK(cudaMemsetAsync(h.dstat, 0, sizeof(DevStatus), h.stream));
  CK(cudaMemsetAsync(h.derr, 0, 4 * sizeof(int32_t), h.stream));
  CK(cudaMemcpyAsync(X, h.X0, vbytes, cudaMemcpyDeviceToDevice, h.stream));
  CKI(launch_spmm(h, X, AX, MX, k));
  CKI(launch_rayleigh(h, X, AX, MX, lam_cur));
  CK(cudaMemcpyAsync(h.hist, lam_cur, sizeof(double) * k, cudaMemcpyDeviceToDevice, h.stream));
  for (;;) {
    CKI(launch_residual(h, AX, MX, lam_cur, h.rho));
    CK(cudaMemcpyAsync(h.hstat, h.dstat, sizeof(DevStatus), cudaMemcpyDeviceToHost, h.stream));
    int32_t herr[4];
    CK(cudaMemcpyAsync(herr, h.derr, sizeof(herr), cudaMemcpyDeviceToHost, h.stream));
    if (h.refactor_tol > 0)
      CK(cudaMemcpyAsync(lam_h.data(), lam_cur, sizeof(double) * k, cudaMemcpyDeviceToHost, h.stream));
    CK(cudaStreamSynchronize(h.stream));
    if (herr[0]) {
      rc = local_status(herr[0]);
      break;
    }
    if (h.hstat->err_breakdown) {
      rc = BPJD_ERR_BREAKDOWN;
      break;
    }
    if (trace_on())
      std::fprintf(stderr,
                   "{\"bpjd_iter\": %d, \"max_rel_resid\": %.6e, \"sum_abs_dlambda\": %.6e, \"kept\": %d, "
                   "\"jacobi_sweeps\": %d, \"rr_kcycles\": [%lld, %lld, %lld, %lld, %lld, %lld, %lld, %lld]}\n",
                   it, h.hstat->max_res, h.hstat->sum_dl, h.hstat->kept, h.hstat->sweeps,
                   h.hstat->rr_cycles[0] / 1000, h.hstat->rr_cycles[1] / 1000, h.hstat->rr_cycles[2] / 1000,
                   h.hstat->rr_cycles[3] / 1000, h.hstat->rr_cycles[4] / 1000, h.hstat->rr_cycles[5] / 1000,
                   h.hstat->rr_cycles[6] / 1000, h.hstat->rr_cycles[7] / 1000);
    if (h.hstat->converged) {
      converged = true;
      break;
    }
    if (it >= h.max_iter) {
      rc = BPJD_ERR_NOCONV;
      break;
    }
    const int nb = (h.subspace == BPJD_W_3K && have_prev) ? 3 : 2;
    if (graph && (have_prev || h.subspace == BPJD_W_2K)) {
      // from here every step has nb blocks: the rest of the loop as one graph
      if (!h.gexec && build_loop_graph(h, b, nb) != BPJD_OK) {
        graph = false;  // capture failed: the loop stays on the host
        goto eager;
      }
      {
        int32_t ctl[4] = {h.factors_valid ? 1 : 0, 0, 0, it};
        if (h.factors_valid)
          CK(cudaMemcpyAsync(h.dlam_fact, h.lam_fact.data(), sizeof(double) * k, cudaMemcpyHostToDevice, h.stream));
        CK(cudaMemcpyAsync(h.dctl, ctl, sizeof(ctl), cudaMemcpyHostToDevice, h.stream));
        CK(cudaGraphLaunch((cudaGraphExec_t)h.gexec, h.stream));
        CK(cudaMemcpyAsync(ctl, h.dctl, sizeof(ctl), cudaMemcpyDeviceToHost, h.stream));
        CK(cudaMemcpyAsync(h.hstat, h.dstat, sizeof(DevStatus), cudaMemcpyDeviceToHost, h.stream));
        CK(cudaMemcpyAsync(herr, h.derr, sizeof(herr), cudaMemcpyDeviceToHost, h.stream));
        CK(cudaStreamSynchronize(h.stream));
        const int steps = ctl[3] - it;
        if (steps & 1) b.advance(h.subspace == BPJD_W_3K);  // the graph ends on its second step's buffers otherwise
        it = ctl[3];
        h.refactorisations += ctl[1];
        h.reuses += ctl[2];
        h.launches += h.graph_step_launches * steps;
        if (herr[0])
          rc = local_status(herr[0]);
        else if (h.hstat->err_breakdown)
          rc = BPJD_ERR_BREAKDOWN;
        else if (h.hstat->converged)
          converged = true;
        else
          rc = BPJD_ERR_NOCONV;
      }
      break;
    }
  eager: {
    bool reuse = h.factors_valid && h.refactor_tol > 0;
    for (int i = 0; reuse && i < k; ++i)
      if (!(std::fabs(lam_h[i] - h.lam_fact[i]) <= h.refactor_tol * std::fabs(lam_h[i]))) reuse = false;
    if ((rc = run_step(h, b, nb, it, reuse, nullptr)) != BPJD_OK) goto fail;
    if (!reuse && h.refactor_tol > 0 && can_reuse_factors(h)) {
      h.factors_valid = true;
      h.lam_fact = lam_h;
    }
  }
    have_prev = true;
    ++it;
  }
  if (rc == BPJD_OK || rc == BPJD_ERR_NOCONV) {
    {
      const int nb = std::min(kSignBlocks, std::max(1, n));
      double* part = h.partial;
      double* sgn = h.partial + (size_t)2 * nb * k;
      k_colmax_partial<<<nb, 256, 0, h.stream>>>(n, k, X, part);
      k_colmax_final<<<1, 64, 0, h.stream>>>(nb, n, k, X, part, sgn);
      k_col_flip<<<kSignBlocks, 256, 0, h.stream>>>((int64_t)n * k, k, sgn, X);
      h.launches += 3;
    }
    CK(cudaGetLastError());
    if (eigvals) CK(cudaMemcpyAsync(eigvals, lam_cur, sizeof(double) * k, cudaMemcpyDeviceToHost, h.stream));
    if (eigvecs)
      CK(cudaMemcpyAsync(eigvecs, X, vbytes, eigvecs_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                         h.stream));
    CK(cudaStreamSynchronize(h.stream));
  }
  h.last_iters = it;
  if (trace_on())
    std::fprintf(stderr, "{\"bpjd_local_factorisations\": %lld, \"bpjd_local_reuses\": %lld}\n",
                 (long long)h.refactorisations, (long long)h.reuses);
  if (st) {
    st->iters = it;
    st->converged = converged ? 1 : 0;
    st->max_rel_resid = h.hstat->max_res;
    st->sum_abs_dlambda = h.hstat->sum_dl;
    st->t_setup_s = h.t_setup;
    st->t_solve_s = now_s() - t0;
    st->status = rc;
  }
  return rc;
fail:
  if (st) st->status = rc;
  return rc;
}

extern "C" int bpjd_dims(const bpjd_handle* hh, int32_t* n, int32_t* nH, int32_t* k) {
  if (!hh) return BPJD_ERR_BAD_ARG;
  const Handle& h = *reinterpret_cast<const Handle*>(hh);
  if (n) *n = h.n;
  if (nH) *nH = h.nH;
  if (k) *k = h.k;
  return BPJD_OK;
}

extern "C" int bpjd_layout(const bpjd_handle* hh, int32_t* B, int64_t* sum_nl, int32_t* nsub, int64_t* nnz) {
  if (!hh) return BPJD_ERR_BAD_ARG;
  const Handle& h = *reinterpret_cast<const Handle*>(hh);
  if (B) *B = h.B;
  if (sum_nl) *sum_nl = h.sum_nl;
  if (nsub) *nsub = h.nsub;
  if (nnz) *nnz = h.A.nnz;
  return BPJD_OK;
}

extern "C" int bpjd_spmm(bpjd_handle* hh, const double* X, double* YA, double* YM, int32_t ncols) {
  if (!hh || !X || !YA || !YM || ncols < 1 || ncols > 64) return BPJD_ERR_BAD_ARG;
  Handle& h = *reinterpret_cast<Handle*>(hh);
  if (launch_spmm(h, X, YA, YM, ncols) != 0) return BPJD_ERR_CUDA;
  return BPJD_OK;
}

extern "C" int bpjd_apply_preconditioner(bpjd_handle* hh, const double* rho, const double* lam, double* Z) {
  if (!hh || !rho || !lam || !Z) return BPJD_ERR_BAD_ARG;
  Handle& h = *reinterpret_cast<Handle*>(hh);
  int rc = BPJD_OK;
  int32_t herr[4];
  CK(cudaMemsetAsync(h.derr, 0, 4 * sizeof(int32_t), h.stream));
  h.factors_valid = false;  // the factors are re-formed at the caller's shifts
  CKI(launch_precond(h, rho, lam, Z));
  CK(cudaMemcpyAsync(herr, h.derr, sizeof(herr), cudaMemcpyDeviceToHost, h.stream));
  CK(cudaStreamSynchronize(h.stream));
  return local_status(herr[0]);
fail:
  return rc;
}

extern "C" int bpjd_set_wait_limit(bpjd_handle* hh, int32_t attempts) {
  if (!hh || attempts < 0) return BPJD_ERR_BAD_ARG;
  reinterpret_cast<Handle*>(hh)->wait_limit = attempts;
  return BPJD_OK;
}

extern "C" int bpjd_block_gram(bpjd_handle* hh, int32_t nu, const double* const* U, int32_t nv,
                               const double* const* V, int32_t symmetric, double* out) {
  if (!hh || !U || !V || !out || nu < 1 || nv < 1 || nu > 6 || nv > 6) return BPJD_ERR_BAD_ARG;
  Handle& h = *reinterpret_cast<Handle*>(hh);
  if (nu * h.k > 64 || nv * h.k > 64 || (symmetric && nu != nv)) return BPJD_ERR_BAD_ARG;
  for (int b = 0; b < nu; ++b)
    if (!U[b]) return BPJD_ERR_BAD_ARG;
  for (int b = 0; b < nv; ++b)
    if (!V[b]) return BPJD_ERR_BAD_ARG;
  if (launch_gram(h, nu, U, nv, 1, V, nullptr, symmetric ? 1 : 0, out, nullptr) != 0) return BPJD_ERR_CUDA;
  return BPJD_OK;
}

extern "C" int bpjd_history(const bpjd_handle* hh, double* lam_hist, int32_t cap) {
  if (!hh || !lam_hist || cap < 0) return BPJD_ERR_BAD_ARG;
  const Handle& h = *reinterpret_cast<const Handle*>(hh);
  int rows = std::min(cap, std::min(h.last_iters + 1, h.hist_rows));
  if (rows <= 0) return 0;
  if (cudaMemcpy(lam_hist, h.hist, sizeof(double) * rows * h.k, cudaMemcpyDeviceToHost) != cudaSuccess)
    return BPJD_ERR_CUDA;
  return rows;
}

extern "C" int bpjd_profile(bpjd_handle* hh, int32_t enable) {
  if (!hh) return BPJD_ERR_BAD_ARG;
  Handle& h = *reinterpret_cast<Handle*>(hh);
  prof_flush(h);
  h.profile = enable != 0;
  for (int c = 0; c < BPJD_PROF_N; ++c) {
    h.prof_ms[c] = 0;
    h.prof_count[c] = 0;
  }
  h.launches = 0;
  return BPJD_OK;
}

extern "C" int bpjd_profile_read(bpjd_handle* hh, double* ms, int64_t* count, int64_t* launches) {
  if (!hh) return BPJD_ERR_BAD_ARG;
  Handle& h = *reinterpret_cast<Handle*>(hh);
  prof_flush(h);
  for (int c = 0; c < BPJD_PROF_N; ++c) {
    if (ms) ms[c] = h.prof_ms[c];
    if (count) count[c] = h.prof_count[c];
  }
  if (launches) *launches = h.launches;
  return BPJD_OK;
}

extern "C" size_t bpjd_device_bytes(const bpjd_handle* hh) {
  if (!hh) return 0;
  return reinterpret_cast<const Handle*>(hh)->bytes;
}
