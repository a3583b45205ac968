// Internal declarations shared by the library's translation units.
#ifndef BPJD_INTERNAL_H_
#define BPJD_INTERNAL_H_

#include <cstddef>
#include <cstdint>
#include <vector>

#include "bpjd.h"

#include <cuda_runtime.h>

namespace bpjd {

// Device-side status written by the reduction kernels; copied to pinned host
// memory once per iteration.
struct DevStatus {
  double max_res;       // max relative residual of the current iterate
  double sum_dl;        // sum |lambda^{k+1} - lambda^k| of the last Rayleigh-Ritz step
  int32_t converged;    // stop rule satisfied
  int32_t err_local;    // a local pivot was <= 0
  int32_t err_breakdown;// Rayleigh-Ritz kept fewer than k directions
  int32_t kept;         // directions kept by the last Rayleigh-Ritz step
  int32_t sweeps;       // Jacobi sweeps of the last Rayleigh-Ritz step
  long long rr_cycles[8];  // SM cycles spent in the phases of the last Rayleigh-Ritz step
  double res[64];       // per-column relative residuals
};

struct CsrDev {
  int32_t n_rows = 0, n_cols = 0;
  int64_t nnz = 0;
  int64_t* row_ptr = nullptr;
  int32_t* col = nullptr;
  double* val = nullptr;
};

struct LocalBatcher;

struct Handle {
  // ---- sizes and options
  int32_t n = 0, nH = 0, nH0 = 0, k = 0, nsub = 0;
  int32_t B = 0;            // band window: lower bandwidth + 1 (max over subdomains)
  int32_t Bpad = 0;         // register-window size of the FP32 local kernel (0: shared-memory kernel)
  int64_t sum_nl = 0;       // sum of local sizes
  int32_t max_nl = 0;
  int32_t precision = BPJD_FP64, subspace = BPJD_W_2K, stop_rule = BPJD_STOP_RESIDUAL;
  // local band factorisations and solves in FP32 (BPJD_MIXED, BPJD_MIXED_LOCAL)
  bool local_f32() const { return precision == BPJD_MIXED || precision == BPJD_MIXED_LOCAL; }
  // SpMM, Gram matrices and row combinations in double-word arithmetic (BPJD_MIXED)
  bool dword() const { return precision == BPJD_MIXED; }
  int32_t max_iter = 500;
  double tol = 1e-8, drop_tol = 1e-10;
  int32_t wait_limit = 1 << 22;  // attempts of every bounded device-side wait (bpjd_set_wait_limit)
  cudaStream_t stream = nullptr;

  // ---- matrices
  CsrDev A, M;              // M may share A's pattern arrays (same_pattern)
  bool same_pattern = false;
  float2* Asplit = nullptr;  // (hi, lo) float pairs of K and M values (double-word SpMM)
  float2* Msplit = nullptr;
  float2* xsplit = nullptr;  // n x k (hi, lo) split of the block the next double-word SpMM reads
  float2* Psplit = nullptr;  // (hi, lo) split of P's values (FP32 prolongation of FP32 preconditioners)
  CsrDev P, PT;             // coarse interpolation and its transpose
  double* Phi = nullptr;    // n_H x n_H row-major, M_H-orthonormal eigenvectors
  double* lamH = nullptr;   // n_H ascending
  double* X0 = nullptr;     // initial guess n x k
  double* lam0 = nullptr;   // k

  // ---- subdomains
  int64_t* sub_ptr = nullptr;
  int32_t* sub_dofs = nullptr;
  int32_t* rt_ptr = nullptr;   // n + 1: inverse map dof -> packed local positions
  int32_t* rt_pos = nullptr;   // sum_nl, packed position sub_ptr[l] + p
  double* bandK = nullptr;     // FP64 local solves: sum_nl x B, row p holds K_l(p, p-B+1 .. p)
  double* bandM = nullptr;
  float* bandKf = nullptr;     // FP32 local solves: sum_nl x max(B, Bpad), the same rows
  float* bandMf = nullptr;     //   left-padded with zeros

  // ---- scratch
  void* Lbuf = nullptr;        // band factors of one chunk of subdomains (FP32 or FP64)
  std::vector<int32_t> chunk_l0;   // chunk c = subdomains [chunk_l0[c], chunk_l0[c + 1])
  std::vector<int64_t> chunk_off;  // sub_ptr of each chunk's first subdomain (record base)
  double refactor_tol = 0.0;       // reuse the local factors while every shift stays within this (0: never)
  bool host_loop = false;          // the host drives every step (no loop graph)
  bool factors_valid = false;      // Lbuf holds the factors of every pair, formed at the shifts lam_fact
  std::vector<double> lam_fact;    // host copy of the shifts of the stored factors
  int64_t refactorisations = 0, reuses = 0;  // local applications of the last solve, by kind

  // ---- the iteration loop as one CUDA graph (conditional nodes decide on the device)
  int32_t* dctl = nullptr;      // device: [0] stored factors valid, [1] factorisations, [2] reuses, [3] steps
  double* dlam_fact = nullptr;  // device copy of the shifts of the stored factors (k)
  void* gexec = nullptr;        // cudaGraphExec_t of the loop, built on first use
  void* gside[3] = {nullptr, nullptr, nullptr};  // streams that capture the conditional bodies
  int64_t graph_step_launches = 0;  // kernels launched per captured step
  double* canon[12] = {};       // buffer assignment at the start of every solve (X, AX, MX, Xn, ..., MPd2)
  void* wpk = nullptr;         // packed local solutions sum_nl x k (FP32 or FP64)
  double* cH = nullptr;        // n_H x k coarse restriction
  double* aH = nullptr;        // n_H x k coarse coordinates
  double* w0 = nullptr;        // n_H x k coarse correction

  // ---- iteration vectors, n x k row-major FP64
  double *X = nullptr, *AX = nullptr, *MX = nullptr;
  double *Xn = nullptr, *AXn = nullptr, *MXn = nullptr;   // next iterate
  double *T = nullptr, *AT = nullptr, *MT = nullptr;
  double *Pd = nullptr, *APd = nullptr, *MPd = nullptr;   // previous-update block (3k)
  double *Pd2 = nullptr, *APd2 = nullptr, *MPd2 = nullptr;
  double *rho = nullptr, *Z = nullptr;
  double* lam = nullptr;       // k
  double* partial = nullptr;   // block partial sums
  size_t partial_cap = 0;      // capacity of partial in doubles
  double* small = nullptr;     // small dense matrices (Gram, C, ...)
  double* hist = nullptr;      // (max_iter + 1) x k Ritz values
  int32_t hist_rows = 0;
  DevStatus* dstat = nullptr;
  DevStatus* hstat = nullptr;  // pinned host mirror
  int32_t* derr = nullptr;     // device error flags

  // ---- serving: local solves packed with those of other handles (batch.cpp)
  LocalBatcher* batch = nullptr;
  void* batch_ev = nullptr;  // cudaEvent_t: this handle's work up to the local solves

  // ---- instrumentation
  bool profile = false;
  std::vector<void*> ev_pool;  // cudaEvent_t
  size_t ev_used = 0;
  std::vector<int> ev_cls;     // class of each recorded pair
  double prof_ms[BPJD_PROF_N] = {0};
  int64_t prof_count[BPJD_PROF_N] = {0};
  int64_t launches = 0;        // kernels launched by the library

  size_t bytes = 0;            // device bytes held
  std::vector<void*> allocs;   // every device allocation (freed in bpjd_free)
  int64_t n_partial_blocks = 0;
  int last_iters = 0;
  double t_setup = 0;          // seconds spent in bpjd_setup
};

// Status of the local-solve error bits (h.derr[0]): a wait that ran out (or copies
// that never completed) outranks a non-positive pivot, which it may have caused.
inline int local_status(int32_t bits) {
  if (bits & 6) return BPJD_ERR_TIMEOUT;
  if (bits & 1) return BPJD_ERR_LOCAL_INDEFINITE;
  return BPJD_OK;
}

// Records an event pair around a kernel-class launch when profiling is on.
struct ProfScope {
  Handle& h;
  int cls;
  size_t idx;
  bool on;
  ProfScope(Handle& hh, int c);
  ~ProfScope();
};
// Resolves recorded event pairs into prof_ms/prof_count (synchronises the stream).
void prof_flush(Handle& h);

// kernels.cu: raises a kernel's dynamic shared-memory limit to the device
// maximum, once per (kernel, device)
int allow_dynamic_smem(const void* kern);

// dense.cpp
// nvec < n: every eigenvalue, eigenvectors of the lowest nvec only (the other
// columns of V / Phi are zero)
int sym_eig_host(int n, std::vector<double> A, std::vector<double>& lam, std::vector<double>& V, int nvec = -1);
int gen_eig_host(int n, const std::vector<double>& K, const std::vector<double>& M, std::vector<double>& lam,
                 std::vector<double>& Phi, int nvec = -1);

// kernels.cu launchers (all asynchronous on h.stream; return cudaError_t as int)
// Xs (double-word path only): the (hi, lo) split of X written by the kernel
// that produced it, read instead of splitting X per nonzero
int launch_spmm(Handle& h, const double* X, double* YA, double* YM, int ncols, const float2* Xs = nullptr);
int launch_csr_times_dense(const CsrDev& P, const double* D, int ldd, int ncols, double* Y, int ldy,
                           cudaStream_t s);
int launch_residual(Handle& h, const double* AX, const double* MX, const double* lam, double* rho);
int launch_rayleigh(Handle& h, const double* X, const double* AX, const double* MX, double* lam);
// reuse = 1: the stored factors are current for lam (forward and backward sweeps only)
int launch_precond(Handle& h, const double* rho, const double* lam, double* Z, int reuse = 0);
// the two parts of launch_precond; modes of launch_local:
enum { kLocalFull = 0, kLocalReuse = 1, kLocalFactorOnly = 2, kLocalForwardOnly = 3, kLocalBackwardOnly = 4 };
int launch_local(Handle& h, const double* rho, const double* lam, int mode);
int launch_coarse_prolong(Handle& h, const double* rho, const double* lam, double* Z);
// Local solves of n handles of one window tier (Bpad) in grouped launches on
// stream s: handles with refactor[j] = 1 factorise at their shifts (with the
// fused forward sweep; the wide tiers 64, 96 and 152 in one launch per handle),
// the others sweep forward on their stored factors, then every handle sweeps
// backward.  Every handle satisfies can_reuse_factors; n <= kGroupedMax.
constexpr int kGroupedMax = 16;
int launch_local_grouped(Handle* const* hs, const double* const* rho, const double* const* lam,
                         const int* refactor, int n, cudaStream_t s);
// batch.cpp: the serving path's packing of local solves across handles.  A
// handle with h.batch set (and the host-driven loop) hands its local solves to
// batch_local, which returns once they are launched, with the handle's stream
// ordered after them; batch_enter / batch_leave bracket every solve.
LocalBatcher* batch_create(int wait_us);
void batch_free(LocalBatcher* b);
void batch_enter(LocalBatcher* b);
void batch_leave(LocalBatcher* b);
bool batch_eligible(const Handle& h);
int batch_local(LocalBatcher* b, Handle& h, const double* rho, const double* lam, bool refactor);
void batch_stats(const LocalBatcher* b, int64_t* flushes, int64_t* jobs);
// whether this handle's local kernels can reuse stored factors (records of every pair resident)
bool can_reuse_factors(const Handle& h);
// sets the dynamic shared-memory limits of every kernel the handle's iterations launch
// (done before a stream capture, where the attribute calls are best avoided)
int prime_kernel_attributes(Handle& h);
int launch_inner(Handle& h, int p, const double* const* U, int q, const double* const* V, double* out);
// double-word block inner products: out1 = U^T V1 (and out2 = U^T V2 when nv = 2);
// sym = 1 requires U^T V symmetric (mu == mv) and forms the upper tiles only
int launch_gram(Handle& h, int nu, const double* const* U, int nvb, int nv, const double* const* V1,
                const double* const* V2, int sym, double* out1, double* out2);
// doubles of partial sums launch_gram_raw needs (one right-hand block set)
size_t gram_partial_doubles(int64_t n, int k, int nu, int nvb, int sym);
// the same with an explicit scratch buffer for the per-block partial sums
// (capacity in doubles) and stream; no handle needed
int launch_gram_raw(int64_t n, int k, int nu, const double* const* U, int nvb, int nv, const double* const* V1,
                    const double* const* V2, int sym, double* out1, double* out2, double* partial,
                    size_t partial_capacity, cudaStream_t stream);
// consistency_only (mixed precision): FP32 update, for the previous-update block P;
// split_out (double-word path only): also the (hi, lo) split of every output value
int launch_combine_rows(Handle& h, int nin, const double* const* Win, const double* C, int ldc,
                        int csub, const double* Zadd, double* out, double alpha, int consistency_only = 0,
                        float2* split_out = nullptr);
// hist_row: history row of the Ritz values (host count), or d_row != NULL: the
// device step counter + 1 (captured iterations)
int launch_rr(Handle& h, int m, const double* G, const double* Hm, const double* lam_old, double* C,
              double* lam_new, int hist_row, const int32_t* d_row = nullptr);
int launch_validate_csr(const CsrDev& c, int32_t* flag, cudaStream_t s);
int launch_same_pattern(const CsrDev& a, const CsrDev& m, int32_t* flag, cudaStream_t s);
int launch_validate_part(Handle& h, int32_t* flag);
// transpose of a validated CSR (rows of the result in ascending original row) into
// caller-allocated arrays (n_cols + 1, nnz, nnz); at most kTransposeMaxCols columns
constexpr int kTransposeMaxCols = 24576;
int launch_csr_transpose(const CsrDev& a, int64_t* rpT, int32_t* ciT, double* valT, cudaStream_t s);
int launch_band_width(Handle& h, const CsrDev& c, int32_t* bw);
int launch_split_values(const double* v, int64_t nnz, float2* out, cudaStream_t s);
// band rows of the local matrices of c (and of a second matrix with c's pattern,
// values val2): FP32 rows of width max(B, Bpad) into outf / outf2 when outf is
// set, else FP64 rows of width B into out / out2
int launch_band_fill(Handle& h, const CsrDev& c, const double* val2, double* out, double* out2, float* outf,
                     float* outf2);
int launch_galerkin(const CsrDev& A, const CsrDev& Msp, const CsrDev& P, const CsrDev& PT, double* KH,
                    double* MH, cudaStream_t s);

}  // namespace bpjd

#endif  // BPJD_INTERNAL_H_
