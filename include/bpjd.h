/*
 * bpjd.h -- C ABI of the GB300 two-level BPJD eigensolver.
 *
 * The library computes the lowest k eigenpairs (multiple and clustered ones
 * included) of the symmetric-definite pencil K x = lambda M x arising from a
 * conforming finite-element discretisation of a symmetric elliptic operator
 * (Section 2.2), with the two-level block preconditioned Jacobi-Davidson
 * method of Section 3 (Algorithm 3.1) and its overlapping-Schwarz
 * preconditioner (Eq. (3.3)):
 *
 *   (B_i^k)^{-1} = (A^H - lambda_i^k)^{-1} Q_{s+1}^H Q^H
 *                  + sum_l (A^(l) - lambda_i^k)^{-1} Q^(l).
 *
 * Conventions shared by every entry point
 *   - Sparse matrices are 0-based CSR with int64 row pointers, int32 column
 *     indices sorted ascending within a row and no duplicates, float64 values.
 *   - Dense blocks of k vectors are ROW-MAJOR n x k ("k contiguous per dof").
 *   - Pointers documented as "device" must be CUDA device pointers of the
 *     current device; "host" pointers are ordinary host memory.
 *   - Every function returns BPJD_OK (0) or a negative BPJD_ERR_* code; no
 *     exception or abort crosses the ABI.  bpjd_status_string() names codes.
 *   - A handle may be used from one host thread at a time; all of its GPU
 *     work is ordered on the stream given in bpjd_opts.stream.
 */
#ifndef BPJD_H_
#define BPJD_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define BPJD_OK                    0
#define BPJD_ERR_BAD_ARG          -1  /* null pointer, k < 1, sizes inconsistent */
#define BPJD_ERR_CSR_INVALID      -2  /* row_ptr not monotone, column out of range/unsorted */
#define BPJD_ERR_MAP_INVALID      -3  /* subdomain dof list unsorted / out of range / empty */
#define BPJD_ERR_K_TOO_LARGE      -4  /* k >= dim V^H: Section 3 needs s < dim(V^H) */
#define BPJD_ERR_GAP              -5  /* lambda_k^H == lambda_{k+1}^H: Assumption 1 fails on V^H */
#define BPJD_ERR_LOCAL_INDEFINITE -6  /* a shifted local matrix K_l - lambda_i M_l has a
                                         non-positive pivot (Eq. (3.1) violated) */
#define BPJD_ERR_BREAKDOWN        -7  /* Rayleigh-Ritz basis lost rank below k */
#define BPJD_ERR_NOCONV           -8  /* max_iter reached before the stop rule held */
#define BPJD_ERR_OOM              -9  /* device allocation failed */
#define BPJD_ERR_CUDA            -10  /* a CUDA runtime call failed */
#define BPJD_ERR_UNSUPPORTED     -11  /* option outside what the library implements, or a local
                                        band window the shared-memory kernel cannot hold
                                        (FP64 above 168, mixed above 240 on a 227 KB SM) */
#define BPJD_ERR_TOO_LARGE       -12  /* request exceeds a fixed capacity (allocation-free entry point)
                                         or, alone, the memory budget of a server */
#define BPJD_ERR_TIMEOUT         -13  /* a bounded device-side wait ran out: a local-solve kernel
                                         waited bpjd_set_wait_limit() attempts for a bulk copy
                                         into shared memory, gave up and returned (its results
                                         are invalid; the handle and the context stay usable) */

/* ---- option values ----------------------------------------------------- */
#define BPJD_FP64        0  /* every step in FP64 */
#define BPJD_MIXED       1  /* the preconditioner in FP32: local band factorisations
                               and solves (tensor cores up to window 152) and the
                               prolongation-add (the coarse solve stays FP64); SpMM,
                               projections, Gram matrices and the Ritz-vector update
                               in double-word FP32 pairs (about 2^-46 relative,
                               FP64-class); residuals and Rayleigh-Ritz in FP64 */
#define BPJD_MIXED_LOCAL 2  /* the preconditioner in FP32 as in BPJD_MIXED, every
                               other step in native FP64: for
                               operators whose residual amplifies product rounding
                               beyond the double-word floor (fourth-order problems on
                               fine meshes: |K||x| / |Kx| ~ 1e8) */

#define BPJD_W_2K        0  /* W^{k+1} = U^k + span{t_i}           (Remark 3.1) */
#define BPJD_W_3K        1  /* W^{k+1} = U^{k-1} + U^k + span{t_i} (Remark 3.1) */

#define BPJD_STOP_RESIDUAL 0 /* every ||K x_i - lambda_i M x_i||_2 / (|lambda_i| ||M x_i||_2) <= tol */
#define BPJD_STOP_DLAMBDA  1 /* sum_i |lambda_i^{k+1} - lambda_i^k| < tol (Algorithm 3.1 Step 4) */

/* ---- input descriptors ------------------------------------------------- */
typedef struct {
  int32_t n_rows, n_cols;
  int64_t nnz;
  const int64_t* row_ptr;   /* n_rows + 1 */
  const int32_t* col_idx;   /* nnz */
  const double*  val;       /* nnz */
} bpjd_csr;

/* Overlapping subdomains Omega_l' (Section 2.3): the dofs of V^(l), i.e. the
 * fine dofs strictly inside Omega_l', ascending, for l = 0..n_sub-1.  The
 * local matrices are the principal submatrices K_l = R_l K R_l^T and
 * M_l = R_l M R_l^T; they are factorised as banded matrices, so an ordering
 * with small bandwidth (lexicographic on a box) keeps the local cost low. */
typedef struct {
  int32_t n_sub;
  const int64_t* sub_ptr;   /* n_sub + 1, sub_ptr[0] = 0 */
  const int32_t* sub_dofs;  /* sub_ptr[n_sub] */
  const int32_t* sub_color; /* n_sub, or NULL; same colour => disjoint (Assumption 2).
                               Informational: the prolongation-add is a gather over
                               an inverse map and needs no colouring. */
  int32_t n_colors;
} bpjd_partition;

typedef struct {
  int32_t k;                /* wanted eigenpairs (the paper's s), 1 <= k <= 32 */
  int32_t precision;        /* BPJD_FP64 | BPJD_MIXED | BPJD_MIXED_LOCAL */
  int32_t subspace;         /* BPJD_W_2K | BPJD_W_3K */
  int32_t stop_rule;        /* BPJD_STOP_RESIDUAL | BPJD_STOP_DLAMBDA */
  double  tol;              /* threshold of the stop rule (default 1e-8) */
  int32_t max_iter;         /* Rayleigh-Ritz steps at most (default 500) */
  double  drop_tol;         /* Rayleigh-Ritz drops Gram eigen-directions below
                               drop_tol * max (default 1e-10) */
  double  H, delta;         /* subdomain diameter and overlap (metadata for logs) */
  int32_t inputs_on_device; /* 1: all pointers of A, M, P, P0 and the partition
                               are device pointers; 0: host pointers */
  void*   stream;           /* cudaStream_t for all work; NULL = legacy default stream */
  size_t  local_scratch_bytes; /* bound on the device scratch that holds the band factors
                               of the local solves (0: default 2 GiB).  Subdomains are
                               solved in chunks whose factors fit; a chunk holds at least
                               one subdomain, so the scratch may exceed the bound by one
                               subdomain's factors (n_l k (B + 8) FP32 values) */
  double  local_refactor_tol;  /* the local band factors of K_l - lambda_i M_l are formed
                               anew only when some shift moved by more than this relative
                               amount since they were formed; otherwise the stored factors
                               are reused (forward and backward sweeps only).  0: default,
                               3e-4 with FP32 local solves, exact shifts (a factorisation
                               at every application, as in Eq. (3.3)) for BPJD_FP64;
                               < 0: exact shifts always.  Reuse needs every factor of one
                               application resident (one chunk) and a band window of at
                               most 152 */
  int32_t host_loop;           /* 0 (default): after its first steps the iteration loop runs
                               as one CUDA graph per handle, the stop test evaluated on the
                               device; 1: the host drives every step (one synchronisation
                               per step).  Results are bit-identical either way */
} bpjd_opts;

typedef struct {
  int32_t iters;            /* Rayleigh-Ritz steps taken */
  int32_t converged;        /* 1 if the stop rule held */
  double  max_rel_resid;    /* of the returned pairs */
  double  sum_abs_dlambda;  /* of the last step */
  double  t_setup_s, t_solve_s;
  int32_t status;
} bpjd_stats;

typedef struct bpjd_handle bpjd_handle;

/* Fills *o with the defaults listed above (k = 1). */
void bpjd_default_opts(bpjd_opts* o);

const char* bpjd_status_string(int code);

/*
 * bpjd_setup -- build the device-resident solver state (Algorithm 3.1 Step 1).
 *
 * A, M : n x n stiffness and mass matrices (symmetric; M SPD).
 * P    : n x n_H nodal interpolation V^H -> V^h (column c = fine values of the
 *        c-th coarse basis function); defines Q^H and A^H by Galerkin products
 *        K_H = P^T K P, M_H = P^T M P (Section 3).
 * P0   : n x n_H0 interpolation from the grid H~ = H/2^tau used for the initial
 *        eigenproblem of Step 1, or NULL to use P (tau = 0).
 * part : overlapping subdomains.
 * Inputs are only read during the call; the handle owns every device buffer
 * until bpjd_free.  Errors: BAD_ARG, CSR_INVALID, MAP_INVALID, K_TOO_LARGE,
 * GAP, OOM, CUDA; on error *out is NULL and nothing leaks.
 */
int bpjd_setup(const bpjd_csr* A, const bpjd_csr* M, const bpjd_csr* P, const bpjd_csr* P0,
               const bpjd_partition* part, const bpjd_opts* opts, bpjd_handle** out);

/*
 * bpjd_solve -- run Algorithm 3.1 Steps 2-4 from the Step 1 initial guess.
 *
 * eigvals : k doubles (host), ascending Ritz values, or NULL.
 * eigvecs : n x k row-major doubles, b-orthonormal (X^T M X = I), or NULL;
 *           host memory if eigvecs_on_device == 0, device memory otherwise.
 * st      : statistics, or NULL.
 * May be called repeatedly; every call restarts from the initial guess.
 * Errors: LOCAL_INDEFINITE, BREAKDOWN, NOCONV (results still written), TIMEOUT,
 * CUDA.
 */
int bpjd_solve(bpjd_handle* h, double* eigvals, double* eigvecs, int32_t eigvecs_on_device,
               bpjd_stats* st);

/* Releases every resource of the handle (NULL is a no-op). */
void bpjd_free(bpjd_handle* h);

/* ---- hot-path steps on device buffers (for tests and measurements) ----- */

/* n, n_H and k of a handle. */
int bpjd_dims(const bpjd_handle* h, int32_t* n, int32_t* n_coarse, int32_t* k);

/* Local-solve layout: band window B (lower bandwidth + 1, maximum over the
 * subdomains), sum of the local sizes n_l, number of subdomains, and nnz of K. */
int bpjd_layout(const bpjd_handle* h, int32_t* band_window, int64_t* sum_local, int32_t* n_sub, int64_t* nnz);

/* Y_A = K X and Y_M = M X for a device n x ncols row-major X (1 <= ncols <= 64).
 * Y_A, Y_M: device n x ncols.  Ordered on the handle's stream. */
int bpjd_spmm(bpjd_handle* h, const double* X, double* YA, double* YM, int32_t ncols);

/* z_i = (B_i)^{-1} rho_i (Eq. (3.3)) for the k columns of the device n x k
 * array rho, with shifts lam (device, k doubles).  Z: device n x k.  Uses the
 * handle's precision.  Returns LOCAL_INDEFINITE if a local pivot is <= 0,
 * TIMEOUT if a bounded wait of the local solves ran out. */
int bpjd_apply_preconditioner(bpjd_handle* h, const double* rho, const double* lam, double* Z);

/* Block inner products out = U^T V in double-word (FP32-pair, FP64-class)
 * arithmetic, the product used for the Gram matrices W^T M W, W^T K W of the
 * Rayleigh-Ritz step (Eq. (3.6)) and the projection coefficients of Eq. (3.5).
 * U: host array of nu device pointers, each an n x k row-major FP64 block
 * (k = the handle's k, n = its size); V likewise with nv blocks.  out: device,
 * (nu k) x (nv k) row-major FP64.  symmetric = 1 asserts U^T V is symmetric
 * (nu == nv) and forms only the upper half.  (nu k), (nv k) <= 64.  Uses the
 * handle's scratch; ordered on the handle's stream. */
int bpjd_block_gram(bpjd_handle* h, int32_t nu, const double* const* U, int32_t nv, const double* const* V,
                    int32_t symmetric, double* out);

/*
 * bpjd_block_gram_noalloc -- bpjd_block_gram without a handle and without any
 * device allocation.  (The paper has no counterpart: this is an interface for
 * callers, not a step of the method.)
 *
 * For callers that cannot call cudaMalloc: e.g. a host application that owns all
 * device memory through its own pool or pre-reserved arena and hands libraries
 * only the buffers they operate on, or a latency-critical loop that must not
 * pay the implicit device synchronisation of an allocation.  The caller passes
 * the inputs and the output; the per-block partial sums live in a file-scope
 * static device array of 8 MiB (2^20 doubles), reserved on every GPU that
 * loads the library until the process exits.  The partial sums need
 * 16 * ntiles * min(456, ceil(n / 32)) doubles, ntiles being the number of
 * 4 x 4 output tiles formed (upper ones only when symmetric).
 *
 * n, k  : rows and columns of every block; U: host array of nu device
 *         pointers (n x k row-major FP64 each), V likewise with nv; out: device
 *         (nu k) x (nv k) row-major FP64; stream: cudaStream_t or NULL.
 * symmetric, size limits and arithmetic as for bpjd_block_gram.
 * Errors: BAD_ARG; TOO_LARGE if n > 2^31 - 1 (rows are indexed with 32-bit
 * integers) or if the partial sums of this (n, k, nu, nv) do not fit the static
 * array (both checked on the host before any launch); CUDA.
 * The first call on a device looks up the device address of the static array
 * (cudaGetSymbolAddress, with that device current); make that first call before
 * any stream capture.  All calls share the one array: calls that overlap on
 * the GPU (other streams, other host threads) race and give wrong results, so
 * order them.  The array keeps the last call's contents; nothing in it has to
 * start at zero, because every partial sum a call reads it has written first.
 */
int bpjd_block_gram_noalloc(int64_t n, int32_t k, int32_t nu, const double* const* U, int32_t nv,
                            const double* const* V, int32_t symmetric, double* out, void* stream);

/* Attempts of every bounded device-side wait of the handle's kernels (the local
 * solves spin on an mbarrier until a bulk copy into shared memory completes;
 * each attempt is one mbarrier.try_wait, which may suspend briefly) before the
 * kernel gives up, flags BPJD_ERR_TIMEOUT for the call and returns after its
 * copies in flight have landed.  Default 1 << 22 (far beyond any normal copy);
 * 0 gives up at once, which exercises the timeout path without a hang.
 * Errors: BAD_ARG (NULL handle or attempts < 0). */
int bpjd_set_wait_limit(bpjd_handle* h, int32_t attempts);

/* Ritz values of every Rayleigh-Ritz step of the last solve (row j = step j,
 * row 0 = initial guess), host array of cap x k doubles; returns rows written. */
int bpjd_history(const bpjd_handle* h, double* lam_hist, int32_t cap);

/* Device bytes held by the handle. */
size_t bpjd_device_bytes(const bpjd_handle* h);

/* ---- instrumentation --------------------------------------------------- */
/* Kernel classes timed when profiling is on. */
#define BPJD_PROF_LOCAL     0  /* banded local factorisation + solves (Q^(l), (B_{l,i})^{-1}) */
#define BPJD_PROF_COARSE    1  /* coarse restriction, spectral solve, expansion */
#define BPJD_PROF_PROLONG   2  /* prolongation-add of coarse and local corrections */
#define BPJD_PROF_SPMM      3  /* K X and M X */
#define BPJD_PROF_INNER     4  /* block inner products (projection, Gram matrices) */
#define BPJD_PROF_COMBINE   5  /* row-wise block updates (projection, Ritz vectors) */
#define BPJD_PROF_RR        6  /* small Rayleigh-Ritz eigenproblem */
#define BPJD_PROF_RESID     7  /* residuals and norms */
#define BPJD_PROF_N         8

/* enable = 1 records a CUDA event pair around every kernel class launch on the
 * handle's stream (small overhead); 0 stops.  Resets the accumulated data. */
int bpjd_profile(bpjd_handle* h, int32_t enable);

/* Accumulated device time (ms) and launch count per class since the last
 * bpjd_profile call, and the total number of kernels the library launched on
 * the handle (counted with or without profiling).  Arrays: BPJD_PROF_N entries;
 * any pointer may be NULL. */
int bpjd_profile_read(bpjd_handle* h, double* ms, int64_t* count, int64_t* kernel_launches);

/* ---- problem generation helpers (host) --------------------------------- */

/* Mesh description of the model problems (Section 2.1, Section 6):
 *   kind 0 = P1 triangles on a uniform nx x ny grid, squares split SW->NE;
 *   kind 1 = P1 tetrahedra, each cube of a uniform grid split into the six
 *            Kuhn tetrahedra;
 *   kind 2 = trilinear bricks (constant kappa only);
 *   kind 3 = the clamped plate Delta^2 u = lambda u (Section 2.1, m = 2) with
 *            Morley triangles on the square grid of kind 0 (nx = ny, equal
 *            sides, kappa NULL).  Dofs are the interior points (X h/2, Y h/2) of
 *            the half-grid, numbered (Y-1)(2n-1) + (X-1): vertex values at even
 *            (X, Y), scaled normal derivatives h du/dy, h du/dx and
 *            h (du/dx - du/dy) at the horizontal, vertical and diagonal edge
 *            midpoints; the stiffness is the broken Hessian form; the coarse
 *            space is BFS (kind 4) on the subdomain grid and P its Morley
 *            interpolant; subdomains follow the box rule on the half-grid;
 *   kind 4 = the clamped plate with Bogner-Fox-Schmit bicubics (Section 2.2,
 *            the paper's element for m = 2) on an n x n square grid (equal
 *            sides, kappa NULL): four dofs per interior node, node-major
 *            4 node + c for (u, h du/dx, h du/dy, h^2 d^2u/dxdy); P is the
 *            nested interpolation from BFS on the subdomain grid; subdomains
 *            take the box rule on nodes with all four dofs;
 *   kind 5 = P1 as kind 0 on the L-shaped domain of Example 6.2: the square
 *            [0, L]^2 of an n x n grid (n and nsub even, equal sides, kappa
 *            NULL) minus the quadrant of its centre (x >= L/2, y <= L/2); dofs
 *            are the square's interior nodes outside the closed quadrant, in
 *            the square's order; subdomains are the boxes of the domain;
 *   kind 6 = trilinear bricks as kind 2 on the L-shaped prism of Example 6.4:
 *            the box minus the prism x >= Lx/2, y >= Ly/2 (x / y cell and
 *            subdomain counts even, kappa NULL), restricted in the same way.
 * kappa: per-element coefficient, layout [ny][nx][2] (kind 0, entry 0 = the
 * triangle below the diagonal) or [nz][ny][nx] (kinds 1, 2); NULL = 1.
 * Subdomains (partition): BPJD_PART_BOXES (0): nsub boxes per axis grown by
 * delta element layers (colours 2^dim); BPJD_PART_TRIANGLES (1, kind 0 only,
 * nx = ny, equal nsub, 2 delta < nx / nsub): the partition of Example 6.1,
 * every coarse square cut along its SW->NE diagonal into two coarse triangles
 * (N = 2 nsub^2), each grown by delta rings of fine triangles (a ring adds
 * every fine triangle sharing a vertex with the region); local dofs are the
 * interior nodes whose six fine triangles all lie in the grown region; id
 * 2 (sx + nsub sy) + T (T = 0 below the diagonal), 8 colours
 * 2 ((sx mod 2) + 2 (sy mod 2)) + T.  The coarse space is P1 on the coarse
 * triangles either way (the coarse squares split SW->NE).  The initial grid of
 * Step 1 is the subdomain grid refined tau times. */
#define BPJD_PART_BOXES     0
#define BPJD_PART_TRIANGLES 1
typedef struct {
  int32_t kind;
  int32_t n[3];
  double  length[3];
  int32_t nsub[3];
  int32_t delta;
  int32_t tau;
  const double* kappa;
  int32_t partition;  /* BPJD_PART_BOXES (0) | BPJD_PART_TRIANGLES */
} bpjd_mesh;

typedef struct {
  bpjd_csr K, M, P, P0;     /* host arrays owned by the problem */
  bpjd_partition part;
} bpjd_problem;

/* Assembles K, M, P, P0 and the partition on the host.  Errors: BAD_ARG (also for
 * a triangle partition on another kind, unequal axes, or 2 delta >= nx / nsub). */
int bpjd_problem_create(const bpjd_mesh* mesh, bpjd_problem** out);
void bpjd_problem_free(bpjd_problem* p);

/* ---- serving: many independent eigenproblems on one GPU ----------------
 *
 * A server solves a stream of independent requests (each one a full
 * bpjd_setup + bpjd_solve of its own pencil and partition) on a few worker
 * threads, each with its own CUDA stream, so that small requests overlap on
 * the GPU.  Admission is under a device-memory budget: a queued request starts
 * when its estimated device footprint fits beside the requests in flight.
 * Among the requests that fit, the default order takes the smallest estimated
 * work first (dofs x k), except that a request waiting longer than
 * starvation_s seconds goes ahead of every younger one (oldest first), so that
 * small requests are not held up behind large ones and large ones still start;
 * BPJD_ADMIT_FIFO keeps arrival order.  With batch_local (the default) the
 * local solves of the requests in flight share their launches: a request that
 * reaches the local part of a preconditioner application waits (at most
 * batch_wait_us) for the other requests in a solve to reach theirs, and all of
 * them run as one grouped launch per kernel kind and window tier over every
 * (request, subdomain, shift) pair, of uneven sizes; the rest of each step stays
 * on the request's own stream.  This is the per-request workflow of
 * Algorithm 3.1 run many times; the paper itself solves one pencil at a time.
 */
#define BPJD_ADMIT_SMALLEST 0  /* smallest estimated work first, with aging (default) */
#define BPJD_ADMIT_FIFO     1  /* arrival order */
#define BPJD_PENDING 1  /* bpjd_server_poll: the request has not finished yet */

typedef struct {
  size_t  hbm_budget_bytes; /* device bytes the admitted requests may hold together;
                               0: 80% of the free device memory at creation */
  int32_t workers;          /* concurrent solves, each on its own stream (default 8, 1..32) */
  int32_t precision;        /* per-request options, as in bpjd_opts; defaults BPJD_MIXED, */
  int32_t subspace;         /*   BPJD_W_3K, BPJD_STOP_RESIDUAL, 1e-8, 500                  */
  int32_t stop_rule;
  double  tol;
  int32_t max_iter;
  int32_t admission;        /* BPJD_ADMIT_SMALLEST (default) | BPJD_ADMIT_FIFO */
  double  starvation_s;     /* aging limit of BPJD_ADMIT_SMALLEST (default 1 s) */
  int32_t host_loop;        /* per-request loop mode, as in bpjd_opts; default 1, each
                               request's loop driven by its worker thread */
  int32_t batch_local;      /* 1 (default): the local solves (Eq. (3.3), first term) of the
                               requests in flight are packed into shared launches, one per
                               kernel kind and window tier, whenever their preconditioner
                               applications coincide (requests of other precisions, or whose
                               factors are solved in chunks, keep their own launches);
                               0: every request launches its own.  Needs host_loop = 1.
                               Results are bitwise those of the request alone. */
  int32_t batch_wait_us;    /* how long a request's local solves wait for those of the other
                               requests in flight before they are launched (default 100) */
} bpjd_server_opts;

typedef struct bpjd_server bpjd_server;

void bpjd_server_default_opts(bpjd_server_opts* o);

/* Packing of the local solves (bpjd_server_opts.batch_local): *launches = how many
   shared launch groups ran so far (each: one launch per kernel kind and window tier),
   *solves = how many requests' preconditioner applications they carried (their ratio
   is the mean number of requests per shared launch).  Zeros when packing is off.
   Errors: BAD_ARG. */
int bpjd_server_batch_stats(const bpjd_server* s, int64_t* launches, int64_t* solves);

/* Starts the worker threads on the current device.  Errors: BAD_ARG, CUDA. */
int bpjd_server_create(const bpjd_server_opts* opts, bpjd_server** out);

/*
 * Queues one request; every input is host memory and is copied before the call
 * returns (the caller may free it at once).  P0 may be NULL (tau = 0).
 * *ticket identifies the request in bpjd_server_poll.  Errors: BAD_ARG,
 * CSR_INVALID or MAP_INVALID (host checks of the inputs), TOO_LARGE (the
 * estimated footprint exceeds the whole budget).
 */
int bpjd_server_submit(bpjd_server* s, const bpjd_csr* A, const bpjd_csr* M, const bpjd_csr* P,
                       const bpjd_csr* P0, const bpjd_partition* part, int32_t k, uint64_t* ticket);

/*
 * Collects a finished request.  wait = 0 returns BPJD_PENDING at once if it is
 * still queued or running; wait = 1 blocks until it finishes.  On completion the
 * request's own status is returned (BPJD_OK or its bpjd_setup / bpjd_solve
 * error) and, where not NULL: eigvals (k), eigvecs (n x k row-major, host),
 * st, and times[3] = {seconds queued, seconds in service, seconds from submit
 * to completion}.  A collected ticket is forgotten (BAD_ARG afterwards).
 */
int bpjd_server_poll(bpjd_server* s, uint64_t ticket, int32_t wait, double* eigvals, double* eigvecs,
                     bpjd_stats* st, double* times);

/* Waits for every queued request to finish, then stops the workers and frees
 * the server (uncollected results are dropped). */
void bpjd_server_free(bpjd_server* s);

#ifdef __cplusplus
}
#endif
#endif /* BPJD_H_ */
