// CUDA kernels of one BPJD iteration (Section 3, Algorithm 3.1) for sm_103a.
//
// Layout: every block of k vectors is row-major n x k (k contiguous per dof),
// FP64.  Reductions over the n rows are done in two deterministic stages
// (fixed per-block partial sums, then a per-entry sum over the blocks), so a
// run is bit-reproducible for a given launch configuration.

#include <cuda_runtime.h>
#include <math_constants.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <map>
#include <mutex>
#include <new>
#include <set>
#include <utility>
#include <type_traits>

#include "bpjd_internal.h"
#include "dword.cuh"

namespace bpjd {

// Raises a kernel's dynamic shared memory limit to the device maximum, once per
// (kernel, device).  A per-launch limit would race between host threads that
// launch the same kernel with different sizes (concurrent solves): one thread
// could lower the limit below another's launch.
static std::mutex g_smem_attr_mu;
static std::set<std::pair<const void*, int>> g_smem_attr_done;

int allow_dynamic_smem(const void* kern) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return (int)cudaErrorInvalidDevice;
  {
    std::lock_guard<std::mutex> lk(g_smem_attr_mu);
    if (g_smem_attr_done.count({kern, dev})) return 0;
  }
  int optin = 0;
  cudaFuncAttributes fa;
  cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kern);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
  if (e != cudaSuccess) return (int)e;
  std::lock_guard<std::mutex> lk(g_smem_attr_mu);
  g_smem_attr_done.insert({kern, dev});
  return 0;
}

namespace {

constexpr int kPartialBlocks = 456;  // 3 x 152 SMs

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------
// CSR SpMM over a block of vectors: YA = A X and (optionally) YM = M X with a
// shared pattern.  LANES consecutive lanes serve one row; lane j of the group
// owns columns j, j + LANES, ... (at most 2 per lane).  The row's column
// indices and values are broadcast to the group; X rows are read as contiguous
// ncols-vectors.
// ---------------------------------------------------------------------------
template <int LANES>
__global__ void __launch_bounds__(256) k_spmm(int n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                              const double* __restrict__ va, const double* __restrict__ vm,
                                              const double* __restrict__ X, double* __restrict__ YA,
                                              double* __restrict__ YM, int ncols) {
  constexpr int RPW = 32 / LANES;
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t row = warp * RPW + lane / LANES;
  const int j0 = lane % LANES;
  if (row >= n) return;
  double a0 = 0, a1 = 0, m0 = 0, m1 = 0;
  const int j1 = j0 + LANES;
  const bool has0 = j0 < ncols, has1 = j1 < ncols;
  for (int64_t e = rp[row]; e < rp[row + 1]; ++e) {
    const int64_t c = ci[e];
    const double av = va[e];
    const double mv = vm ? vm[e] : 0.0;
    const double* xr = X + c * ncols;
    if (has0) {
      double x = xr[j0];
      a0 = fma(av, x, a0);
      m0 = fma(mv, x, m0);
    }
    if (has1) {
      double x = xr[j1];
      a1 = fma(av, x, a1);
      m1 = fma(mv, x, m1);
    }
  }
  if (has0) {
    YA[row * ncols + j0] = a0;
    if (YM) YM[row * ncols + j0] = m0;
  }
  if (has1) {
    YA[row * ncols + j1] = a1;
    if (YM) YM[row * ncols + j1] = m1;
  }
}

// Y[r, j] = sum_e P[r, c_e] D[c_e, j] for j < ncols (sparse times small dense).
__global__ void k_csr_dense(int n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                            const double* __restrict__ pv, const double* __restrict__ D, int ldd, int ncols,
                            double* __restrict__ Y, int ldy) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * ncols) return;
  int64_t r = t / ncols;
  int j = (int)(t % ncols);
  double acc = 0;
  for (int64_t e = rp[r]; e < rp[r + 1]; ++e) acc = fma(pv[e], D[(int64_t)ci[e] * ldd + j], acc);
  Y[r * ldy + j] = acc;
}

// ---------------------------------------------------------------------------
// Column sums in two stages.  Block size is a multiple of k and so is the grid
// stride, hence thread t always works on column t % k.
// ---------------------------------------------------------------------------
__device__ void block_column_partials(double acc0, double acc1, int k, double* partial /* [blocks][2k] */) {
  extern __shared__ double sred[];
  const int tid = threadIdx.x;
  sred[tid] = acc0;
  sred[blockDim.x + tid] = acc1;
  __syncthreads();
  if (tid < k) {
    double s0 = 0, s1 = 0;
    for (int t = tid; t < (int)blockDim.x; t += k) {
      s0 += sred[t];
      s1 += sred[blockDim.x + t];
    }
    partial[(int64_t)blockIdx.x * 2 * k + tid] = s0;
    partial[(int64_t)blockIdx.x * 2 * k + k + tid] = s1;
  }
}

// rho = lam .* MX - AX, and per-column partial sums of rho^2 and MX^2.
__global__ void k_residual(int64_t nk, int k, const double* __restrict__ AX, const double* __restrict__ MX,
                           const double* __restrict__ lam, double* __restrict__ rho, double* partial) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int col = (int)(t % k);
  const double l = lam[col];
  double r2 = 0, m2 = 0;
  for (; t < nk; t += stride) {
    double mx = MX[t];
    double r = l * mx - AX[t];
    rho[t] = r;
    r2 = fma(r, r, r2);
    m2 = fma(mx, mx, m2);
  }
  block_column_partials(r2, m2, k, partial);
}

// x . Ax and x . Mx per column.
__global__ void k_rq_partial(int64_t nk, int k, const double* __restrict__ X, const double* __restrict__ AX,
                             const double* __restrict__ MX, double* partial) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double s0 = 0, s1 = 0;
  for (; t < nk; t += stride) {
    double x = X[t];
    s0 = fma(x, AX[t], s0);
    s1 = fma(x, MX[t], s1);
  }
  block_column_partials(s0, s1, k, partial);
}

// sums[q] = sum_b partial[b * 2k + q] for q < 2k: warp w sums q = w, w + 8, ...,
// lane l the blocks b = l, l + 32, ... in order, then a fixed butterfly.
__device__ void column_partial_sums(int nblk, int k, const double* __restrict__ partial, double* sums) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int q = w; q < 2 * k; q += nw) {
    double a = 0;
    for (int b = lane; b < nblk; b += 32) a += partial[(int64_t)b * 2 * k + q];
    a = warp_sum(a);
    if (lane == 0) sums[q] = a;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(256) k_residual_finish(int nblk, int k, const double* partial, const double* lam,
                                                         int stop_rule, double tol, DevStatus* st) {
  __shared__ double sums[128];
  __shared__ double res[64];
  column_partial_sums(nblk, k, partial, sums);
  const int i = threadIdx.x;
  if (i < k) {
    const double r = sqrt(sums[i]) / (fabs(lam[i]) * sqrt(sums[k + i]));
    res[i] = r;
    st->res[i] = r;
  }
  __syncthreads();
  if (i == 0) {
    double mx = 0;
    for (int j = 0; j < k; ++j) mx = fmax(mx, res[j]);
    st->max_res = mx;
    if (stop_rule == BPJD_STOP_RESIDUAL) st->converged = (mx <= tol) ? 1 : 0;
  }
}

__global__ void __launch_bounds__(256) k_rq_finish(int nblk, int k, const double* partial, double* lam) {
  __shared__ double sums[128];
  column_partial_sums(nblk, k, partial, sums);
  const int i = threadIdx.x;
  if (i < k) lam[i] = sums[i] / sums[k + i];
}

// ---------------------------------------------------------------------------
// Block inner products out = U^T V with U = [U_0 .. U_{p-1}], V = [V_0 .. V_{q-1}],
// each U_b, V_b an n x k row-major array.  Stage 1 writes per-block partials.
// ---------------------------------------------------------------------------
struct Ptrs6 {
  const double* p[6];
};
constexpr int kInnerRows = 16;
constexpr int kInnerMaxOut = 36;  // (96 x 96) / 256

__global__ void __launch_bounds__(256) k_inner(int n, int k, int p, Ptrs6 U, int q, Ptrs6 V, int rows_per_block,
                                               double* partial) {
  extern __shared__ double sm[];
  const int mu = p * k, mv = q * k;
  double* Us = sm;                       // [kInnerRows][mu]
  double* Vs = sm + kInnerRows * mu;     // [kInnerRows][mv]
  const int nout = mu * mv;
  double acc[kInnerMaxOut];
#pragma unroll
  for (int o = 0; o < kInnerMaxOut; ++o) acc[o] = 0;
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
  const int64_t r1 = min((int64_t)n, r0 + rows_per_block);
  for (int64_t rb = r0; rb < r1; rb += kInnerRows) {
    const int nr = (int)min((int64_t)kInnerRows, r1 - rb);
    for (int t = threadIdx.x; t < kInnerRows * mu; t += blockDim.x) {
      int r = t / mu, c = t % mu;
      Us[t] = (r < nr) ? U.p[c / k][(rb + r) * k + (c % k)] : 0.0;
    }
    for (int t = threadIdx.x; t < kInnerRows * mv; t += blockDim.x) {
      int r = t / mv, c = t % mv;
      Vs[t] = (r < nr) ? V.p[c / k][(rb + r) * k + (c % k)] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int oo = 0; oo < kInnerMaxOut; ++oo) {
      int o = threadIdx.x + oo * blockDim.x;
      if (o < nout) {
        int a = o / mv, b = o % mv;
        double s = acc[oo];
        for (int r = 0; r < kInnerRows; ++r) s = fma(Us[r * mu + a], Vs[r * mv + b], s);
        acc[oo] = s;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int oo = 0; oo < kInnerMaxOut; ++oo) {
    int o = threadIdx.x + oo * blockDim.x;
    if (o < nout) partial[(int64_t)blockIdx.x * nout + o] = acc[oo];
  }
}

// ---------------------------------------------------------------------------
// Block inner products in double-word arithmetic (Dot2 on the FP32 pipe):
// out_v = U^T V_v for v < NV, with U = [U_0 .. U_{nu-1}] (mu = nu k columns)
// and V_v = [V_v,0 ..] (mv columns), all n x k FP64 row-major blocks.  With
// sym = 1 only the 4 x 4 output tiles on or above the diagonal are formed
// (U^T V symmetric).  Rows are staged in shared memory in chunks, split into
// (hi, lo) float pairs once; each thread owns one output tile and a slice of
// the chunk rows; slices are combined in FP64 at the end of the block and the
// per-block partial sums are reduced over blocks in FP64 by k_gram_reduce.
// ---------------------------------------------------------------------------
constexpr int kGramRows = 64;
constexpr int kGramBlocks = 304;  // two resident blocks on each of the 152 SMs: one wave

__device__ __forceinline__ void gram_tile_of(int t, int TU, int TV, int sym, int& ta, int& tb) {
  if (!sym) {
    ta = t / TV;
    tb = t % TV;
    return;
  }
  int a = 0;
  while (t >= TU - a) {
    t -= TU - a;
    ++a;
  }
  ta = a;
  tb = a + t;
}

__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Per-block Gram partials in double-word arithmetic (Dot2 per entry).  The
// row range of a block is processed in chunks of R rows: the FP64 rows of
// every U / V block are copied asynchronously into a raw staging buffer two
// chunks ahead (double buffered), split into (hi, lo) planes once per chunk,
// and every thread accumulates a 4 x 4 tile of the output for every NV over
// its slice of the chunk's rows.  Plane layout: one segment of R x k values per
// block (U blocks, then V1, then V2), row-major.
// VEC: k is a multiple of 4, so the four columns of a tile lie in one block,
// contiguous and 16-byte aligned in the planes (vector loads, no padding).
template <int NV, bool VEC>
__global__ void __launch_bounds__(256, 2) k_gram_dw(int n, int k, int nu, Ptrs6 U, int nvb, Ptrs6 V1, Ptrs6 V2, int sym,
                                                 int rows_per_block, int R, double* partial) {
  extern __shared__ __align__(16) float gsm[];
  const int mu = nu * k, mv = nvb * k;
  const int TU = (mu + 3) / 4, TV = (mv + 3) / 4;
  const int ntiles = sym ? TU * (TU + 1) / 2 : TU * TV;
  const int S = max(1, (int)blockDim.x / ntiles);
  const int nseg = nu + NV * nvb;
  const int SEG = R * k;    // values per segment
  const int CH = nseg * SEG;  // values per chunk
  double* raw = reinterpret_cast<double*>(gsm);    // [2][CH]
  float* ph = reinterpret_cast<float*>(raw + 2 * CH);  // [CH]
  float* pl = ph + CH;                                 // [CH]
  const int tid = threadIdx.x;
  const int tile = tid % ntiles, slice = tid / ntiles;
  const bool worker = slice < S;
  int ta = 0, tb = 0;
  gram_tile_of(tile, TU, TV, sym, ta, tb);
  // plane offsets of this thread's four U columns and four V columns (-1: past the end)
  int uo[4], vo[4];
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    const int cu = 4 * ta + x, cv = 4 * tb + x;
    uo[x] = (cu < mu) ? (cu / k) * SEG + cu % k : -1;
    vo[x] = (cv < mv) ? (nu + cv / k) * SEG + cv % k : -1;
  }
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
  const int64_t r1 = min((int64_t)n, r0 + rows_per_block);
  const int nch = (int)((r1 - r0 + R - 1) / R);
  auto seg_ptr = [&](int sg) -> const double* {
    if (sg < nu) return U.p[sg];
    sg -= nu;
    if (sg < nvb) return V1.p[sg];
    return V2.p[sg - nvb];
  };
  auto issue = [&](int c) {
    if (c < nch) {
      const int64_t rb = r0 + (int64_t)c * R;
      const int64_t lim = (r1 - rb) * k;  // values of this chunk inside the row range
      double* dst = raw + (c & 1) * CH;
      for (int sg = 0; sg < nseg; ++sg) {
        const double* src = seg_ptr(sg) + rb * k;
        for (int e = tid; e < SEG; e += blockDim.x)
          if (e < lim) cp_async8(dst + sg * SEG + e, src + e);
      }
    }
    cp_async_commit();
  };
  dot2 acc[NV][4][4];
#pragma unroll
  for (int v = 0; v < NV; ++v)
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) acc[v][x][y].zero();
  issue(0);
  issue(1);
  for (int c = 0; c < nch; ++c) {
    cp_async_wait1();
    __syncthreads();  // chunk c has landed for every thread; the planes are free
    {
      const int nr = (int)min((int64_t)R, r1 - (r0 + (int64_t)c * R));
      const double* src = raw + (c & 1) * CH;
      if (nr == R) {
        for (int e = tid; e < CH; e += blockDim.x) {
          const dw sp = split_f64(src[e]);
          ph[e] = sp.hi;
          pl[e] = sp.lo;
        }
      } else {  // last chunk of the range: rows past its end are zero
        for (int e = tid; e < CH; e += blockDim.x) {
          const int r = (e % SEG) / k;
          const dw sp = split_f64(r < nr ? src[e] : 0.0);
          ph[e] = sp.hi;
          pl[e] = sp.lo;
        }
      }
    }
    __syncthreads();  // planes ready; the raw buffer of chunk c is free
    issue(c + 2);
    if (worker && VEC) {
      for (int r = slice; r < R; r += S) {
        const int ro = r * k;
        const float4 uh = *reinterpret_cast<const float4*>(ph + uo[0] + ro);
        const float4 ul = *reinterpret_cast<const float4*>(pl + uo[0] + ro);
        const float a_h[4] = {uh.x, uh.y, uh.z, uh.w};
        const float a_l[4] = {ul.x, ul.y, ul.z, ul.w};
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const int o = vo[0] + v * mv * R + ro;
          const float4 vh = *reinterpret_cast<const float4*>(ph + o);
          const float4 vl = *reinterpret_cast<const float4*>(pl + o);
          const float b_h[4] = {vh.x, vh.y, vh.z, vh.w};
          const float b_l[4] = {vl.x, vl.y, vl.z, vl.w};
#pragma unroll
          for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 4; ++y) acc[v][x][y].mac(a_h[x], a_l[x], b_h[y], b_l[y]);
        }
      }
    } else if (worker) {
      for (int r = slice; r < R; r += S) {
        const int ro = r * k;
        float a_h[4], a_l[4];
#pragma unroll
        for (int x = 0; x < 4; ++x) {
          a_h[x] = (uo[x] >= 0) ? ph[uo[x] + ro] : 0.f;
          a_l[x] = (uo[x] >= 0) ? pl[uo[x] + ro] : 0.f;
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          float b_h[4], b_l[4];
#pragma unroll
          for (int y = 0; y < 4; ++y) {
            const int o = vo[y] + v * mv * R;  // V2 segments follow the V1 segments
            b_h[y] = (vo[y] >= 0) ? ph[o + ro] : 0.f;
            b_l[y] = (vo[y] >= 0) ? pl[o + ro] : 0.f;
          }
#pragma unroll
          for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 4; ++y) acc[v][x][y].mac(a_h[x], a_l[x], b_h[y], b_l[y]);
        }
      }
    }
  }
  cp_async_wait0();
  __syncthreads();
  // combine the slices of every tile in FP64 (shared memory reused)
  double* red = reinterpret_cast<double*>(gsm);
  const int per = NV * 16;
  double mine[NV * 16];
#pragma unroll
  for (int v = 0; v < NV; ++v)
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) mine[v * 16 + x * 4 + y] = acc[v][x][y].value();
  for (int sl = 1; sl < S; ++sl) {
    if (worker && slice == sl)
      for (int e = 0; e < per; ++e) red[tile * per + e] = mine[e];
    __syncthreads();
    if (worker && slice == 0)
      for (int e = 0; e < per; ++e) mine[e] += red[tile * per + e];
    __syncthreads();
  }
  if (worker && slice == 0) {
    double* out = partial + (int64_t)blockIdx.x * ntiles * per;
    for (int e = 0; e < per; ++e) out[(e / 16) * ntiles * 16 + tile * 16 + (e % 16)] = mine[e];
  }
}

// Sum of the per-block Gram partials: a block serves 32 consecutive entries;
// warp w adds blocks b = w, w + 8, ... in order, warp 0 adds the eight results
// in order (fixed order: bit-reproducible).
__global__ void __launch_bounds__(256) k_gram_reduce(int nblk, int nv, int mu, int mv, int sym,
                                                     const double* __restrict__ partial, double* out1,
                                                     double* out2) {
  __shared__ double red[8][32];
  const int TU = (mu + 3) / 4, TV = (mv + 3) / 4;
  const int ntiles = sym ? TU * (TU + 1) / 2 : TU * TV;
  const int total = nv * ntiles * 16;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int t = blockIdx.x * 32 + lane;
  double s = 0;
  if (t < total)
    for (int b = w; b < nblk; b += 8) s += partial[(int64_t)b * total + t];
  red[w][lane] = s;
  __syncthreads();
  if (w != 0 || t >= total) return;
  s = red[0][lane];
#pragma unroll
  for (int q = 1; q < 8; ++q) s += red[q][lane];
  const int v = t / (ntiles * 16);
  const int rem = t % (ntiles * 16);
  const int tile = rem / 16, e = rem % 16;
  int ta, tb;
  gram_tile_of(tile, TU, TV, sym, ta, tb);
  const int a = 4 * ta + e / 4, c = 4 * tb + e % 4;
  if (a >= mu || c >= mv) return;
  double* out = (v == 0) ? out1 : out2;
  out[a * mv + c] = s;
  if (sym) out[c * mv + a] = s;
}

// Row-wise block update in double-word arithmetic:
// out[r, j] = Zadd[r, j] + sign * sum_b sum_a W_b[r, a] C[(b k + a) ldc + j].
// A block stages kCombRows rows of W split into (hi, lo) floats and the split
// coefficient matrix; each thread forms outputs with Dot2 and converts once to
// FP64.
constexpr int kCombRows = 64;
__global__ void __launch_bounds__(256) k_combine_dw(int64_t n, int k, int nin, Ptrs6 W, const double* __restrict__ C,
                                                    int ldc, int csub, const double* __restrict__ Zadd,
                                                    double* __restrict__ out, double sign, float2* __restrict__ outs) {
  extern __shared__ __align__(16) float csm[];
  const int m = nin * k;
  float* Ch = csm;                       // m x csub
  float* Cl = Ch + m * csub;
  float* Wh = Cl + m * csub;             // kCombRows x m
  float* Wl = Wh + kCombRows * m;
  for (int t = threadIdx.x; t < m * csub; t += blockDim.x) {
    const dw s = split_f64(C[(t / csub) * ldc + (t % csub)]);
    Ch[t] = s.hi;
    Cl[t] = s.lo;
  }
  const int64_t row0 = (int64_t)blockIdx.x * kCombRows;
  const int nr = (int)min((int64_t)kCombRows, n - row0);
  // staged entries t = tid, tid + blockDim, ... of the nr x m row block: (row, entry)
  // advanced incrementally, the block and column of entry a read from a table (no
  // integer division per element)
  __shared__ unsigned char eb[96], ec[96];
  for (int a = threadIdx.x; a < m; a += blockDim.x) {
    eb[a] = (unsigned char)(a / k);
    ec[a] = (unsigned char)(a % k);
  }
  __syncthreads();
  {
    int r = threadIdx.x / m, a = threadIdx.x % m;
    const int dr = blockDim.x / m, da = blockDim.x % m;
    while (r < nr) {
      const dw s = split_f64(W.p[eb[a]][(row0 + r) * k + ec[a]]);
      Wh[r * m + a] = s.hi;
      Wl[r * m + a] = s.lo;
      a += da;
      r += dr;
      if (a >= m) {
        a -= m;
        ++r;
      }
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nr * csub; t += blockDim.x) {
    const int r = t / csub, j = t % csub;
    dot2 acc;
    acc.zero();
    const float* wh = Wh + r * m;
    const float* wl = Wl + r * m;
    for (int a = 0; a < m; ++a) acc.mac(wh[a], wl[a], Ch[a * csub + j], Cl[a * csub + j]);
    double v = sign * acc.value();
    const int64_t o = (row0 + r) * csub + j;
    if (Zadd) v += Zadd[o];
    out[o] = v;
    if (outs) {
      const dw sp = split_f64(v);
      outs[o] = make_float2(sp.hi, sp.lo);
    }
  }
}

// CSR SpMM in double-word arithmetic with pre-split matrix values (hi/lo
// float arrays of K and M): YA = K X, YM = M X.  LANES lanes serve one row;
// lane j of the group owns columns j + LANES c, c < CPL.  The X entries are
// split on the fly (integer operations only), or (XS) read as the (hi, lo)
// pairs that the kernel producing X wrote beside it (split_f64 of the same
// values: the same products).
template <int LANES, int CPL, bool XS>
__global__ void __launch_bounds__(256, 4) k_spmm_dw(int n, const int64_t* __restrict__ rp,
                                                    const int32_t* __restrict__ ci,
                                                    const float2* __restrict__ va, const float2* __restrict__ vm,
                                                    const double* __restrict__ X, const float2* __restrict__ Xs,
                                                    double* __restrict__ YA, double* __restrict__ YM, int ncols) {
  constexpr int RPW = 32 / LANES;
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t row = warp * RPW + lane / LANES;
  const int j0 = lane % LANES;
  if (row >= n) return;
  dot2 a[CPL], m[CPL];
#pragma unroll
  for (int c = 0; c < CPL; ++c) {
    a[c].zero();
    m[c].zero();
  }
  for (int64_t e = rp[row]; e < rp[row + 1]; ++e) {
    const int64_t col = ci[e];
    const float2 av = va[e];
    const float2 mv = vm ? vm[e] : make_float2(0.f, 0.f);
    const double* xr = X + col * ncols;
    const float2* xsr = Xs + col * ncols;
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
      const int j = j0 + LANES * c;
      if (j < ncols) {
        dw x;
        if (XS) {
          const float2 p = xsr[j];
          x.hi = p.x;
          x.lo = p.y;
        } else {
          x = split_f64(xr[j]);
        }
        a[c].mac(av.x, av.y, x.hi, x.lo);
        m[c].mac(mv.x, mv.y, x.hi, x.lo);
      }
    }
  }
#pragma unroll
  for (int c = 0; c < CPL; ++c) {
    const int j = j0 + LANES * c;
    if (j < ncols) {
      YA[row * ncols + j] = a[c].value();
      if (YM) YM[row * ncols + j] = m[c].value();
    }
  }
}

// Row-wise block update in FP32 (hi parts of W and C):
// out[r, j] = Zadd[r, j] + sign * sum_b sum_a W_b[r, a] C[(b k + a) ldc + j],
// for the previous-update block P of the search space, which only has to be
// consistent with its own products K P and M P (formed afterwards in
// double-word arithmetic from the stored P).  A block stages kCombRows rows of
// W and the coefficients.
__global__ void __launch_bounds__(256) k_combine_f32(int64_t n, int k, int nin, Ptrs6 W, const double* __restrict__ C,
                                                     int ldc, int csub, const double* __restrict__ Zadd,
                                                     double* __restrict__ out, float sign, float2* __restrict__ outs) {
  extern __shared__ __align__(16) float csm[];
  const int m = nin * k;
  float* Cs = csm;              // m x csub
  float* Ws = Cs + m * csub;    // kCombRows x m
  for (int t = threadIdx.x; t < m * csub; t += blockDim.x) Cs[t] = f64_hi(C[(t / csub) * ldc + (t % csub)]);
  const int64_t row0 = (int64_t)blockIdx.x * kCombRows;
  const int nr = (int)min((int64_t)kCombRows, n - row0);
  for (int b = 0; b < nin; ++b) {
    const double* src = W.p[b] + row0 * k;
    for (int t = threadIdx.x; t < nr * k; t += blockDim.x) Ws[(t / k) * m + b * k + (t % k)] = f64_hi(src[t]);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nr * csub; t += blockDim.x) {
    const int r = t / csub, j = t % csub;
    float acc = 0.f;
    const float* w = Ws + r * m;
    for (int a = 0; a < m; ++a) acc = fmaf(w[a], Cs[a * csub + j], acc);
    const int64_t o = (row0 + r) * csub + j;
    float v = sign * acc;
    if (Zadd) v += f64_hi(Zadd[o]);
    const double vd = f32_to_f64_bits(v);
    out[o] = vd;
    if (outs) {
      const dw sp = split_f64(vd);
      outs[o] = make_float2(sp.hi, sp.lo);
    }
  }
}

__global__ void k_split_values(int64_t nnz, const double* __restrict__ v, float2* __restrict__ out) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nnz) return;
  const dw s = split_f64(v[t]);
  out[t] = make_float2(s.hi, s.lo);
}

__global__ void k_sum_partials(int nblk, int len, const double* partial, double* out) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= len) return;
  double s = 0;
  for (int b = 0; b < nblk; ++b) s += partial[(int64_t)b * len + j];
  out[j] = s;
}

// out[r, j] = alpha_z * Zadd[r, j] + sign * sum_b sum_a W_b[r, a] C[(b k + a) * ldc + j]
__global__ void k_combine_rows(int64_t n, int k, int nin, Ptrs6 W, const double* __restrict__ C, int ldc,
                               int csub, const double* __restrict__ Zadd, double* __restrict__ out,
                               double sign) {
  extern __shared__ double Cs[];
  const int m = nin * k;
  for (int t = threadIdx.x; t < m * csub; t += blockDim.x) Cs[t] = C[(t / csub) * ldc + (t % csub)];
  __syncthreads();
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n * csub) return;
  int64_t r = t / csub;
  int j = (int)(t % csub);
  double acc = 0;
  for (int b = 0; b < nin; ++b) {
    const double* wr = W.p[b] + r * k;
    for (int a = 0; a < k; ++a) acc = fma(wr[a], Cs[(b * k + a) * csub + j], acc);
  }
  double v = sign * acc;
  if (Zadd) v += Zadd[r * csub + j];
  out[r * csub + j] = v;
}

// ---------------------------------------------------------------------------
// Local solves: one warp per (subdomain l, column i) computes
//   w = (K_l - lambda_i M_l)^{-1} R_l rho_i
// by a banded Cholesky factorisation streamed through a (B x B) window held
// in shared memory (B = lower bandwidth + 1), with the forward substitution
// fused into the factorisation and the band factor written to scratch for the
// backward substitution.  The window is stored as a full symmetric B x B
// block with circular row/column slots (slot of row p = p mod B); step j
// eliminates row j, updates the remaining b rows by a rank-1 update and loads
// row j + B of the shifted band matrix into the freed slot.  Rows past n_l
// are identity rows.  A pivot <= 0 sets err (Eq. (3.1) violated).
// ---------------------------------------------------------------------------
template <typename TP>
__global__ void k_local_band(int npairs, int k, const int64_t* __restrict__ sub_ptr,
                             const int32_t* __restrict__ sub_dofs, int B, const TP* __restrict__ bandK,
                             const TP* __restrict__ bandM, const double* __restrict__ lam,
                             const double* __restrict__ rho, TP* __restrict__ Lbuf, TP* __restrict__ wpk,
                             int32_t* err, int64_t rec_base) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int pair = blockIdx.x * (blockDim.x >> 5) + wib;
  if (pair >= npairs) return;
  const int BB = B * B;
  TP* W = reinterpret_cast<TP*>(smraw) + (size_t)wib * (BB + 3 * B);
  TP* rw = W + BB;   // right-hand side window
  TP* lc = rw + B;   // current column of L by slot
  TP* xs = lc + B;   // solution window (backward sweep)
  const int l = pair / k, i = pair % k;
  const int64_t off = sub_ptr[l];
  const int nl = (int)(sub_ptr[l + 1] - off);
  const int32_t* dofs = sub_dofs + off;
  const int b = B - 1;
  const TP lm = (TP)lam[i];
  TP* Lp = Lbuf + ((size_t)(off - rec_base) * k + (size_t)i * nl) * B;
  auto aval = [&](int p, int q) -> TP {  // shifted local matrix entry, q <= p <= q + b
    if (p >= nl) return (p == q) ? TP(1) : TP(0);
    const size_t e = (size_t)(off + p) * B + (q - p + b);
    return bandK[e] - lm * bandM[e];
  };
  // initial window: rows 0..B-1
  for (int e = lane; e < BB; e += 32) W[e] = TP(0);
  __syncwarp();
  for (int p = 0; p < B; ++p) {
    for (int e = lane; e <= b; e += 32) {
      int q = p - b + e;
      if (q < 0) continue;
      TP v = aval(p, q);
      W[(p % B) * B + (q % B)] = v;
      W[(q % B) * B + (p % B)] = v;
    }
    __syncwarp();
  }
  for (int p = lane; p < B; p += 32) rw[p] = (p < nl) ? (TP)rho[(int64_t)dofs[p] * k + i] : TP(0);
  __syncwarp();
  for (int j = 0; j < nl; ++j) {
    const int s = j % B;
    const TP piv = W[s * B + s];
    if (!(piv > TP(0))) {
      if (lane == 0) atomicOr(err, 1);
      return;
    }
    const TP inv = TP(1) / sqrt(piv);
    for (int u = lane; u < B; u += 32) lc[u] = (u == s) ? TP(0) : W[u * B + s] * inv;
    const TP yj = rw[s] * inv;
    __syncwarp();
    // L column j: slot 0 = 1/L_jj, slot t = L(j + t, j)
    for (int t = lane; t < B; t += 32) Lp[(size_t)j * B + t] = (t == 0) ? inv : lc[(j + t) % B];
    if (lane == 0) wpk[(off + j) * k + i] = yj;
    // rank-1 update of the window (row/column s is left alone: lc[s] = 0)
    {
      int e = lane, u = 0, v = lane;
      while (v >= B) {
        v -= B;
        ++u;
      }
      for (; e < BB; e += 32) {
        W[e] -= lc[u] * lc[v];
        v += 32;
        while (v >= B) {
          v -= B;
          ++u;
        }
      }
    }
    for (int u = lane; u < B; u += 32) rw[u] -= lc[u] * yj;
    __syncwarp();
    // load row j + B into slot s
    const int pn = j + B;
    for (int e = lane; e <= b; e += 32) {
      int q = pn - b + e;  // q in j+1 .. j+B
      TP v = aval(pn, q);
      W[s * B + (q % B)] = v;
      W[(q % B) * B + s] = v;
    }
    if (lane == 0) rw[s] = (pn < nl) ? (TP)rho[(int64_t)dofs[pn] * k + i] : TP(0);
    __syncwarp();
  }
  // backward substitution with L^T
  for (int u = lane; u < B; u += 32) xs[u] = TP(0);
  __syncwarp();
  for (int j = nl - 1; j >= 0; --j) {
    const TP* row = Lp + (size_t)j * B;
    TP part = 0;
    for (int t = 1 + lane; t < B; t += 32) {
      if (j + t < nl) part += row[t] * xs[(j + t) % B];
    }
    part = warp_sum(part);
    if (lane == 0) {
      TP xj = (wpk[(off + j) * k + i] - part) * row[0];
      xs[j % B] = xj;
      wpk[(off + j) * k + i] = xj;
    }
    __syncwarp();
  }
}


// ---------------------------------------------------------------------------
// Bulk-copy and mbarrier helpers (inline PTX).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// Bounded wait on an mbarrier phase; false after `limit` attempts (the limit is
// a launch parameter: bpjd_set_wait_limit).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int limit) {
  for (int it = 0; it < limit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
// Before a kernel that gave up waiting returns, the thread that issued the bulk
// copies waits for the ones still in flight (they write this CTA's shared
// memory), with a fixed bound of its own; false if even that runs out.
__device__ __forceinline__ bool mbar_drain(uint64_t* bar, uint32_t parity) {
  for (int it = 0; it < (1 << 22); ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
// Error bits of the local-solve kernels (h.derr[0]): a non-positive pivot, a
// bounded wait that ran out, and copies still in flight when the drain gave up.
constexpr int32_t kErrPivot = 1, kErrTimeout = 2, kErrDrain = 4;

constexpr int kLocalWarps = 4;

// ---------------------------------------------------------------------------
// Local solves, forward phase, blocked: banded Cholesky factorisation of
// K_l - lambda_i M_l eight columns at a time, with the forward substitution
// L y = rho_l (FP32, window BMAX a multiple of 8, at most 48).  One CTA of four
// warps per (subdomain l, four shifts), one warp per shift.
//
// A block of eight columns j0..j0+7 couples to the rows j0..j0+BMAX+6, so the
// window holds W = BMAX + 8 rows in W/8 slot blocks used cyclically.  The
// window (stored negated, both triangles as far as they are read) lives in
// the accumulators of m16n8k8 tensor-core tiles: lane (g, q) = (lane / 4,
// lane mod 4) of tile (rt, ct) holds slot rows rt 16 + g (+8) and slot columns
// ct 8 + 2 q (+1).  Per block step:
//   1. the pivot column block (tile column sb) goes to shared memory;
//   2. each lane takes one or two window rows of it and the warp factorises
//      the 8-column panel column by column (pivot and L entries by shuffle),
//      eliminating the right-hand side alongside and storing the columns of
//      L in slot order (1/L_jj at the pivot slot);
//   3. the panel L (W x 8) returns to shared memory and the trailing update
//      W <- W - L L^T runs as tensor-core products of every tile, each
//      operand split into a TF32 head and a TF32 tail (head x head + head x
//      tail + tail x head: FP32-level accuracy);
//   4. the eight band rows entering the freed slot block are written into the
//      row tiles (the lower triangle is all that step 1 ever reads).
// The band rows of K_l and M_l enter shared memory one window cycle (W rows)
// ahead through bulk copies shared by the four warps.
// ---------------------------------------------------------------------------
template <int BMAX>
struct MmaShape {
  static constexpr int W = BMAX + 8;        // window rows
  static constexpr int NBW = W / 8;         // slot blocks
  static constexpr int RT = (W + 15) / 16;  // row tiles of 16
  static constexpr int CT = NBW;            // column tiles of 8
  static constexpr int NH = (W + 31) / 32;  // window rows per lane in the panel
  static constexpr int PSTR = 12;           // row stride of the panel buffer (bank-conflict free)
  static constexpr int PW = RT * 16 * PSTR + W;
  static constexpr size_t smem_floats = (size_t)4 * W * BMAX + (size_t)kLocalWarps * PW;
};

// Position of slot block b in the elimination order that follows pivot block sb
// (0 = the next to be eliminated); -1 for sb itself and for blocks past the window.
template <int NBW>
__device__ __forceinline__ int elim_pos(int b, int sb) {
  if (b == sb || b >= NBW) return -1;
  const int p = b - sb - 1;
  return (p < 0) ? p + NBW : p;
}

// A window tile (row tile rt = slot blocks 2 rt, 2 rt + 1; column tile ct = slot block
// ct) is read again only where its rows come at or after its columns in the
// elimination order (pivot columns, diagonal blocks); the relative order of two
// blocks in the window never changes, so the trailing update skips the other tiles
// and the pivot's own column tile (whose slot block is refilled by entering rows).
template <int NBW>
__device__ __forceinline__ bool tile_live(int sb, int rt, int ct) {
  if (ct == sb) return false;
  const int pr = max(elim_pos<NBW>(2 * rt, sb), elim_pos<NBW>(2 * rt + 1, sb));
  return pr >= elim_pos<NBW>(ct, sb);
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void mma_tf32(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Block index of a local-solve kernel body: the launch's own (a launch of one
// handle) or relative to the first block of the body's segment (grouped launch).
struct BlockIdx {
  __device__ __forceinline__ int operator()() const { return (int)blockIdx.x; }
};
struct SegBlockIdx {
  int blk0;
  __device__ __forceinline__ int operator()() const { return (int)blockIdx.x - blk0; }
};

template <int BMAX, class BID>
__device__ __forceinline__ void k_local_factor_mma_body(BID bidf,
    int nsub, int k, const int64_t* __restrict__ sub_ptr, const int32_t* __restrict__ sub_dofs,
    const float* __restrict__ bandK, const float* __restrict__ bandM, const double* __restrict__ lam,
    const double* __restrict__ rho, float* __restrict__ Lbuf, float* __restrict__ wpk, int32_t* err,
    int wait_limit, int64_t rec_base) {
  using S = MmaShape<BMAX>;
  constexpr int W = S::W, NBW = S::NBW, RT = S::RT, CT = S::CT, NH = S::NH, PSTR = S::PSTR;
  constexpr int WB = W * BMAX;
  constexpr unsigned FULL = 0xffffffffu;
  static_assert(BMAX % 8 == 0 && BMAX <= 48, "window must be a multiple of 8, at most 48");
  extern __shared__ __align__(128) float tsm[];
  __shared__ __align__(8) uint64_t bars[2];
  const int lane_id = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int lane_g = lane_id >> 2, lane_q = lane_id & 3;
  const int groups_per_sub = (k + kLocalWarps - 1) / kLocalWarps;
  const int l = bidf() / groups_per_sub;
  const int i = (bidf() % groups_per_sub) * kLocalWarps + wib;
  const bool active = (i < k);
  const int ii = active ? i : 0;
  const int64_t off = sub_ptr[l];
  const int nl = (int)(sub_ptr[l + 1] - off);
  const int32_t* dofs = sub_dofs + off;
  const float lm = (float)lam[ii];
  float* Lrec = Lbuf + ((size_t)(off - rec_base) * k + (size_t)ii * nl) * BMAX;  // record of column j at Lrec + j BMAX
  float* yout = wpk + off * k + ii;                                // y_j at yout[j k]
  const float* gK = bandK + (size_t)off * BMAX;  // band row p at gK + p * BMAX, diagonal at BMAX - 1
  const float* gM = bandM + (size_t)off * BMAX;
  float* pbuf = tsm + 4 * WB + wib * S::PW;  // [RT 16][PSTR] panel / tensor-core operand
  float* srw = pbuf + RT * 16 * PSTR;        // [W] right-hand sides of the entering rows
  // chunk c = band rows [W (c + 1), W (c + 2)) ∩ [0, nl), into buffer c & 1
  int last_issued = -1, last_done = -1;  // thread 0: chunks issued / waited for successfully
  auto issue_chunk = [&](int c) {
    const int r0 = W * (c + 1);
    if (r0 >= nl) return;
    last_issued = c;
    const int rows = min(W, nl - r0);
    const uint32_t bytes = (uint32_t)rows * BMAX * sizeof(float);
    uint64_t* b = &bars[c & 1];
    mbar_expect_tx(b, 2 * bytes);
    bulk_load(tsm + (c & 1) * WB, gK + (size_t)r0 * BMAX, bytes, b);
    bulk_load(tsm + 2 * WB + (c & 1) * WB, gM + (size_t)r0 * BMAX, bytes, b);
  };
  if (threadIdx.x == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int e = lane_id; e < RT * 16 * PSTR; e += 32) pbuf[e] = 0.f;
  __syncthreads();
  if (threadIdx.x == 0) issue_chunk(0);
  // initial window: rows 0..W-1, negated, both triangles
  auto a0 = [&](int p, int qq) -> float {  // entry (p, qq) of the shifted matrix, qq <= p < W
    if (p >= nl) return (p == qq) ? 1.f : 0.f;
    const int d = p - qq;
    if (d > BMAX - 1) return 0.f;
    const int e = BMAX - 1 - d;
    return gK[(size_t)p * BMAX + e] - lm * gM[(size_t)p * BMAX + e];
  };
  auto rhs = [&](int p) -> float { return (p < nl) ? (float)rho[(int64_t)dofs[p] * k + ii] : 0.f; };
  float acc[RT][CT][4];
#pragma unroll
  for (int rt = 0; rt < RT; ++rt)
#pragma unroll
    for (int ct = 0; ct < CT; ++ct)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int u = rt * 16 + lane_g + 8 * (e >> 1), v = ct * 8 + 2 * lane_q + (e & 1);
        acc[rt][ct][e] = (u < W) ? -((u >= v) ? a0(u, v) : a0(v, u)) : 0.f;
      }
  float r[NH], rn[NH];
#pragma unroll
  for (int h = 0; h < NH; ++h) {
    const int w = lane_id + 32 * h;
    r[h] = (w < W) ? rhs(w) : 0.f;
    rn[h] = (w < W) ? rhs(W + w) : 0.f;
  }
  bool bad = false, timeout = false;
  int jm = 0;  // j0 mod BMAX
  for (int c = 0; c * W < nl; ++c) {
    __syncthreads();  // every warp is done with chunk c - 1: its buffer may be refilled
    if (threadIdx.x == 0 && !timeout) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue_chunk(c + 1);
    }
#pragma unroll
    for (int h = 0; h < NH; ++h) {
      const int w = lane_id + 32 * h;
      if (w < W) srw[w] = rn[h];
      rn[h] = (w < W) ? rhs(W * (c + 2) + w) : 0.f;
    }
    const bool have_chunk = W * (c + 1) < nl;
    if (have_chunk && !timeout) {
      if (mbar_wait_bounded(&bars[c & 1], (uint32_t)((c >> 1) & 1), wait_limit))
        last_done = c;
      else
        timeout = true;
    }
    const float* cK = tsm + (c & 1) * WB;
    const float* cM = tsm + 2 * WB + (c & 1) * WB;
    const int crow0 = W * (c + 1);  // band row of chunk row 0
#pragma unroll
    for (int sb = 0; sb < NBW; ++sb) {
      const int j0 = c * W + 8 * sb;
      if (j0 >= nl) break;
      // an opaque zero keeps the lane-dependent offsets of this block step from
      // being hoisted out of the cycle loop (NBW copies would occupy registers)
      int zero;
      asm volatile("mov.u32 %0, 0;" : "=r"(zero));
      const int g = lane_g + zero, q = lane_q + zero, lane = lane_id + zero;
      // 1. pivot column block -> pbuf[slot][0..7] (negated window values)
      __syncwarp();
#pragma unroll
      for (int rt = 0; rt < RT; ++rt) {
        *reinterpret_cast<float2*>(pbuf + (rt * 16 + g) * PSTR + 2 * q) = make_float2(acc[rt][sb][0], acc[rt][sb][1]);
        *reinterpret_cast<float2*>(pbuf + (rt * 16 + g + 8) * PSTR + 2 * q) =
            make_float2(acc[rt][sb][2], acc[rt][sb][3]);
      }
      __syncwarp();
      float p[NH][8];
      int dr[NH], pos[NH];
#pragma unroll
      for (int h = 0; h < NH; ++h) {
        const int w = lane + 32 * h;
        const float4 x0 = *reinterpret_cast<const float4*>(pbuf + (w < W ? w : 0) * PSTR);
        const float4 x1 = *reinterpret_cast<const float4*>(pbuf + (w < W ? w : 0) * PSTR + 4);
        const bool ok = w < W;
        p[h][0] = ok ? x0.x : 0.f;
        p[h][1] = ok ? x0.y : 0.f;
        p[h][2] = ok ? x0.z : 0.f;
        p[h][3] = ok ? x0.w : 0.f;
        p[h][4] = ok ? x1.x : 0.f;
        p[h][5] = ok ? x1.y : 0.f;
        p[h][6] = ok ? x1.z : 0.f;
        p[h][7] = ok ? x1.w : 0.f;
        int d = w - 8 * sb;
        d += (d < 0) ? W : 0;
        dr[h] = ok ? d : W + 8;  // rows past the window never store
        int ps = jm + d;
        ps -= (ps >= BMAX) ? BMAX : 0;
        ps -= (ps >= BMAX) ? BMAX : 0;
        pos[h] = ps;  // record position of this row: row mod BMAX
      }
      __syncwarp();  // pbuf is rewritten with L below
      // 2. panel factorisation, eight columns
      float* rec = Lrec + (size_t)j0 * BMAX;
#pragma unroll
      for (int cc = 0; cc < 8; ++cc) {
        const int ws = 8 * sb + cc;  // pivot slot
        const int own = ws & 31, hs = ws >> 5;
        const float piv = -__shfl_sync(FULL, p[hs][cc], own);
        const float rj = __shfl_sync(FULL, r[hs], own);
        bad |= !(piv > 0.f);
        const float inv = rsqrtf(piv);
        const float yj = rj * inv;
        float lv[NH];
#pragma unroll
        for (int h = 0; h < NH; ++h) {
          lv[h] = -p[h][cc] * inv;
          r[h] = fmaf(-lv[h], yj, r[h]);
        }
#pragma unroll
        for (int c2 = cc + 1; c2 < 8; ++c2) {
          const int w2 = 8 * sb + c2;
          const float l2 = __shfl_sync(FULL, lv[w2 >> 5], w2 & 31);
#pragma unroll
          for (int h = 0; h < NH; ++h) p[h][c2] = fmaf(lv[h], l2, p[h][c2]);
        }
        if (active && j0 + cc < nl) {
#pragma unroll
          for (int h = 0; h < NH; ++h) {
            const int tt = dr[h] - cc;
            if (tt >= 0 && tt < BMAX) rec[(size_t)cc * BMAX + pos[h]] = (tt == 0) ? inv : lv[h];
          }
          if (lane == 0) yout[(size_t)(j0 + cc) * k] = yj;
        }
#pragma unroll
        for (int h = 0; h < NH; ++h) p[h][cc] = lv[h];
      }
      // 3. L (W x 8) -> pbuf, tensor-core update of every tile: acc += L L^T
#pragma unroll
      for (int h = 0; h < NH; ++h) {
        const int w = lane + 32 * h;
        if (w < W) {
          *reinterpret_cast<float4*>(pbuf + w * PSTR) = make_float4(p[h][0], p[h][1], p[h][2], p[h][3]);
          *reinterpret_cast<float4*>(pbuf + w * PSTR + 4) = make_float4(p[h][4], p[h][5], p[h][6], p[h][7]);
        }
      }
      __syncwarp();
      uint32_t ah[RT][4], al[RT][4];
#pragma unroll
      for (int rt = 0; rt < RT; ++rt) {
        float x[4];
        x[0] = pbuf[(rt * 16 + g) * PSTR + q];
        x[1] = pbuf[(rt * 16 + g + 8) * PSTR + q];
        x[2] = pbuf[(rt * 16 + g) * PSTR + q + 4];
        x[3] = pbuf[(rt * 16 + g + 8) * PSTR + q + 4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          ah[rt][e] = to_tf32(x[e]);
          al[rt][e] = to_tf32(x[e] - __uint_as_float(ah[rt][e]));
        }
      }
#pragma unroll
      for (int rt = 0; rt < RT; ++rt)
#pragma unroll
        for (int ct = 0; ct < CT; ++ct) {
          if (!tile_live<NBW>(sb, rt, ct)) continue;  // compile-time: sb, rt, ct are unrolled
          const int bt = ct >> 1, bo = ct & 1;  // B operand = rows ct 8 .. of L: A fragment of tile bt
          mma_tf32(acc[rt][ct], al[rt], ah[bt][bo], ah[bt][bo + 2]);
          mma_tf32(acc[rt][ct], ah[rt], al[bt][bo], al[bt][bo + 2]);
          mma_tf32(acc[rt][ct], ah[rt], ah[bt][bo], ah[bt][bo + 2]);
        }
      // 4. band rows crow0 + 8 sb + du enter slot block sb (row tile sb / 2, half sb % 2),
      //    negated; this lane's row is du = g, its columns the slots ct 8 + 2 q + e2
      const int rtn = sb >> 1, hn = sb & 1;
      const int rowg = 8 * sb + g;
      const bool realg = crow0 + rowg < nl && !timeout;
      const float* kg = cK + rowg * BMAX;
      const float* mg = cM + rowg * BMAX;
#pragma unroll
      for (int ct = 0; ct < CT; ++ct)
#pragma unroll
        for (int e2 = 0; e2 < 2; ++e2) {
          float val;
          if (ct != sb) {
            // column slot v = ct 8 + 2 q + e2 holds row j0 + dv, dv = ((ct - sb) mod NBW) 8 + 2 q + e2;
            // entry (crow0 + 8 sb + g, j0 + dv) sits at band position dv - g - 9
            const int ps = ((ct - sb + NBW) % NBW) * 8 + e2 - 9 + 2 * q - g;
            val = (realg && ps >= 0) ? fmaf(lm, mg[ps], -kg[ps]) : 0.f;
          } else {
            const int du2 = 2 * q + e2;
            const int lo = (g >= du2) ? rowg : 8 * sb + du2;   // the later row of the pair
            const int ps = BMAX - 1 - ((g >= du2) ? g - du2 : du2 - g);
            const bool rl = crow0 + lo < nl && !timeout;
            val = rl ? fmaf(lm, cM[lo * BMAX + ps], -cK[lo * BMAX + ps]) : ((g == du2) ? -1.f : 0.f);
          }
          acc[rtn][ct][2 * hn + e2] = val;
        }
#pragma unroll
      for (int h = 0; h < NH; ++h) {
        const int w = lane + 32 * h;
        if (w < W && (w >> 3) == sb) r[h] = srw[w];
      }
      jm += 8;
      jm -= (jm >= BMAX) ? BMAX : 0;
    }
  }
  if ((bad || timeout) && lane_id == 0 && active) atomicOr(err, timeout ? kErrTimeout : kErrPivot);
  // thread 0 issued every copy: the ones it did not see complete (at most one per
  // barrier, since no copy is issued after a wait runs out) finish before the CTA exits
  if (threadIdx.x == 0)
    for (int c = last_done + 1; c <= last_issued; ++c)
      if (!mbar_drain(&bars[c & 1], (uint32_t)((c >> 1) & 1))) atomicOr(err, kErrDrain);
}

template <int BMAX>
__global__ void __launch_bounds__(128, (BMAX <= 40) ? 3 : 2) k_local_factor_mma(
    int nsub, int k, const int64_t* __restrict__ sub_ptr, const int32_t* __restrict__ sub_dofs,
    const float* __restrict__ bandK, const float* __restrict__ bandM, const double* __restrict__ lam,
    const double* __restrict__ rho, float* __restrict__ Lbuf, float* __restrict__ wpk, int32_t* err,
    int wait_limit, int64_t rec_base) {
  k_local_factor_mma_body<BMAX, BlockIdx>(BlockIdx(), nsub, k, sub_ptr, sub_dofs, bandK, bandM, lam, rho, Lbuf, wpk,
                                          err,
                                wait_limit, rec_base);
}

// ---------------------------------------------------------------------------
// Local solves, forward phase, blocked, for wide windows (B_pad = 64 or 96,
// e.g. 3-D subdomains): one CTA per (subdomain, shift) with one thread per
// window row (W = B_pad + 8 rows, NW = W / 32 rounded up warps).  The window
// lives (negated) in m16n8k8 accumulator tiles; warp w owns the column tiles
// ct = w, w + NW, ... of every row tile.  Per block step of eight columns:
//   1. the warp owning the pivot column block writes it to shared memory;
//   2. every thread reads its row of the panel and the 8 x 8 diagonal block,
//      factorises the diagonal block redundantly in registers and solves for
//      its own row of L (no barrier per column), eliminating its right-hand
//      side entry; pivot rows store 1/L_jj, all rows their L entries;
//   3. the L panel returns to shared memory and each warp applies the
//      trailing update W <- W - L L^T to its tiles (TF32 head/tail split);
//   4. each warp writes the entering band rows into its column tiles (values
//      read from the FP32 band in global memory at the start of the step).
// Records and y have the layout of k_local_factor_mma, so k_local_backward
// completes the solve.
// ---------------------------------------------------------------------------
template <int BMAX>
struct WideShape {
  static constexpr int W = BMAX + 8;
  static constexpr int NBW = W / 8;
  static constexpr int RT = (W + 15) / 16;
  static constexpr int CT = NBW;
  // warps per CTA: one window row per thread, and at most three column tiles per warp
  // (two above 128 rows, where the CTA has a whole SM: 80 accumulator registers)
  static constexpr int CTMAX = (W > 128) ? 2 : 3;
  static constexpr int NW = ((W + 31) / 32 > (CT + CTMAX - 1) / CTMAX) ? (W + 31) / 32 : (CT + CTMAX - 1) / CTMAX;
  static constexpr int CTW = (CT + NW - 1) / NW;  // column tiles per warp (at most)
  static constexpr int PSTR = 12;
  static constexpr int MINB = (W > 128) ? 1 : 2;  // resident CTAs per SM the registers are sized for
};

template <int BMAX>
__global__ void __launch_bounds__(WideShape<BMAX>::NW * 32, WideShape<BMAX>::MINB) k_local_factor_wide(
    int npairs, int k, const int64_t* __restrict__ sub_ptr, const int32_t* __restrict__ sub_dofs,
    const float* __restrict__ bandK, const float* __restrict__ bandM, const double* __restrict__ lam,
    const double* __restrict__ rho, float* __restrict__ Lbuf, float* __restrict__ wpk, int32_t* err,
    int64_t rec_base) {
  using S = WideShape<BMAX>;
  constexpr int W = S::W, NBW = S::NBW, RT = S::RT, CT = S::CT, NW = S::NW, CTW = S::CTW, PSTR = S::PSTR;
  static_assert(BMAX % 8 == 0 && CTW * 4 * RT <= 128, "window too wide for the register tiles");
  __shared__ __align__(16) float pbuf[RT * 16 * PSTR];  // panel, then L operand; rows >= W stay zero
  __shared__ float srhs[8];
  const int tid = threadIdx.x, lane_id = tid & 31, wid = tid >> 5;
  const int lane_g = lane_id >> 2, lane_q = lane_id & 3;
  const int pair = blockIdx.x;
  if (pair >= npairs) return;
  const int l = pair / k, i = pair % k;
  const int64_t off = sub_ptr[l];
  const int nl = (int)(sub_ptr[l + 1] - off);
  const int32_t* dofs = sub_dofs + off;
  const float lm = (float)lam[i];
  float* Lrec = Lbuf + ((size_t)(off - rec_base) * k + (size_t)i * nl) * BMAX;
  float* yout = wpk + off * k + i;
  const float* gK = bandK + (size_t)off * BMAX;  // band row p at gK + p * BMAX, diagonal at BMAX - 1
  const float* gM = bandM + (size_t)off * BMAX;
  for (int e = tid; e < RT * 16 * PSTR; e += blockDim.x) pbuf[e] = 0.f;
  // shifted entry (p, q), q <= p (identity rows beyond nl)
  auto a0 = [&](int p, int q) -> float {
    if (p >= nl) return (p == q) ? 1.f : 0.f;
    const int d = p - q;
    if (d > BMAX - 1 || q < 0) return 0.f;
    const int e = BMAX - 1 - d;
    return gK[(size_t)p * BMAX + e] - lm * gM[(size_t)p * BMAX + e];
  };
  auto rhs = [&](int p) -> float { return (p < nl) ? (float)rho[(int64_t)dofs[p] * k + i] : 0.f; };
  // initial window rows 0..W-1 (negated, both triangles) in this warp's column tiles
  float acc[RT][CTW][4];
#pragma unroll
  for (int rt = 0; rt < RT; ++rt)
#pragma unroll
    for (int jl = 0; jl < CTW; ++jl)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int ct = wid + NW * jl;
        const int u = rt * 16 + lane_g + 8 * (e >> 1), v = ct * 8 + 2 * lane_q + (e & 1);
        acc[rt][jl][e] = (ct < CT && u < W) ? -((u >= v) ? a0(u, v) : a0(v, u)) : 0.f;
      }
  float r = (tid < W) ? rhs(tid) : 0.f;  // right-hand side of this thread's window row
  bool bad = false;
  int jm = 0;  // j0 mod BMAX
  __syncthreads();
  for (int c = 0; c * W < nl; ++c) {
#pragma unroll
    for (int sb = 0; sb < NBW; ++sb) {
      const int j0 = c * W + 8 * sb;
      if (j0 >= nl) break;
      int zero;
      asm volatile("mov.u32 %0, 0;" : "=r"(zero));
      const int g = lane_g + zero, q = lane_q + zero, t = tid + zero;
      // entering band rows j0 + W + g (this lane's row of the entering block) for the
      // row part of this warp's column tiles, read now and written in step 4
      const int pnew = j0 + W + g;
      const bool realg = pnew < nl;
      float ek[CTW][2], em[CTW][2];
#pragma unroll
      for (int jl = 0; jl < CTW; ++jl)
#pragma unroll
        for (int e2 = 0; e2 < 2; ++e2) {
          const int ct = wid + NW * jl;
          float kv = 0.f, mv = 0.f;
          int pr = pnew, ps = -1;
          if (ct < CT) {
            if (ct != sb) {
              // column slot ct 8 + 2 q + e2 holds row j0 + dv, dv = ((ct - sb) mod NBW) 8 + 2 q + e2
              ps = ((ct - sb + NBW) % NBW) * 8 + e2 - 9 + 2 * q - g;
            } else {
              const int du2 = 2 * q + e2;
              pr = (g >= du2) ? pnew : j0 + W + du2;  // the later row of the pair
              ps = BMAX - 1 - ((g >= du2) ? g - du2 : du2 - g);
            }
          }
          if (ps >= 0 && pr < nl) {
            kv = gK[(size_t)pr * BMAX + ps];
            mv = gM[(size_t)pr * BMAX + ps];
          }
          ek[jl][e2] = kv;
          em[jl][e2] = mv;
        }
      const int d8 = t - 8 * sb;  // position of this row in the pivot block (0..7 there)
      const float rnew = (d8 >= 0 && d8 < 8) ? rhs(pnew - g + d8) : 0.f;
      // 1. pivot column block -> pbuf[slot][0..7]; pivot right-hand sides -> srhs
      if (wid == sb % NW) {
#pragma unroll
        for (int rt = 0; rt < RT; ++rt) {
          *reinterpret_cast<float2*>(pbuf + (rt * 16 + g) * PSTR + 2 * q) =
              make_float2(acc[rt][sb / NW][0], acc[rt][sb / NW][1]);
          *reinterpret_cast<float2*>(pbuf + (rt * 16 + g + 8) * PSTR + 2 * q) =
              make_float2(acc[rt][sb / NW][2], acc[rt][sb / NW][3]);
        }
      }
      if (d8 >= 0 && d8 < 8) srhs[d8] = r;
      __syncthreads();
      // 2. own row of the panel and the diagonal block, both negated back
      int dr = t - 8 * sb;
      dr += (dr < 0) ? W : 0;
      const bool row_ok = t < W;
      float p[8];
      {
        const float4 x0 = *reinterpret_cast<const float4*>(pbuf + (row_ok ? t : 0) * PSTR);
        const float4 x1 = *reinterpret_cast<const float4*>(pbuf + (row_ok ? t : 0) * PSTR + 4);
        p[0] = -x0.x; p[1] = -x0.y; p[2] = -x0.z; p[3] = -x0.w;
        p[4] = -x1.x; p[5] = -x1.y; p[6] = -x1.z; p[7] = -x1.w;
      }
      float D[8][8];  // lower triangle used
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const float4 x0 = *reinterpret_cast<const float4*>(pbuf + (8 * sb + a) * PSTR);
        const float4 x1 = *reinterpret_cast<const float4*>(pbuf + (8 * sb + a) * PSTR + 4);
        D[a][0] = -x0.x; D[a][1] = -x0.y; D[a][2] = -x0.z; D[a][3] = -x0.w;
        D[a][4] = -x1.x; D[a][5] = -x1.y; D[a][6] = -x1.z; D[a][7] = -x1.w;
      }
      float yv[8];
#pragma unroll
      for (int a = 0; a < 8; ++a) yv[a] = srhs[a];
      __syncthreads();  // pbuf and srhs are rewritten below
      // Cholesky of the diagonal block (every thread), inverse diagonal in dinv
      float dinv[8];
#pragma unroll
      for (int cc = 0; cc < 8; ++cc) {
        float s = D[cc][cc];
#pragma unroll
        for (int b = 0; b < cc; ++b) s = fmaf(-D[cc][b], D[cc][b], s);
        bad |= !(s > 0.f);
        const float inv = rsqrtf(s);
        dinv[cc] = inv;
        D[cc][cc] = s * inv;
#pragma unroll
        for (int a = cc + 1; a < 8; ++a) {
          float v = D[a][cc];
#pragma unroll
          for (int b = 0; b < cc; ++b) v = fmaf(-D[a][b], D[cc][b], v);
          D[a][cc] = v * inv;
        }
      }
      // y = L_dd^{-1} rhs of the pivot rows
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        float v = yv[a];
#pragma unroll
        for (int b = 0; b < a; ++b) v = fmaf(-D[a][b], yv[b], v);
        yv[a] = v * dinv[a];
      }
      // own row of L: l = p L_dd^{-T}; for a pivot row (dr < 8) this reproduces row dr
      // of L_dd, whose entries past the diagonal are cleared
      float lr[8];
#pragma unroll
      for (int cc = 0; cc < 8; ++cc) {
        float v = p[cc];
#pragma unroll
        for (int b = 0; b < cc; ++b) v = fmaf(-lr[b], D[cc][b], v);
        lr[cc] = v * dinv[cc];
      }
      if (dr < 8) {
#pragma unroll
        for (int cc = 0; cc < 8; ++cc)
          if (cc > dr) lr[cc] = 0.f;
      } else {
#pragma unroll
        for (int cc = 0; cc < 8; ++cc) r = fmaf(-lr[cc], yv[cc], r);
      }
      if (!row_ok) {
#pragma unroll
        for (int cc = 0; cc < 8; ++cc) lr[cc] = 0.f;
      }
      // records: column j0 + cc holds L(row, j0 + cc) at row mod BMAX, 1/L_jj at the pivot
      if (row_ok) {
        int pos = jm + dr;
        pos -= (pos >= BMAX) ? BMAX : 0;
        pos -= (pos >= BMAX) ? BMAX : 0;
        float* rec = Lrec + (size_t)j0 * BMAX + pos;
#pragma unroll
        for (int cc = 0; cc < 8; ++cc) {
          const int tt = dr - cc;
          if (j0 + cc < nl && tt >= 0 && tt < BMAX) rec[(size_t)cc * BMAX] = (tt == 0) ? dinv[cc] : lr[cc];
        }
      }
      if (t == 0) {
#pragma unroll
        for (int cc = 0; cc < 8; ++cc)
          if (j0 + cc < nl) yout[(size_t)(j0 + cc) * k] = yv[cc];
      }
      // 3. L panel -> pbuf, trailing update of this warp's tiles
      if (row_ok) {
        *reinterpret_cast<float4*>(pbuf + t * PSTR) = make_float4(lr[0], lr[1], lr[2], lr[3]);
        *reinterpret_cast<float4*>(pbuf + t * PSTR + 4) = make_float4(lr[4], lr[5], lr[6], lr[7]);
      }
      __syncthreads();
      uint32_t bh[CTW][2], bl[CTW][2];
#pragma unroll
      for (int jl = 0; jl < CTW; ++jl) {
        const int ct = wid + NW * jl;
        const int row = (ct < CT ? ct : 0) * 8 + g;
        const float x0 = pbuf[row * PSTR + q], x1 = pbuf[row * PSTR + q + 4];
        bh[jl][0] = to_tf32(x0);
        bl[jl][0] = to_tf32(x0 - __uint_as_float(bh[jl][0]));
        bh[jl][1] = to_tf32(x1);
        bl[jl][1] = to_tf32(x1 - __uint_as_float(bh[jl][1]));
      }
#pragma unroll
      for (int rt = 0; rt < RT; ++rt) {
        float x[4];
        x[0] = pbuf[(rt * 16 + g) * PSTR + q];
        x[1] = pbuf[(rt * 16 + g + 8) * PSTR + q];
        x[2] = pbuf[(rt * 16 + g) * PSTR + q + 4];
        x[3] = pbuf[(rt * 16 + g + 8) * PSTR + q + 4];
        uint32_t ah[4], al[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          ah[e] = to_tf32(x[e]);
          al[e] = to_tf32(x[e] - __uint_as_float(ah[e]));
        }
#pragma unroll
        for (int jl = 0; jl < CTW; ++jl) {
          const int ct = wid + NW * jl;
          if (ct >= CT || !tile_live<NBW>(sb, rt, ct)) continue;  // warp-uniform
          mma_tf32(acc[rt][jl], al, bh[jl][0], bh[jl][1]);
          mma_tf32(acc[rt][jl], ah, bl[jl][0], bl[jl][1]);
          mma_tf32(acc[rt][jl], ah, bh[jl][0], bh[jl][1]);
        }
      }
      // 4. entering rows into slot block sb (row tile sb / 2, half sb % 2), negated
      {
        const int rtn = sb >> 1, hn = sb & 1;
#pragma unroll
        for (int jl = 0; jl < CTW; ++jl)
#pragma unroll
          for (int e2 = 0; e2 < 2; ++e2) {
            const int ct = wid + NW * jl;
            float val = fmaf(lm, em[jl][e2], -ek[jl][e2]);
            if (ct == sb) {
              const int du2 = 2 * q + e2;
              const int pr = (g >= du2) ? pnew : j0 + W + du2;
              if (pr >= nl) val = (g == du2) ? -1.f : 0.f;
            }
            acc[rtn][jl][2 * hn + e2] = val;
          }
      }
      if (d8 >= 0 && d8 < 8) r = rnew;
      __syncthreads();  // pbuf is rewritten by the next extraction
      jm += 8;
      jm -= (jm >= BMAX) ? BMAX : 0;
    }
  }
  if (bad && tid == 0) atomicOr(err, 1);
}

// ---------------------------------------------------------------------------
// Local solves, backward phase: L^T x = y for every (subdomain, shift), L in
// slot order as written by the factorisation (row j of the record holds
// L(row(v), j) at slot v and 1/L_jj at slot j mod BMAX).  A warp serves four
// shifts of one subdomain, eight lanes each; lane e of a group owns the window
// slots e + 8 c and keeps x of their rows in registers, so a row costs one
// eight-lane reduction.  The records enter shared memory R rows at a time (half
// a window group up to windows of 48, 16 rows beyond) through one bulk copy
// per shift, double buffered; a window group holds an even number of chunks,
// so slots and buffers are static in the unrolled loop; y of the next chunk is
// loaded into registers one chunk ahead.
// ---------------------------------------------------------------------------
template <int BMAX>
struct BwdShape {
  // rows per staged chunk: R divides BMAX into an even number of chunks
  static constexpr int R = (BMAX <= 48) ? BMAX / 2 : ((BMAX % 32 == 0) ? 16 : BMAX / 8);
  static constexpr int NCH = BMAX / R;  // chunks per window group (even)
  static constexpr int PS = R * BMAX + 8;  // per-shift buffer stride: shifts land on different banks
  static constexpr int WPB = 2;            // warps per block
  static constexpr size_t smem_floats = (size_t)WPB * 2 * 4 * PS;
};

template <int BMAX, class BID>
__device__ __forceinline__ void k_local_backward_body(BID bidf, int nsub, int k, const int64_t* __restrict__ sub_ptr,
                                                       const float* __restrict__ Lbuf, float* __restrict__ wpk,
                                                       int32_t* err, int wait_limit, int64_t rec_base) {
  using S = BwdShape<BMAX>;
  constexpr int TC = BMAX / 8, R = S::R, PS = S::PS, WPB = S::WPB;
  constexpr int NY = (R + 7) / 8;
  constexpr unsigned FULL = 0xffffffffu;
  static_assert(BMAX % 8 == 0, "window must be a multiple of 8");
  extern __shared__ __align__(128) float bsm[];
  __shared__ __align__(8) uint64_t bars[WPB][2];
  const int lane = threadIdx.x & 31, e = lane & 7, p = lane >> 3, wib = threadIdx.x >> 5;
  const int wglob = bidf() * WPB + wib;
  const int wps = (k + 3) / 4;  // warps per subdomain
  const int l = wglob / wps;
  if (l >= nsub) return;  // whole warps only; no block-wide barrier follows
  const int i0 = (wglob % wps) * 4;
  const int nact = min(4, k - i0);  // shifts served by this warp
  const bool active = p < nact;
  const int ii = active ? i0 + p : i0;
  const int64_t off = sub_ptr[l];
  const int nl = (int)(sub_ptr[l + 1] - off);
  float* buf = bsm + (size_t)wib * 2 * 4 * PS;  // [2][4][PS]
  uint64_t* bar = bars[wib];
  const float* Lsub = Lbuf + (size_t)(off - rec_base) * k * BMAX;  // record of shift i at Lsub + i nl BMAX
  float* yp = wpk + off * k + ii;
  if (lane == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  const int chtop = (nl - 1) / R;
  // lane 0: lowest chunk issued and lowest chunk waited for successfully (chunks go
  // from chtop down to 0)
  int low_issued = chtop + 1, low_done = chtop + 1;
  // chunk ch = rows [ch R, min(nl, ch R + R)) of each served shift, into buffer ch & 1
  auto issue = [&](int ch) {
    if (ch < 0) return;
    low_issued = ch;
    const int r0 = ch * R;
    const int rows = min(R, nl - r0);
    const uint32_t bytes = (uint32_t)rows * BMAX * sizeof(float);
    uint64_t* b = &bar[ch & 1];
    mbar_expect_tx(b, bytes * nact);
    for (int q = 0; q < nact; ++q)
      bulk_load(buf + ((ch & 1) * 4 + q) * PS, Lsub + ((size_t)(i0 + q) * nl + r0) * BMAX, bytes, b);
  };
  auto load_y = [&](int ch, float* y) {
#pragma unroll
    for (int q = 0; q < NY; ++q) {
      const int r = e + 8 * q;
      const int j = ch * R + r;
      y[q] = (ch >= 0 && r < R && j < nl) ? yp[(size_t)j * k] : 0.f;
    }
  };
  if (lane == 0) issue(chtop);
  float ycur[NY], ynext[NY];
  load_y(chtop, ynext);
  float xw[TC];
#pragma unroll
  for (int c = 0; c < TC; ++c) xw[c] = 0.f;
  uint32_t ph[2] = {0u, 0u};
  bool timeout = false;
  constexpr int NCH = S::NCH;
  static_assert(NCH % 2 == 0, "chunk parity must be static inside a window group");
  for (int g = chtop / NCH; g >= 0; --g) {
#pragma unroll
    for (int hc = NCH - 1; hc >= 0; --hc) {
      const int ch = g * NCH + hc;
      const int half = hc & 1;  // buffer of chunk ch
      if (ch > chtop) continue;
      __syncwarp();  // the buffer of chunk ch - 1 (chunk ch + 1's) is no longer read
      if (lane == 0 && !timeout) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue(ch - 1);
      }
#pragma unroll
      for (int q = 0; q < NY; ++q) ycur[q] = ynext[q];
      load_y(ch - 1, ynext);
      if (!timeout) {
        if (mbar_wait_bounded(&bar[half], ph[half], wait_limit))
          low_done = ch;
        else
          timeout = true;
      }
      ph[half] ^= 1u;
      const float* Lb = buf + (half * 4 + p) * PS;
#pragma unroll
      for (int r = R - 1; r >= 0; --r) {
        const int j = ch * R + r;
        const int s = hc * R + r;  // j mod BMAX
        if (j < nl) {
          const float* row = Lb + r * BMAX;
          float part = 0.f, dg = 0.f;
#pragma unroll
          for (int c = 0; c < TC; ++c) {
            const float lv = row[e + 8 * c];
            if (c == s / 8 && e == s % 8)
              dg = lv;
            else
              part = fmaf(lv, xw[c], part);
          }
          part += __shfl_xor_sync(FULL, part, 1);
          part += __shfl_xor_sync(FULL, part, 2);
          part += __shfl_xor_sync(FULL, part, 4);
          dg = __shfl_sync(FULL, dg, (lane & ~7) | (s % 8));
          const float y = __shfl_sync(FULL, ycur[r / 8], (lane & ~7) | (r % 8));
          const float xj = (y - part) * dg;
          if (e == s % 8) xw[s / 8] = xj;
          if (e == 0 && active && !timeout) yp[(size_t)j * k] = xj;
        }
      }
    }
  }
  if (timeout && lane == 0) atomicOr(err, kErrTimeout);
  // lane 0 issued every copy of this warp: drain the ones it did not see complete
  // (chunk ch is the floor((chtop - ch) / 2)-th use of its barrier)
  if (lane == 0)
    for (int ch = low_done - 1; ch >= low_issued; --ch)
      if (!mbar_drain(&bar[ch & 1], (uint32_t)(((chtop - ch) >> 1) & 1))) atomicOr(err, kErrDrain);
}

template <int BMAX>
__global__ void __launch_bounds__(64, 1) k_local_backward(int nsub, int k, const int64_t* __restrict__ sub_ptr,
                                                       const float* __restrict__ Lbuf, float* __restrict__ wpk,
                                                       int32_t* err, int wait_limit, int64_t rec_base) {
  k_local_backward_body<BMAX, BlockIdx>(BlockIdx(), nsub, k, sub_ptr, Lbuf, wpk, err, wait_limit, rec_base);
}

// ---------------------------------------------------------------------------
// Local solves, forward substitution L y = R_l rho_i with stored band factors,
// for the applications that reuse the factors of an earlier one (the
// factorisation kernels fuse this sweep into the factorisation).  Same warp
// layout, records and staging as k_local_backward: four shifts per warp, eight
// lanes per shift, lane e keeping the pending right-hand sides of the window
// slots e + 8 c (slot = row mod BMAX); records enter shared memory in chunks of
// R rows by bulk copies, double buffered, in ascending order.  Column j
// (right-looking, the operation order of the fused sweep): y_j = r_j / L_jj,
// then r_r -= L(r, j) y_j for the rows r of column j's band, and row j + BMAX
// enters the freed slot.
// ---------------------------------------------------------------------------
template <int BMAX, class BID>
__device__ __forceinline__ void k_local_forward_body(BID bidf, int nsub, int k, const int64_t* __restrict__ sub_ptr,
                                                      const int32_t* __restrict__ sub_dofs,
                                                      const double* __restrict__ rho, const float* __restrict__ Lbuf,
                                                      float* __restrict__ wpk, int32_t* err, int wait_limit,
                                                      int64_t rec_base) {
  using S = BwdShape<BMAX>;
  constexpr int TC = BMAX / 8, R = S::R, PS = S::PS, WPB = S::WPB;
  constexpr int NY = (R + 7) / 8;
  constexpr unsigned FULL = 0xffffffffu;
  static_assert(BMAX % 8 == 0, "window must be a multiple of 8");
  extern __shared__ __align__(128) float fsm[];
  __shared__ __align__(8) uint64_t bars[WPB][2];
  const int lane = threadIdx.x & 31, e = lane & 7, p = lane >> 3, wib = threadIdx.x >> 5;
  const int wglob = bidf() * WPB + wib;
  const int wps = (k + 3) / 4;  // warps per subdomain
  const int l = wglob / wps;
  if (l >= nsub) return;  // whole warps only; no block-wide barrier follows
  const int i0 = (wglob % wps) * 4;
  const int nact = min(4, k - i0);  // shifts served by this warp
  const bool active = p < nact;
  const int ii = active ? i0 + p : i0;
  const int64_t off = sub_ptr[l];
  const int nl = (int)(sub_ptr[l + 1] - off);
  const int32_t* dofs = sub_dofs + off;
  float* buf = fsm + (size_t)wib * 2 * 4 * PS;  // [2][4][PS]
  uint64_t* bar = bars[wib];
  const float* Lsub = Lbuf + (size_t)(off - rec_base) * k * BMAX;  // record of shift i at Lsub + i nl BMAX
  float* yp = wpk + off * k + ii;
  if (lane == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  const int nch = (nl + R - 1) / R;
  int hi_issued = -1, hi_done = -1;  // lane 0: last chunk issued / waited for successfully
  // chunk ch = rows [ch R, min(nl, ch R + R)) of each served shift, into buffer ch & 1
  auto issue = [&](int ch) {
    if (ch >= nch) return;
    hi_issued = ch;
    const int r0 = ch * R;
    const int rows = min(R, nl - r0);
    const uint32_t bytes = (uint32_t)rows * BMAX * sizeof(float);
    uint64_t* b = &bar[ch & 1];
    mbar_expect_tx(b, bytes * nact);
    for (int q = 0; q < nact; ++q)
      bulk_load(buf + ((ch & 1) * 4 + q) * PS, Lsub + ((size_t)(i0 + q) * nl + r0) * BMAX, bytes, b);
  };
  auto rhs = [&](int row) -> float { return (row < nl) ? (float)rho[(int64_t)dofs[row] * k + ii] : 0.f; };
  // right-hand sides of the rows entering during chunk ch (rows ch R + r + BMAX), lane r % 8,
  // fetched in two stages so that no load waits on another: the dof indices two chunks
  // ahead, the values (from indices already in registers) one chunk ahead
  auto load_dofs = [&](int ch, int* dv) {
#pragma unroll
    for (int q = 0; q < NY; ++q) {
      const int r = e + 8 * q, row = ch * R + r + BMAX;
      dv[q] = (r < R && row < nl) ? dofs[row] : -1;
    }
  };
  auto load_vals = [&](const int* dv, float* v) {
#pragma unroll
    for (int q = 0; q < NY; ++q) v[q] = (dv[q] >= 0) ? (float)rho[(int64_t)dv[q] * k + ii] : 0.f;
  };
  if (lane == 0) issue(0);
  float rw[TC];
#pragma unroll
  for (int c = 0; c < TC; ++c) rw[c] = rhs(e + 8 * c);
  float incur[NY], innext[NY];
  int dnext[NY];
  {
    int d0[NY];
    load_dofs(0, d0);
    load_vals(d0, innext);
    load_dofs(1, dnext);
  }
  uint32_t ph[2] = {0u, 0u};
  bool timeout = false;
  constexpr int NCH = S::NCH;
  static_assert(NCH % 2 == 0, "chunk parity must be static inside a window group");
  for (int g = 0; g * NCH < nch; ++g) {
#pragma unroll
    for (int hc = 0; hc < NCH; ++hc) {
      const int ch = g * NCH + hc;
      const int half = hc & 1;  // buffer of chunk ch
      if (ch >= nch) continue;
      __syncwarp();  // the buffer of chunk ch - 1 (chunk ch + 1's) is no longer read
      if (lane == 0 && !timeout) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue(ch + 1);
      }
#pragma unroll
      for (int q = 0; q < NY; ++q) incur[q] = innext[q];
      load_vals(dnext, innext);  // chunk ch + 1
      load_dofs(ch + 2, dnext);
      if (!timeout) {
        if (mbar_wait_bounded(&bar[half], ph[half], wait_limit))
          hi_done = ch;
        else
          timeout = true;
      }
      ph[half] ^= 1u;
      const float* Lb = buf + (half * 4 + p) * PS;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int j = ch * R + r;
        const int s = hc * R + r;  // j mod BMAX
        if (j < nl) {
          const float* row = Lb + r * BMAX;
          const float rj = __shfl_sync(FULL, rw[s / 8], (lane & ~7) | (s % 8));
          const float yj = rj * row[s];  // 1 / L_jj at the diagonal slot
          if (e == 0 && active && !timeout) yp[(size_t)j * k] = yj;
#pragma unroll
          for (int c = 0; c < TC; ++c)
            if (!(c == s / 8 && e == s % 8)) rw[c] = fmaf(-row[e + 8 * c], yj, rw[c]);
          const float nv = __shfl_sync(FULL, incur[r / 8], (lane & ~7) | (r % 8));
          if (e == s % 8) rw[s / 8] = nv;
        }
      }
    }
  }
  if (timeout && lane == 0) atomicOr(err, kErrTimeout);
  // lane 0 issued every copy of this warp: drain the ones it did not see complete
  if (lane == 0)
    for (int ch = hi_done + 1; ch <= hi_issued; ++ch)
      if (!mbar_drain(&bar[ch & 1], (uint32_t)((ch >> 1) & 1))) atomicOr(err, kErrDrain);
}

template <int BMAX>
__global__ void __launch_bounds__(64, 1) k_local_forward(int nsub, int k, const int64_t* __restrict__ sub_ptr,
                                                      const int32_t* __restrict__ sub_dofs,
                                                      const double* __restrict__ rho, const float* __restrict__ Lbuf,
                                                      float* __restrict__ wpk, int32_t* err, int wait_limit,
                                                      int64_t rec_base) {
  k_local_forward_body<BMAX, BlockIdx>(BlockIdx(), nsub, k, sub_ptr, sub_dofs, rho, Lbuf, wpk, err, wait_limit,
                                       rec_base);
}


// ---------------------------------------------------------------------------
// Blocked sweeps with the stored band factors (window tiers up to 48): the
// rows are taken eight at a time, one block per staged chunk, so that a
// block's eight columns are handled together instead of one dependent row at a
// time.  Layout as in k_local_backward (four shifts per warp, eight lanes per
// shift, lane e keeping window slots e + 8 t, slot = row mod BMAX).  The blocks
// of records enter shared memory by bulk copies into a ring of nbuf buffers per
// warp, so the copies run nbuf - 1 blocks ahead; nbuf is a launch parameter,
// the largest ring whose shared memory still lets every warp of the launch be
// resident at once (sweep_ring_buffers).
//   backward: for the block's columns q (rows j0 + q), the partial sums over the
//   solved window rows run in parallel (lane partials, three xor shuffles
//   each), then the 8 x 8 triangle is solved redundantly in every lane;
//   forward: the 8 x 8 triangle first (the fused sweep's operation order), then
//   every other window row takes the block's eight updates in column order, and
//   the eight entering rows take theirs, so that y equals the fused sweep's bit
//   for bit.
// The per-row values that come from global memory (y for the backward sweep,
// the gathered right-hand side rho for the forward sweep) are loaded NCH blocks
// ahead into a register ring indexed by the block's window slot block (the dof
// index of the gather 2 NCH blocks ahead), so that a block step does not wait
// for a global load issued one step earlier.
// ---------------------------------------------------------------------------
template <int BMAX>
struct BlkShape {
  static constexpr int NCH = BMAX / 8;      // blocks (chunks) per window group
  static constexpr int PS = 8 * BMAX + 4;   // per-shift buffer stride
  static constexpr int WPB = 2;             // warps per block
  static constexpr int NBUF_MAX = 16;       // ring buffers per warp, at most
  // dynamic shared memory of a block with nbuf buffers per warp
  static size_t smem_floats(int nbuf) { return (size_t)WPB * nbuf * 4 * PS; }
};

template <int BMAX, bool FWD, class BID>
__device__ __forceinline__ void k_local_sweep_blk_body(BID bidf, int nsub, int k, const int64_t* __restrict__ sub_ptr,
                                                        const int32_t* __restrict__ sub_dofs,
                                                        const double* __restrict__ rho,
                                                        const float* __restrict__ Lbuf, float* __restrict__ wpk,
                                                        int32_t* err, int wait_limit, int64_t rec_base,
                                                        int nbuf) {
  using S = BlkShape<BMAX>;
  constexpr int TC = BMAX / 8, NCH = S::NCH, PS = S::PS, WPB = S::WPB;
  constexpr unsigned FULL = 0xffffffffu;
  static_assert(BMAX % 8 == 0 && BMAX <= 48, "window tier of the blocked sweeps");
  extern __shared__ __align__(128) float ssm[];
  __shared__ __align__(8) uint64_t bars[WPB][S::NBUF_MAX];
  const int lane = threadIdx.x & 31, e = lane & 7, p = lane >> 3, wib = threadIdx.x >> 5;
  const int wglob = bidf() * WPB + wib;
  const int wps = (k + 3) / 4;  // warps per subdomain
  const int l = wglob / wps;
  if (l >= nsub) return;  // whole warps only; no block-wide barrier follows
  const int i0 = (wglob % wps) * 4;
  const int nact = min(4, k - i0);  // shifts served by this warp
  const bool active = p < nact;
  const int ii = active ? i0 + p : i0;
  const int64_t off = sub_ptr[l];
  const int nl = (int)(sub_ptr[l + 1] - off);
  const int32_t* dofs = sub_dofs + off;
  float* buf = ssm + (size_t)wib * nbuf * 4 * PS;  // [nbuf][4][PS]
  uint64_t* bar = bars[wib];
  const float* Lsub = Lbuf + (size_t)(off - rec_base) * k * BMAX;  // record of shift i at Lsub + i nl BMAX
  float* yp = wpk + off * k + ii;
  if (lane == 0) {
    for (int b = 0; b < nbuf; ++b) mbar_init(&bar[b], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  const int nblk = (nl + 7) / 8;
  // Blocks are copied and consumed in processing order: position q is block q
  // (forward) or nblk - 1 - q (backward), in buffer q mod nbuf, whose wait has
  // parity (q / nbuf) & 1.  Lane 0 issues the copies and counts the positions
  // issued and waited for (for the drain on a timeout).
  int n_issued = 0, n_done = 0;
  // position q = rows [8 ch, min(nl, 8 ch + 8)) of each served shift, into buffer b
  auto issue = [&](int q, int b) {
    if (q >= nblk) return;
    const int ch = FWD ? q : nblk - 1 - q;
    const int r0 = 8 * ch;
    const int rows = min(8, nl - r0);
    const uint32_t bytes = (uint32_t)rows * BMAX * sizeof(float);
    mbar_expect_tx(&bar[b], bytes * nact);
    for (int t = 0; t < nact; ++t)
      bulk_load(buf + (b * 4 + t) * PS, Lsub + ((size_t)(i0 + t) * nl + r0) * BMAX, bytes, &bar[b]);
    n_issued = q + 1;
  };
  auto rhs = [&](int row) -> float { return (row < nl) ? (float)rho[(int64_t)dofs[row] * k + ii] : 0.f; };
  float w[TC];  // backward: x of the window rows; forward: their pending right-hand sides
#pragma unroll
  for (int t = 0; t < TC; ++t) w[t] = FWD ? rhs(e + 8 * t) : 0.f;
  // per block, lane e's row j0 + e: y (backward) or the entering row's right-hand
  // side (forward); ring slot b holds the value of the next block of window slot
  // block b (NCH blocks ahead), dring[b] the dof index of the block after that
  float vring[NCH];
  int dring[NCH];
  auto row_of = [&](int ch) { return 8 * ch + e + (FWD ? BMAX : 0); };
  auto dof_of = [&](int ch) -> int {
    const int r = row_of(ch);
    return (ch >= 0 && ch < nblk && r < nl) ? dofs[r] : -1;
  };
  auto fetch = [&](int ch) -> float {
    const int r = row_of(ch);
    if (ch < 0 || ch >= nblk || r >= nl) return 0.f;
    return FWD ? 0.f : yp[(size_t)r * k];
  };
  int qpos = 0, qbuf = 0;   // processing position and its buffer
  uint32_t qpar = 0;        // parity of its wait
  int ibuf = nbuf - 1;      // buffer of position qpos + nbuf - 1, issued at position qpos
  bool timeout = false;
  const int g0 = FWD ? 0 : (nblk - 1) / NCH, g1 = FWD ? (nblk - 1) / NCH : 0;
  if (FWD) {
    if (lane == 0)
      for (int b = 0; b < nbuf - 1; ++b) issue(b, b);
#pragma unroll
    for (int b = 0; b < NCH; ++b) {
      const int d = dof_of(b);
      vring[b] = (d >= 0) ? (float)rho[(int64_t)d * k + ii] : 0.f;
      dring[b] = dof_of(b + NCH);
    }
  } else {
    if (lane == 0)
      for (int b = 0; b < nbuf - 1; ++b) issue(b, b);
#pragma unroll
    for (int b = 0; b < NCH; ++b) {
      // the first block processed in window slot block b
      const int c0 = g0 * NCH + b;
      vring[b] = fetch(c0 < nblk ? c0 : c0 - NCH);
      dring[b] = -1;
    }
  }
  for (int g = g0; FWD ? (g <= g1) : (g >= g1); g += FWD ? 1 : -1) {
#pragma unroll
    for (int hq = 0; hq < NCH; ++hq) {
      const int hc = FWD ? hq : NCH - 1 - hq;  // window slot block of this block
      const int ch = g * NCH + hc;
      if (ch >= nblk) continue;
      __syncwarp();  // the buffer of the previous position is no longer read
      if (lane == 0 && !timeout) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        // the previous position's buffer takes the position nbuf - 1 ahead
        issue(qpos + nbuf - 1, ibuf);
      }
      ibuf = (ibuf + 1 == nbuf) ? 0 : ibuf + 1;
      const float vcur = vring[hc];
      if (FWD) {
        vring[hc] = (dring[hc] >= 0) ? (float)rho[(int64_t)dring[hc] * k + ii] : 0.f;
        dring[hc] = dof_of(ch + 2 * NCH);
      } else {
        vring[hc] = fetch(ch - NCH);
      }
      if (!timeout) {
        if (mbar_wait_bounded(&bar[qbuf], qpar, wait_limit))
          n_done = qpos + 1;
        else
          timeout = true;
      }
      const float* Lb = buf + (qbuf * 4 + p) * PS;  // records of rows 8 ch .. 8 ch + 7 (shift p)
      ++qpos;
      if (++qbuf == nbuf) {
        qbuf = 0;
        qpar ^= 1u;
      }
      const int j0 = 8 * ch;
      const int nr = min(8, nl - j0);
      const int s0 = 8 * hc;  // slot of row j0
      float xb[8];
      if (FWD) {
        // the block's pending right-hand sides, then its 8 x 8 triangle
#pragma unroll
        for (int q = 0; q < 8; ++q) xb[q] = __shfl_sync(FULL, w[hc], (lane & ~7) | q);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          float r = xb[q];
#pragma unroll
          for (int d = 0; d < q; ++d) r = fmaf(-Lb[d * BMAX + s0 + q], xb[d], r);
          xb[q] = (q < nr) ? r * Lb[q * BMAX + s0 + q] : 0.f;
        }
        // other window rows: the block's updates in column order
#pragma unroll
        for (int t = 0; t < TC; ++t) {
          if (t == hc) continue;
#pragma unroll
          for (int d = 0; d < 8; ++d)
            if (d < nr) w[t] = fmaf(-Lb[d * BMAX + e + 8 * t], xb[d], w[t]);
        }
        // the entering row j0 + BMAX + e takes slot s0 + e and the updates of the
        // block's later columns
        {
          const float nv = __shfl_sync(FULL, vcur, (lane & ~7) | e);
          float r = nv;
#pragma unroll
          for (int d = 1; d < 8; ++d)
            if (d > e && d < nr) r = fmaf(-Lb[d * BMAX + s0 + e], xb[d], r);
          w[hc] = r;
        }
      } else {
        // partial sums over the solved window rows for the block's columns: lane e's
        // slot s0 + e holds row j0 + e + BMAX, in column q's band iff e < q
        float part[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          float a = 0.f;
#pragma unroll
          for (int t = 0; t < TC; ++t) {
            const float lv = Lb[q * BMAX + e + 8 * t];
            a = (t != hc || e < q) ? fmaf(lv, w[t], a) : a;
          }
          part[q] = a;
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          part[q] += __shfl_xor_sync(FULL, part[q], 1);
          part[q] += __shfl_xor_sync(FULL, part[q], 2);
          part[q] += __shfl_xor_sync(FULL, part[q], 4);
        }
        // the 8 x 8 triangle, descending
#pragma unroll
        for (int qq = 0; qq < 8; ++qq) {
          const int q = 7 - qq;
          const float yq = __shfl_sync(FULL, vcur, (lane & ~7) | q);
          float r = yq - part[q];
#pragma unroll
          for (int d = q + 1; d < 8; ++d) r = fmaf(-Lb[q * BMAX + s0 + d], xb[d], r);
          xb[q] = (q < nr) ? r * Lb[q * BMAX + s0 + q] : 0.f;
        }
        // lane e's slot takes row j0 + e
        float v = 0.f;
#pragma unroll
        for (int d = 0; d < 8; ++d) v = (e == d) ? xb[d] : v;
        w[hc] = v;
      }
      {
        float v = 0.f;
#pragma unroll
        for (int d = 0; d < 8; ++d) v = (e == d) ? xb[d] : v;
        if (active && !timeout && e < nr) yp[(size_t)(j0 + e) * k] = v;
      }
    }
  }
  if (timeout && lane == 0) atomicOr(err, kErrTimeout);
  // lane 0 issued every copy of this warp: drain the positions it did not see
  // complete (each buffer's phases complete in order)
  if (lane == 0)
    for (int q = n_done; q < n_issued; ++q)
      if (!mbar_drain(&bar[q % nbuf], (uint32_t)((q / nbuf) & 1))) atomicOr(err, kErrDrain);
}

template <int BMAX, bool FWD>
__global__ void __launch_bounds__(64, 1) k_local_sweep_blk(int nsub, int k, const int64_t* __restrict__ sub_ptr,
                                                        const int32_t* __restrict__ sub_dofs,
                                                        const double* __restrict__ rho,
                                                        const float* __restrict__ Lbuf, float* __restrict__ wpk,
                                                        int32_t* err, int wait_limit, int64_t rec_base,
                                                        int nbuf) {
  k_local_sweep_blk_body<BMAX, FWD, BlockIdx>(BlockIdx(), nsub, k, sub_ptr, sub_dofs, rho, Lbuf, wpk, err, wait_limit,
                                    rec_base, nbuf);
}

// ---------------------------------------------------------------------------
// Local solves for wide bands (window up to 128, e.g. 3-D subdomains): one CTA
// per (subdomain, shift) with one thread per window column (thread v owns
// column v, slot u = row mod BMAX).  Per elimination
// step the raw pivot column is published in shared memory and one CTA barrier
// later every column applies its rank-one update w_v -= c_s * (c_v / pivot),
// stores its entry of L and receives its entry of the incoming band row
// (prefetched PD steps ahead); a second barrier lets the owner of the pivot
// slot gather that row as its new column.  The backward substitution keeps
// x_{row of slot v} in thread v and needs one barrier per row.
// ---------------------------------------------------------------------------
template <int BMAX>
__global__ void __launch_bounds__(((BMAX + 31) / 32) * 32) k_local_band_team(
    int npairs, int k, const int64_t* __restrict__ sub_ptr, const int32_t* __restrict__ sub_dofs,
    const float* __restrict__ bandK, const float* __restrict__ bandM, const double* __restrict__ lam,
    const double* __restrict__ rho, float* __restrict__ Lbuf, float* __restrict__ wpk, int32_t* err,
    int64_t rec_base) {
  constexpr int PD = 4;  // prefetch distance (steps) of the incoming band entries
  constexpr int PB = 4;  // prefetch distance (rows) of the backward substitution
  constexpr int NW = (BMAX + 31) / 32;
  static_assert(BMAX % PD == 0, "the prefetch ring index must be static within a window group");
  __shared__ __align__(16) float sc[BMAX];  // raw pivot column of the current step
  __shared__ __align__(16) float sa[BMAX];  // incoming band row
  __shared__ float srw;
  __shared__ float sred[2][NW];
  const int v = threadIdx.x;
  const bool own = v < BMAX;
  const int pair = blockIdx.x;
  if (pair >= npairs) return;
  const int l = pair / k, i = pair % k;
  const int64_t off = sub_ptr[l];
  const int nl = (int)(sub_ptr[l + 1] - off);
  const int32_t* dofs = sub_dofs + off;
  const float lm = (float)lam[i];
  float* Lp = Lbuf + ((size_t)(off - rec_base) * k + (size_t)i * nl) * BMAX;
  const float* gK = bandK + (size_t)off * BMAX;
  const float* gM = bandM + (size_t)off * BMAX;
  auto aval = [&](int p, int q) -> float {  // shifted entry (p, q), q <= p
    if (p >= nl) return (p == q) ? 1.f : 0.f;
    const int d = p - q;
    if (d >= BMAX || q < 0) return 0.f;
    const size_t e = (size_t)p * BMAX + (BMAX - 1 - d);
    return gK[e] - lm * gM[e];
  };
  auto rhs = [&](int p) -> float { return (p < nl) ? (float)rho[(int64_t)dofs[p] * k + i] : 0.f; };
  // entry of row j + BMAX that column v receives at step j (slot s = j mod BMAX)
  auto incoming = [&](int j, int s) -> float {
    int t = v - s;
    t += (t <= 0) ? BMAX : 0;
    return own ? aval(j + BMAX, j + t) : 0.f;
  };
  float w[BMAX];
#pragma unroll
  for (int u = 0; u < BMAX; ++u) w[u] = own ? ((u >= v) ? aval(u, v) : aval(v, u)) : 0.f;
  float rw = own ? rhs(v) : 0.f;
  float pre[PD], rpre[PD];
#pragma unroll
  for (int d = 0; d < PD; ++d) {
    pre[d] = incoming(d, d);
    rpre[d] = rhs(d + BMAX);
  }
  bool bad = false;
  for (int j0 = 0; j0 < nl; j0 += BMAX) {
    // an opaque zero keeps per-slot comparisons from being hoisted out of the loop
    int zero;
    asm volatile("mov.u32 %0, 0;" : "=r"(zero));
    const int vz = v + zero;
#pragma unroll
    for (int s = 0; s < BMAX; ++s) {
      const int j = j0 + s;
      if (j >= nl) break;
      const int pd = s % PD;  // j0 is a multiple of BMAX, hence of PD
      if (own) sc[vz] = w[s];
      if (vz == s) srw = rw;
      __syncthreads();
      float piv = sc[s];
      if (!(piv > 0.f)) {  // the same value in every thread
        bad = true;
        piv = 1.f;
      }
      const float inv = rsqrtf(piv);
      const float yj = srw * inv;
      const float lv = w[s] * inv;  // L(row of slot v, j); sqrt(pivot) for v = s
      const float cv = lv * inv;
#pragma unroll
      for (int u4 = 0; u4 < BMAX; u4 += 4) {
        const float4 q = *reinterpret_cast<const float4*>(sc + u4);
        w[u4 + 0] = fmaf(-q.x, cv, w[u4 + 0]);
        w[u4 + 1] = fmaf(-q.y, cv, w[u4 + 1]);
        w[u4 + 2] = fmaf(-q.z, cv, w[u4 + 2]);
        w[u4 + 3] = fmaf(-q.w, cv, w[u4 + 3]);
      }
      rw = fmaf(-lv, yj, rw);
      if (own) Lp[(size_t)j * BMAX + vz] = (vz == s) ? inv : lv;
      if (vz == 0) wpk[(off + j) * k + i] = yj;
      // row j + BMAX (prefetched PD steps ago) enters slot s
      const float anew = pre[pd];
      const float rnew = rpre[pd];
      w[s] = anew;
      if (own) sa[vz] = anew;
      pre[pd] = incoming(j + PD, (s + PD) % BMAX);
      rpre[pd] = rhs(j + PD + BMAX);
      __syncthreads();
      if (vz == s) {
#pragma unroll
        for (int u4 = 0; u4 < BMAX; u4 += 4) {
          const float4 q = *reinterpret_cast<const float4*>(sa + u4);
          w[u4 + 0] = q.x;
          w[u4 + 1] = q.y;
          w[u4 + 2] = q.z;
          w[u4 + 3] = q.w;
        }
        rw = rnew;
      }
    }
  }
  if (bad) {
    if (v == 0) atomicOr(err, 1);
    return;
  }
  // backward substitution with L^T: thread v holds x of the row in slot v
  // (zero for rows not reached yet and for rows beyond nl, whose L entries are zero)
  float xv = 0.f;
  float lr[PB], yr[PB], dr[PB];
  auto load_row = [&](int j, float& lrow, float& y, float& dinv) {
    lrow = 0.f;
    y = 0.f;
    dinv = 0.f;
    if (j < 0) return;
    const float* row = Lp + (size_t)j * BMAX;
    if (own) lrow = row[v];
    y = wpk[(off + j) * k + i];
    dinv = row[j % BMAX];
  };
#pragma unroll
  for (int d = 0; d < PB; ++d) load_row(nl - 1 - d, lr[d], yr[d], dr[d]);
  int par = 0;
  for (int j1 = nl - 1; j1 >= 0; j1 -= PB) {
#pragma unroll
    for (int d = 0; d < PB; ++d) {
      const int j = j1 - d;
      if (j < 0) break;
      const int s = j % BMAX;
      const float lv = lr[d], y = yr[d], dinv = dr[d];
      load_row(j - PB, lr[d], yr[d], dr[d]);
      float part = (own && v != s) ? lv * xv : 0.f;
      part = warp_sum(part);
      if ((v & 31) == 0) sred[par][v >> 5] = part;
      __syncthreads();
      float tot = 0.f;
#pragma unroll
      for (int q = 0; q < NW; ++q) tot += sred[par][q];
      const float xj = (y - tot) * dinv;
      if (v == s) xv = xj;
      if (v == 0) wpk[(off + j) * k + i] = xj;
      par ^= 1;
    }
  }
}

// c[a, i] = sum_{g} P[g, a] rho[g, i] using P^T (CSR n_H x n); one block per coarse dof.
// Block reduction of KC per-thread column accumulators in a fixed order:
// warp butterflies, then the warps' sums added in warp order by thread i.
// Returns the total of column i in thread i (i < KC), 0 elsewhere.
template <int KC>
__device__ __forceinline__ double block_sum_columns(double (&acc)[KC], double* red /* [32][KC] */) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int i = 0; i < KC; ++i) {
    const double v = warp_sum(acc[i]);
    if (lane == 0) red[w * KC + i] = v;
  }
  __syncthreads();
  double s = 0;
  if ((int)threadIdx.x < KC)
    for (int q = 0; q < nw; ++q) s += red[q * KC + threadIdx.x];
  return s;
}

// c[a, i] = sum_r P^T[a, r] rho[r, i]: one block per coarse row a, a thread per
// entry of the row with all KC columns of rho[r, :] in registers.
template <int KC>
__global__ void __launch_bounds__(256) k_coarse_restrict(int nH, int k, const int64_t* __restrict__ rp,
                                                         const int32_t* __restrict__ ci,
                                                         const double* __restrict__ pv,
                                                         const double* __restrict__ rho, double* c) {
  __shared__ double red[8 * KC];
  const int a = blockIdx.x;
  double acc[KC];
#pragma unroll
  for (int i = 0; i < KC; ++i) acc[i] = 0.0;
  for (int64_t e = rp[a] + threadIdx.x; e < rp[a + 1]; e += blockDim.x) {
    const double p = pv[e];
    const double* row = rho + (int64_t)ci[e] * k;
#pragma unroll
    for (int i = 0; i < KC; ++i)
      if (i < k) acc[i] = fma(p, row[i], acc[i]);
  }
  const double s = block_sum_columns<KC>(acc, red);
  if ((int)threadIdx.x < k) c[(int64_t)a * k + threadIdx.x] = s;
}

// Coarse term of Eq. (3.3) in the eigenbasis Phi of (K_H, M_H):
// a[j, i] = (phi_j . c_i) / (lambda_j^H - lambda_i) for j >= k (Q_{s+1}^H), 0 for j < k.
template <int KC>
__global__ void __launch_bounds__(256) k_coarse_spectral(int nH, int k, const double* __restrict__ Phi,
                                                         const double* __restrict__ lamH,
                                                         const double* __restrict__ lam,
                                                         const double* __restrict__ c, double* a) {
  __shared__ double red[8 * KC];
  const int j = blockIdx.x;
  double acc[KC];
#pragma unroll
  for (int i = 0; i < KC; ++i) acc[i] = 0.0;
  if (j >= k)
    for (int r = threadIdx.x; r < nH; r += blockDim.x) {
      const double ph = Phi[(int64_t)r * nH + j];
      const double* row = c + (int64_t)r * k;
#pragma unroll
      for (int i = 0; i < KC; ++i)
        if (i < k) acc[i] = fma(ph, row[i], acc[i]);
    }
  const double s = block_sum_columns<KC>(acc, red);
  if ((int)threadIdx.x < k) a[(int64_t)j * k + threadIdx.x] = (j >= k) ? s / (lamH[j] - lam[threadIdx.x]) : 0.0;
}

// w0 = Phi a (n_H x k): one block per coarse row r.
template <int KC>
__global__ void __launch_bounds__(256) k_coarse_expand(int nH, int k, const double* __restrict__ Phi,
                                                       const double* __restrict__ a, double* w0) {
  __shared__ double red[8 * KC];
  const int r = blockIdx.x;
  double acc[KC];
#pragma unroll
  for (int i = 0; i < KC; ++i) acc[i] = 0.0;
  for (int j = k + threadIdx.x; j < nH; j += blockDim.x) {
    const double ph = Phi[(int64_t)r * nH + j];
    const double* row = a + (int64_t)j * k;
#pragma unroll
    for (int i = 0; i < KC; ++i)
      if (i < k) acc[i] = fma(ph, row[i], acc[i]);
  }
  const double s = block_sum_columns<KC>(acc, red);
  if ((int)threadIdx.x < k) w0[(int64_t)r * k + threadIdx.x] = s;
}

// z[g, i] = sum_{c} P[g, c] w0[c, i] + sum_{local copies of g} w[pos, i]
template <typename TP>
__global__ void k_prolong_add(int64_t n, int k, const int64_t* __restrict__ prp, const int32_t* __restrict__ pci,
                              const double* __restrict__ pv, const double* __restrict__ w0,
                              const int32_t* __restrict__ rtp, const int32_t* __restrict__ rtpos,
                              const TP* __restrict__ wpk, double* __restrict__ Z) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n * k) return;
  int64_t g = t / k;
  int i = (int)(t % k);
  double z = 0;
  for (int64_t e = prp[g]; e < prp[g + 1]; ++e) z = fma(pv[e], w0[(int64_t)pci[e] * k + i], z);
  for (int e = rtp[g]; e < rtp[g + 1]; ++e) z += (double)wpk[(int64_t)rtpos[e] * k + i];
  Z[t] = z;
}

// The prolongation-add in FP32 for the FP32 preconditioner: one thread per fine
// row with its KC columns in registers, P values as the hi parts of their split,
// w0 truncated to FP32 by integer operations, the FP32 local solutions added in
// the inverse map's order (the order of k_prolong_add); Z stays FP64.
template <int KC>
__global__ void __launch_bounds__(256) k_prolong_add_f32(int64_t n, int k, const int64_t* __restrict__ prp,
                                                         const int32_t* __restrict__ pci,
                                                         const float2* __restrict__ pvs,
                                                         const double* __restrict__ w0,
                                                         const int32_t* __restrict__ rtp,
                                                         const int32_t* __restrict__ rtpos,
                                                         const float* __restrict__ wpk, double* __restrict__ Z) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= n) return;
  float z[KC];
#pragma unroll
  for (int i = 0; i < KC; ++i) z[i] = 0.f;
  for (int64_t e = prp[g]; e < prp[g + 1]; ++e) {
    const float p = pvs[e].x;
    const double* row = w0 + (int64_t)pci[e] * k;
#pragma unroll
    for (int i = 0; i < KC; ++i)
      if (i < k) z[i] = fmaf(p, f64_hi(row[i]), z[i]);
  }
  for (int e = rtp[g]; e < rtp[g + 1]; ++e) {
    const float* row = wpk + (int64_t)rtpos[e] * k;
#pragma unroll
    for (int i = 0; i < KC; ++i)
      if (i < k) z[i] += row[i];
  }
  double* out = Z + g * k;
#pragma unroll
  for (int i = 0; i < KC; ++i)
    if (i < k) out[i] = f32_to_f64_bits(z[i]);
}

// ---------------------------------------------------------------------------
// Device-side setup: input validation, band structure of the local matrices.
// ---------------------------------------------------------------------------
// flag |= 1 if the CSR is malformed (row pointers not monotone or not spanning
// [0, nnz], a column out of range, columns not strictly increasing in a row)
__global__ void k_validate_csr(int n_rows, int n_cols, int64_t nnz, const int64_t* __restrict__ rp,
                               const int32_t* __restrict__ ci, int32_t* flag) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r == 0 && (rp[0] != 0 || rp[n_rows] != nnz)) atomicOr(flag, 1);
  if (r >= n_rows) return;
  const int64_t a = rp[r], b = rp[r + 1];
  if (b < a || a < 0 || b > nnz) {
    atomicOr(flag, 1);
    return;
  }
  for (int64_t e = a; e < b; ++e) {
    const int32_t c = ci[e];
    if (c < 0 || c >= n_cols || (e > a && c <= ci[e - 1])) {
      atomicOr(flag, 1);
      return;
    }
  }
}

// flag |= 2 if two CSR patterns differ (same n and nnz assumed)
__global__ void k_same_pattern(int n, int64_t nnz, const int64_t* __restrict__ rpA, const int32_t* __restrict__ ciA,
                               const int64_t* __restrict__ rpM, const int32_t* __restrict__ ciM, int32_t* flag) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t <= n && rpA[t] != rpM[t]) atomicOr(flag, 2);
  if (t < nnz && ciA[t] != ciM[t]) atomicOr(flag, 2);
}

__device__ __forceinline__ int sub_of(int nsub, const int64_t* __restrict__ sub_ptr, int64_t idx) {
  int lo = 0, hi = nsub;  // sub_ptr[lo] <= idx < sub_ptr[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (sub_ptr[mid] <= idx)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

// local index of global dof c in the ascending list d[0..nl), -1 if absent
__device__ __forceinline__ int local_index(const int32_t* __restrict__ d, int nl, int32_t c) {
  int lo = 0, hi = nl;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (d[mid] < c)
      lo = mid + 1;
    else
      hi = mid;
  }
  return (lo < nl && d[lo] == c) ? lo : -1;
}

// flag |= 4 if a subdomain dof list is out of range or not strictly ascending
__global__ void k_validate_part(int nsub, int n, int64_t total, const int64_t* __restrict__ sub_ptr,
                                const int32_t* __restrict__ dofs, int32_t* flag) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= total) return;
  const int l = sub_of(nsub, sub_ptr, t);
  const int32_t g = dofs[t];
  if (g < 0 || g >= n || (t > sub_ptr[l] && g <= dofs[t - 1])) atomicOr(flag, 4);
}

// maximum lower bandwidth max(p - q) over the local matrices (q, p local indices
// of a stored entry (dofs[p], dofs[q]), q <= p)
__global__ void k_band_width(int nsub, int64_t total, const int64_t* __restrict__ sub_ptr,
                             const int32_t* __restrict__ dofs, const int64_t* __restrict__ rp,
                             const int32_t* __restrict__ ci, int32_t* bw) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= total) return;
  const int l = sub_of(nsub, sub_ptr, t);
  const int64_t off = sub_ptr[l];
  const int nl = (int)(sub_ptr[l + 1] - off);
  const int p = (int)(t - off);
  const int32_t g = dofs[t];
  int m = 0;
  for (int64_t e = rp[g]; e < rp[g + 1]; ++e) {
    const int32_t c = ci[e];
    if (c > g) break;
    const int q = local_index(dofs + off, nl, c);
    if (q >= 0) m = max(m, p - q);
  }
  if (m > 0) atomicMax(bw, m);
}

// ---------------------------------------------------------------------------
// Setup kernels
// ---------------------------------------------------------------------------
// Band rows of the local matrices (principal submatrices of a CSR matrix on the
// ascending subdomain dof lists), one thread per local row p of a subdomain:
// the row of width W holds A_l(p, p - B + 1 .. p) in its last B positions
// (the diagonal last), zero where A_l has no entry and in the W - B leading
// pad positions; values rounded to T.  val2 / out2 (optional): a second
// matrix with the same pattern, filled alongside.
template <typename T>
__global__ void k_band_fill(int nsub, int64_t total, const int64_t* __restrict__ sub_ptr,
                            const int32_t* __restrict__ dofs, const int64_t* __restrict__ rp,
                            const int32_t* __restrict__ ci, const double* __restrict__ val,
                            const double* __restrict__ val2, int B, int W, T* __restrict__ out,
                            T* __restrict__ out2) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= total) return;
  const int l = sub_of(nsub, sub_ptr, t);
  const int64_t off = sub_ptr[l];
  const int nl = (int)(sub_ptr[l + 1] - off);
  const int p = (int)(t - off);
  const int32_t g = dofs[t];
  T* o = out + t * W;
  T* o2 = out2 ? out2 + t * W : nullptr;
  for (int e = 0; e < W; ++e) o[e] = T(0);
  if (o2)
    for (int e = 0; e < W; ++e) o2[e] = T(0);
  for (int64_t e = rp[g]; e < rp[g + 1]; ++e) {
    const int32_t c = ci[e];
    if (c > g) break;
    const int q = local_index(dofs + off, nl, c);
    if (q >= 0 && p - q < B) {
      const int slot = (W - B) + (q - p + B - 1);
      o[slot] = (T)val[e];
      if (o2) o2[slot] = (T)val2[e];
    }
  }
}

// Galerkin products K_H = P^T K P and M_H = P^T M P in two deterministic passes.
// Pass 1 (thread per fine row r): the sparse rows (K P)[r, :] and (M P)[r, :],
// at most `width` coarse columns each (32 first; wider on overflow, e.g. for the
// 16-entry rows of the BFS interpolation), accumulated in a fixed order.
__global__ void k_kp_rows(int n, int width, const int64_t* __restrict__ arp, const int32_t* __restrict__ aci,
                          const double* __restrict__ av, const int64_t* __restrict__ mrp,
                          const int32_t* __restrict__ mci, const double* __restrict__ mv,
                          const int64_t* __restrict__ prp, const int32_t* __restrict__ pci,
                          const double* __restrict__ pv, int32_t* kpc, double* kpk, double* kpm, int32_t* cnt,
                          int32_t* overflow) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  int32_t* cols = kpc + (int64_t)r * width;
  double* vk = kpk + (int64_t)r * width;
  double* vm = kpm + (int64_t)r * width;
  int m = 0;
  bool full = false;
  auto add = [&](int32_t b, double x, bool isk) {
    int s = 0;
    while (s < m && cols[s] != b) ++s;
    if (s == m) {
      if (m == width) {
        full = true;
        return;
      }
      cols[m] = b;
      vk[m] = 0.0;
      vm[m] = 0.0;
      ++m;
    }
    if (isk)
      vk[s] += x;
    else
      vm[s] += x;
  };
  for (int64_t f = arp[r]; f < arp[r + 1]; ++f) {
    const int64_t c = aci[f];
    for (int64_t g = prp[c]; g < prp[c + 1]; ++g) add(pci[g], av[f] * pv[g], true);
  }
  for (int64_t f = mrp[r]; f < mrp[r + 1]; ++f) {
    const int64_t c = mci[f];
    for (int64_t g = prp[c]; g < prp[c + 1]; ++g) add(pci[g], mv[f] * pv[g], false);
  }
  if (full) *overflow = 1;
  cnt[r] = m;
}

// Pass 2 (one block per coarse row a): K_H[a, b] = sum_{r in P^T row a}
// P[r, a] (K P)[r, b].  Warp w takes a contiguous part of the P^T row and
// accumulates into its own dense row in shared memory, lane s adding entry s
// of (K P)[r, :] (distinct columns b, so no two lanes meet); the rows of P^T
// are visited in ascending order and the warps' rows are added in warp order,
// so every entry is summed in a fixed order.  The loads of the next
// kGalerkinUnroll rows are issued before their updates.
constexpr int kGalerkinUnroll = 8;
__global__ void k_galerkin_rows(int nH, int width, const int64_t* __restrict__ ptr, const int32_t* __restrict__ ptc,
                                const double* __restrict__ ptv, const int32_t* __restrict__ kpc,
                                const double* __restrict__ kpk, const double* __restrict__ kpm,
                                const int32_t* __restrict__ cnt, double* KH, double* MH) {
  extern __shared__ double rowbuf[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int a = blockIdx.x;
  double* kr = rowbuf + (size_t)wib * 2 * nH;
  double* mr = kr + nH;
  for (int t = lane; t < nH; t += 32) {
    kr[t] = 0.0;
    mr[t] = 0.0;
  }
  __syncwarp();
  const int64_t e0 = ptr[a], e1 = ptr[a + 1];
  const int64_t len = (e1 - e0 + nw - 1) / nw;
  const int64_t eb = e0 + wib * len, ee = min(e1, eb + len);
  constexpr int GU = kGalerkinUnroll;
  for (int64_t e = eb; e < ee; e += GU) {
    int32_t rr[GU], m[GU], b[GU];
    double p[GU], xk[GU], xm[GU];
#pragma unroll
    for (int u = 0; u < GU; ++u) {
      const bool ok = e + u < ee;
      rr[u] = ok ? ptc[e + u] : 0;
      p[u] = ok ? ptv[e + u] : 0.0;
      m[u] = ok ? cnt[rr[u]] : 0;
    }
    // entries hb + lane of each (K P) row, 32 at a time (one pass for rows of <= 32)
    for (int hb = 0; hb < width; hb += 32) {
#pragma unroll
      for (int u = 0; u < GU; ++u) {
        const bool ok = hb + lane < m[u];
        const int64_t o = (int64_t)rr[u] * width + hb + lane;
        b[u] = ok ? kpc[o] : 0;
        xk[u] = ok ? kpk[o] : 0.0;
        xm[u] = ok ? kpm[o] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < GU; ++u)
        if (hb + lane < m[u]) {
          kr[b[u]] += p[u] * xk[u];
          mr[b[u]] += p[u] * xm[u];
        }
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nH; t += blockDim.x) {
    double sk = 0.0, sm = 0.0;
    for (int q = 0; q < nw; ++q) {
      sk += rowbuf[(size_t)q * 2 * nH + t];
      sm += rowbuf[(size_t)q * 2 * nH + nH + t];
    }
    KH[(int64_t)a * nH + t] = sk;
    MH[(int64_t)a * nH + t] = sm;
  }
}


int col_block(int k) { return k * (256 / k); }

}  // namespace

// ===========================================================================
// instrumentation
// ===========================================================================
ProfScope::ProfScope(Handle& hh, int c) : h(hh), cls(c), idx(0), on(hh.profile) {
  if (!on) return;
  idx = h.ev_used;
  while (h.ev_pool.size() < idx + 2) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    h.ev_pool.push_back((void*)e);
  }
  h.ev_used += 2;
  h.ev_cls.push_back(cls);
  cudaEventRecord((cudaEvent_t)h.ev_pool[idx], h.stream);
}
ProfScope::~ProfScope() {
  if (on) cudaEventRecord((cudaEvent_t)h.ev_pool[idx + 1], h.stream);
}
void prof_flush(Handle& h) {
  if (h.ev_used == 0) return;
  cudaStreamSynchronize(h.stream);
  for (size_t p = 0; p < h.ev_cls.size(); ++p) {
    float ms = 0;
    cudaEventElapsedTime(&ms, (cudaEvent_t)h.ev_pool[2 * p], (cudaEvent_t)h.ev_pool[2 * p + 1]);
    h.prof_ms[h.ev_cls[p]] += ms;
    h.prof_count[h.ev_cls[p]] += 1;
  }
  h.ev_used = 0;
  h.ev_cls.clear();
}

// ===========================================================================
// launchers
// ===========================================================================
int launch_spmm(Handle& h, const double* X, double* YA, double* YM, int ncols, const float2* Xs) {
  ProfScope ps(h, BPJD_PROF_SPMM);
  const int n = h.n;
  auto go = [&](auto lanes_tag, const CsrDev& A, const double* vm, double* ya, double* ym) {
    constexpr int LANES = decltype(lanes_tag)::value;
    constexpr int RPW = 32 / LANES;
    int64_t warps = (n + RPW - 1) / RPW;
    int64_t blocks = (warps * 32 + 255) / 256;
    k_spmm<LANES><<<(unsigned)blocks, 256, 0, h.stream>>>(n, A.row_ptr, A.col, A.val, vm, X, ya, ym, ncols);
    h.launches += 1;
  };
  if (h.dword() && h.Asplit) {
    // lanes per row and columns per lane: every lane of a row group busy for k = 4, 8, 12, 16, 24, 32
    auto god = [&](auto lanes_tag, auto cpl_tag, const float2* va, const float2* vm, double* ya, double* ym,
                   const CsrDev& A) {
      constexpr int LANES = decltype(lanes_tag)::value;
      constexpr int CPL = decltype(cpl_tag)::value;
      constexpr int RPW = 32 / LANES;
      int64_t warps = (n + RPW - 1) / RPW;
      int64_t blocks = (warps * 32 + 255) / 256;
      if (Xs)
        k_spmm_dw<LANES, CPL, true><<<(unsigned)blocks, 256, 0, h.stream>>>(n, A.row_ptr, A.col, va, vm, X, Xs, ya,
                                                                           ym, ncols);
      else
        k_spmm_dw<LANES, CPL, false><<<(unsigned)blocks, 256, 0, h.stream>>>(n, A.row_ptr, A.col, va, vm, X, Xs, ya,
                                                                            ym, ncols);
      h.launches += 1;
    };
    using I = std::integral_constant<int, 1>;
    using I2 = std::integral_constant<int, 2>;
    using I3 = std::integral_constant<int, 3>;
    using I4 = std::integral_constant<int, 4>;
    using I8 = std::integral_constant<int, 8>;
    auto dispatch_dw = [&](const CsrDev& A, const float2* va, const float2* vm, double* ya, double* ym) {
      if (ncols <= 4)
        god(I4(), I(), va, vm, ya, ym, A);
      else if (ncols <= 8)
        god(I4(), I2(), va, vm, ya, ym, A);
      else if (ncols <= 12)
        god(I4(), I3(), va, vm, ya, ym, A);
      else if (ncols <= 16)
        god(I4(), I4(), va, vm, ya, ym, A);
      else if (ncols <= 24)
        god(I8(), I3(), va, vm, ya, ym, A);
      else
        god(I8(), I4(), va, vm, ya, ym, A);
    };
    if (h.same_pattern) {
      dispatch_dw(h.A, h.Asplit, h.Msplit, YA, YM);
    } else {
      dispatch_dw(h.A, h.Asplit, nullptr, YA, nullptr);
      dispatch_dw(h.M, h.Msplit, nullptr, YM, nullptr);
    }
    return (int)cudaGetLastError();
  }
  auto dispatch = [&](const CsrDev& A, const double* vm, double* ya, double* ym) {
    if (ncols <= 4)
      go(std::integral_constant<int, 4>(), A, vm, ya, ym);
    else if (ncols <= 8)
      go(std::integral_constant<int, 8>(), A, vm, ya, ym);
    else if (ncols <= 16)
      go(std::integral_constant<int, 16>(), A, vm, ya, ym);
    else
      go(std::integral_constant<int, 32>(), A, vm, ya, ym);
  };
  if (h.same_pattern) {
    dispatch(h.A, h.M.val, YA, YM);
  } else {
    dispatch(h.A, nullptr, YA, nullptr);
    dispatch(h.M, nullptr, YM, nullptr);
  }
  return (int)cudaGetLastError();
}

int launch_csr_times_dense(const CsrDev& P, const double* D, int ldd, int ncols, double* Y, int ldy,
                           cudaStream_t s) {
  int64_t tot = (int64_t)P.n_rows * ncols;
  k_csr_dense<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(P.n_rows, P.row_ptr, P.col, P.val, D, ldd, ncols, Y,
                                                            ldy);
  return (int)cudaGetLastError();
}

int launch_residual(Handle& h, const double* AX, const double* MX, const double* lam, double* rho) {
  const int k = h.k;
  ProfScope ps(h, BPJD_PROF_RESID);
  const int bs = col_block(k);
  const int64_t nk = (int64_t)h.n * k;
  int nblk = (int)std::min<int64_t>(kPartialBlocks, (nk + bs - 1) / bs);
  h.launches += 2;
  k_residual<<<nblk, bs, 2 * bs * sizeof(double), h.stream>>>(nk, k, AX, MX, lam, rho, h.partial);
  k_residual_finish<<<1, 256, 0, h.stream>>>(nblk, k, h.partial, lam, h.stop_rule, h.tol, h.dstat);
  return (int)cudaGetLastError();
}

int launch_rayleigh(Handle& h, const double* X, const double* AX, const double* MX, double* lam) {
  const int k = h.k;
  const int bs = col_block(k);
  const int64_t nk = (int64_t)h.n * k;
  int nblk = (int)std::min<int64_t>(kPartialBlocks, (nk + bs - 1) / bs);
  h.launches += 2;
  k_rq_partial<<<nblk, bs, 2 * bs * sizeof(double), h.stream>>>(nk, k, X, AX, MX, h.partial);
  k_rq_finish<<<1, 256, 0, h.stream>>>(nblk, k, h.partial, lam);
  return (int)cudaGetLastError();
}

int launch_inner(Handle& h, int p, const double* const* U, int q, const double* const* V, double* out) {
  const int k = h.k;
  Ptrs6 u{}, v{};
  for (int b = 0; b < p; ++b) u.p[b] = U[b];
  for (int b = 0; b < q; ++b) v.p[b] = V[b];
  const int nout = p * k * q * k;
  if (nout > kInnerMaxOut * 256) return (int)cudaErrorInvalidValue;
  ProfScope ps(h, BPJD_PROF_INNER);
  h.launches += 2;
  int nblk = (int)std::min<int64_t>(kPartialBlocks, ((int64_t)h.n + 63) / 64);
  int rpb = (int)(((int64_t)h.n + nblk - 1) / nblk);
  size_t sm = (size_t)kInnerRows * (p + q) * k * sizeof(double);
  k_inner<<<nblk, 256, sm, h.stream>>>(h.n, k, p, u, q, v, rpb, h.partial);
  k_sum_partials<<<(nout + 255) / 256, 256, 0, h.stream>>>(nblk, nout, h.partial, out);
  return (int)cudaGetLastError();
}

size_t gram_partial_doubles(int64_t n, int k, int nu, int nvb, int sym) {
  const int mu = nu * k, mv = nvb * k;
  const int TU = (mu + 3) / 4, TV = (mv + 3) / 4;
  const int ntiles = sym ? TU * (TU + 1) / 2 : TU * TV;
  const int nblk = (int)std::min<int64_t>(kGramBlocks, (n + kGramRows - 1) / kGramRows);
  const int rpb = (int)(((n + nblk - 1) / nblk + kGramRows - 1) / kGramRows * kGramRows);
  const int nblk2 = (int)((n + rpb - 1) / rpb);
  return (size_t)nblk2 * ntiles * 16;
}

int launch_gram_raw(int64_t n, int k, int nu, const double* const* U, int nvb, int nv, const double* const* V1,
                    const double* const* V2, int sym, double* out1, double* out2, double* partial,
                    size_t partial_capacity, cudaStream_t stream) {
  const int mu = nu * k, mv = nvb * k;
  const int TU = (mu + 3) / 4, TV = (mv + 3) / 4;
  const int ntiles = sym ? TU * (TU + 1) / 2 : TU * TV;
  if (ntiles > 256 || nv < 1 || nv > 2 || nu > 6 || nvb > 6 || n < 1) return (int)cudaErrorInvalidValue;
  Ptrs6 u{}, v1{}, v2{};
  for (int b = 0; b < nu; ++b) u.p[b] = U[b];
  for (int b = 0; b < nvb; ++b) {
    v1.p[b] = V1[b];
    if (nv > 1) v2.p[b] = V2[b];
  }
  const int nblk = (int)std::min<int64_t>(kGramBlocks, (n + kGramRows - 1) / kGramRows);
  const int rpb = (int)(((n + nblk - 1) / nblk + kGramRows - 1) / kGramRows * kGramRows);
  const int nblk2 = (int)((n + rpb - 1) / rpb);
  const int total = nv * ntiles * 16;
  if ((size_t)nblk2 * total > partial_capacity) return (int)cudaErrorInvalidValue;
  // chunk rows: a divisor of kGramRows keeping the staging (two raw FP64 buffers
  // and the hi/lo planes, 24 bytes per value) within 100 KB (few blocks: long
  // chunks, fewer barriers per row)
  const int nseg = nu + nv * nvb;
  int R = kGramRows;
  while (R > 1 && (size_t)24 * R * k * nseg > 100 * 1024) R /= 2;
  const size_t stage = (size_t)24 * R * k * nseg;
  const size_t red = (size_t)ntiles * nv * 16 * sizeof(double);
  const size_t sm = std::max(stage, red);
  auto go = [&](auto nv_tag, auto vec_tag) {
    constexpr int NV = decltype(nv_tag)::value;
    constexpr bool VEC = decltype(vec_tag)::value;
    allow_dynamic_smem((const void*)k_gram_dw<NV, VEC>);
    k_gram_dw<NV, VEC><<<nblk2, 256, sm, stream>>>((int)n, k, nu, u, nvb, v1, v2, sym, rpb, R, partial);
  };
  const bool vec = (k % 4) == 0;
  if (nv == 2) {
    if (vec)
      go(std::integral_constant<int, 2>(), std::true_type());
    else
      go(std::integral_constant<int, 2>(), std::false_type());
  } else {
    if (vec)
      go(std::integral_constant<int, 1>(), std::true_type());
    else
      go(std::integral_constant<int, 1>(), std::false_type());
  }
  k_gram_reduce<<<(total + 31) / 32, 256, 0, stream>>>(nblk2, nv, mu, mv, sym, partial, out1, out2);
  return (int)cudaGetLastError();
}

int launch_gram(Handle& h, int nu, const double* const* U, int nvb, int nv, const double* const* V1,
                const double* const* V2, int sym, double* out1, double* out2) {
  ProfScope ps(h, BPJD_PROF_INNER);
  h.launches += 2;
  return launch_gram_raw(h.n, h.k, nu, U, nvb, nv, V1, V2, sym, out1, out2, h.partial, h.partial_cap, h.stream);
}

int launch_combine_rows(Handle& h, int nin, const double* const* Win, const double* C, int ldc, int csub,
                        const double* Zadd, double* out, double sign, int consistency_only, float2* split_out) {
  ProfScope ps(h, BPJD_PROF_COMBINE);
  h.launches += 1;
  if (nin < 1 || nin > 6 || nin * h.k > 96 || csub < 1 || csub > 256) return (int)cudaErrorInvalidValue;
  Ptrs6 w{};
  for (int b = 0; b < nin; ++b) w.p[b] = Win[b];
  if (h.dword() && consistency_only) {
    const int m = nin * h.k;
    const size_t sm = (size_t)(m * csub + kCombRows * m) * sizeof(float);
    allow_dynamic_smem((const void*)k_combine_f32);
    const int64_t blocks = ((int64_t)h.n + kCombRows - 1) / kCombRows;
    k_combine_f32<<<(unsigned)blocks, 256, sm, h.stream>>>(h.n, h.k, nin, w, C, ldc, csub, Zadd, out, (float)sign,
                                                           split_out);
    return (int)cudaGetLastError();
  }
  if (h.dword()) {
    const int m = nin * h.k;
    const size_t sm = (size_t)(2 * m * csub + 2 * kCombRows * m) * sizeof(float);
    allow_dynamic_smem((const void*)k_combine_dw);
    const int64_t blocks = ((int64_t)h.n + kCombRows - 1) / kCombRows;
    k_combine_dw<<<(unsigned)blocks, 256, sm, h.stream>>>(h.n, h.k, nin, w, C, ldc, csub, Zadd, out, sign,
                                                          split_out);
    return (int)cudaGetLastError();
  }
  int64_t tot = (int64_t)h.n * csub;
  size_t sm = (size_t)nin * h.k * csub * sizeof(double);
  k_combine_rows<<<(unsigned)((tot + 255) / 256), 256, sm, h.stream>>>(h.n, h.k, nin, w, C, ldc, csub, Zadd, out,
                                                                        sign);
  return (int)cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Grouped local solves: the (subdomain, shift) work of several solver handles
// of one window tier in one grid.  Segment j owns the blocks [blk0_j,
// blk0_{j+1}); a block runs the same kernel body as a launch of its handle
// alone would, on that handle's arrays, so every pair is computed exactly as
// it is alone.  (The wide tiers' factorisations keep one launch per handle.)
// ---------------------------------------------------------------------------
constexpr int kMaxSegs = 16;
struct LocalSeg {
  const int64_t* sub_ptr;
  const int32_t* sub_dofs;
  const float* bandK;
  const float* bandM;
  const double* lam;
  const double* rho;
  float* Lbuf;
  float* wpk;
  int32_t* err;
  int nsub, k, wait_limit, blk0;
};
struct LocalSegs {
  int n;
  LocalSeg s[kMaxSegs];
};
__device__ __forceinline__ int seg_of(const LocalSegs& g, int b) {
  int j = 0;
  while (j + 1 < g.n && b >= g.s[j + 1].blk0) ++j;
  return j;
}

template <int BMAX>
__global__ void __launch_bounds__(128, (BMAX <= 40) ? 3 : 2)
    k_local_factor_mma_grp(const __grid_constant__ LocalSegs g) {
  const LocalSeg& q = g.s[seg_of(g, blockIdx.x)];
  k_local_factor_mma_body<BMAX, SegBlockIdx>(SegBlockIdx{q.blk0}, q.nsub, q.k, q.sub_ptr, q.sub_dofs, q.bandK,
                                             q.bandM, q.lam,
                                q.rho, q.Lbuf, q.wpk, q.err, q.wait_limit, 0);
}
template <int BMAX, bool FWD>
__global__ void __launch_bounds__(64, 1) k_local_sweep_blk_grp(const __grid_constant__ LocalSegs g, int nbuf) {
  const LocalSeg& q = g.s[seg_of(g, blockIdx.x)];
  k_local_sweep_blk_body<BMAX, FWD, SegBlockIdx>(SegBlockIdx{q.blk0}, q.nsub, q.k, q.sub_ptr, q.sub_dofs, q.rho,
                                                 q.Lbuf, q.wpk,
                                    q.err, q.wait_limit, 0, nbuf);
}
template <int BMAX>
__global__ void __launch_bounds__(64, 1) k_local_forward_grp(const __grid_constant__ LocalSegs g) {
  const LocalSeg& q = g.s[seg_of(g, blockIdx.x)];
  k_local_forward_body<BMAX, SegBlockIdx>(SegBlockIdx{q.blk0}, q.nsub, q.k, q.sub_ptr, q.sub_dofs, q.rho, q.Lbuf,
                                          q.wpk, q.err,
                             q.wait_limit, 0);
}
template <int BMAX>
__global__ void __launch_bounds__(64, 1) k_local_backward_grp(const __grid_constant__ LocalSegs g) {
  const LocalSeg& q = g.s[seg_of(g, blockIdx.x)];
  k_local_backward_body<BMAX, SegBlockIdx>(SegBlockIdx{q.blk0}, q.nsub, q.k, q.sub_ptr, q.Lbuf, q.wpk, q.err,
                                           q.wait_limit, 0);
}

// Device facts for launch shapes, read once per device: SM count, shared memory
// per SM and the share the driver reserves per block.
struct SmFacts {
  int sms = 0, smem_sm = 0, smem_reserved = 0, smem_block = 0;
};
SmFacts sm_facts() {
  static std::mutex mu;
  static std::map<int, SmFacts> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  auto it = cache.find(dev);
  if (it != cache.end()) return it->second;
  SmFacts f;
  cudaDeviceGetAttribute(&f.sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&f.smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&f.smem_reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  cudaDeviceGetAttribute(&f.smem_block, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (f.sms < 1) f.sms = 1;
  cache[dev] = f;
  return f;
}

// Ring depth of the blocked sweeps for a launch of `blocks` blocks: the deepest
// ring (more copies in flight per warp) whose shared memory still lets every
// block of the launch be resident at once (one wave), between 2 and NBUF_MAX.
template <int BM>
int sweep_ring_buffers(int64_t blocks) {
  using S = BlkShape<BM>;
  const SmFacts f = sm_facts();
  const int64_t per_sm = std::max<int64_t>(1, (blocks + f.sms - 1) / f.sms);
  const int64_t room = (int64_t)f.smem_sm / per_sm - f.smem_reserved - 1024;  // static part: the barriers
  const int64_t per_buf = (int64_t)S::WPB * 4 * S::PS * sizeof(float);
  int64_t nb = room / per_buf;
  nb = std::min<int64_t>(nb, ((int64_t)f.smem_block - 1024) / per_buf);
  return (int)std::max<int64_t>(2, std::min<int64_t>(S::NBUF_MAX, nb));
}

bool can_reuse_factors(const Handle& h) {
  if (!h.local_f32() || h.chunk_l0.size() != 2) return false;
  switch (h.Bpad) {
    case 16: case 24: case 32: case 40: case 48: case 64: case 96: case 152: return true;
    default: return false;
  }
}

// The local part of Eq. (3.3): mode kLocalFull factorises every (subdomain, shift)
// pair and solves (chunk by chunk); kLocalReuse runs the forward and backward
// sweeps on stored factors; the three single-kernel modes serve the captured
// iteration, where the factorisation and the forward sweep sit in the two
// branches of a device-decided conditional node ahead of the shared backward sweep.
int launch_local(Handle& h, const double* rho, const double* lam, int mode) {
  const int k = h.k;
  const int B = h.B;
  if (mode != kLocalFull && mode != kLocalFactorOnly) {
    if (!can_reuse_factors(h)) return (int)cudaErrorInvalidValue;
    // sweeps with the stored factors (all resident: one chunk)
    ProfScope ps(h, BPJD_PROF_LOCAL);
    const int nsub = h.nsub;
    const int bwd_blocks = (nsub * ((k + 3) / 4) + 1) / 2;
    const bool fwd = mode != kLocalBackwardOnly, bwd = mode != kLocalForwardOnly;
    h.launches += (fwd ? 1 : 0) + (bwd ? 1 : 0);
    auto sweeps = [&](auto bm) {
      constexpr int BM = decltype(bm)::value;
      if constexpr (BM <= 48) {
        // blocked sweeps, eight rows per step
        const int nbuf = sweep_ring_buffers<BM>(bwd_blocks);
        const size_t ssm = sizeof(float) * BlkShape<BM>::smem_floats(nbuf);
        if (fwd) {
          allow_dynamic_smem((const void*)k_local_sweep_blk<BM, true>);
          k_local_sweep_blk<BM, true><<<bwd_blocks, 32 * BlkShape<BM>::WPB, ssm, h.stream>>>(
              nsub, k, h.sub_ptr, h.sub_dofs, rho, (const float*)h.Lbuf, (float*)h.wpk, h.derr, h.wait_limit, 0,
              nbuf);
        }
        if (bwd) {
          allow_dynamic_smem((const void*)k_local_sweep_blk<BM, false>);
          k_local_sweep_blk<BM, false><<<bwd_blocks, 32 * BlkShape<BM>::WPB, ssm, h.stream>>>(
              nsub, k, h.sub_ptr, h.sub_dofs, rho, (const float*)h.Lbuf, (float*)h.wpk, h.derr, h.wait_limit, 0,
              nbuf);
        }
        return;
      }
      const size_t bsm = sizeof(float) * BwdShape<BM>::smem_floats;
      if (fwd) {
        allow_dynamic_smem((const void*)k_local_forward<BM>);
        k_local_forward<BM><<<bwd_blocks, 32 * BwdShape<BM>::WPB, bsm, h.stream>>>(
            nsub, k, h.sub_ptr, h.sub_dofs, rho, (const float*)h.Lbuf, (float*)h.wpk, h.derr, h.wait_limit, 0);
      }
      if (bwd) {
        allow_dynamic_smem((const void*)k_local_backward<BM>);
        k_local_backward<BM><<<bwd_blocks, 32 * BwdShape<BM>::WPB, bsm, h.stream>>>(
            nsub, k, h.sub_ptr, (const float*)h.Lbuf, (float*)h.wpk, h.derr, h.wait_limit, 0);
      }
    };
    switch (h.Bpad) {
      case 16: sweeps(std::integral_constant<int, 16>()); break;
      case 24: sweeps(std::integral_constant<int, 24>()); break;
      case 32: sweeps(std::integral_constant<int, 32>()); break;
      case 40: sweeps(std::integral_constant<int, 40>()); break;
      case 48: sweeps(std::integral_constant<int, 48>()); break;
      case 64: sweeps(std::integral_constant<int, 64>()); break;
      case 96: sweeps(std::integral_constant<int, 96>()); break;
      case 152: sweeps(std::integral_constant<int, 152>()); break;
      default: return (int)cudaErrorInvalidValue;
    }
    if (mode == kLocalReuse) ++h.reuses;
    return (int)cudaGetLastError();
  }
  if (mode == kLocalFactorOnly && !can_reuse_factors(h)) return (int)cudaErrorInvalidValue;
  if (mode == kLocalFull) ++h.refactorisations;
  // local band solves, chunk by chunk of subdomains (the factor records of one
  // chunk fit the record scratch)
  {
    ProfScope ps(h, BPJD_PROF_LOCAL);
    const bool f32 = h.local_f32();
    const int nchunks = (int)h.chunk_l0.size() - 1;
    for (int ch = 0; ch < nchunks; ++ch) {
      const int l0 = h.chunk_l0[ch];
      const int nsub = h.chunk_l0[ch + 1] - l0;
      const int64_t* sptr = h.sub_ptr + l0;
      const int64_t rec_base = h.chunk_off[ch];
      const int npairs_c = nsub * k;
      // factorisation (+ backward substitution)
      h.launches += (f32 && h.Bpad > 0 && h.Bpad != 128 && mode == kLocalFull) ? 2 : 1;
      if (f32 && h.Bpad > 0) {
        const int blocks = nsub * ((k + kLocalWarps - 1) / kLocalWarps);
        const int bwd_blocks = (nsub * ((k + 3) / 4) + 1) / 2;
#define BPJD_LOCAL_TILE(BM)                                                                                    \
  case BM: {                                                                                                   \
    const size_t sm = sizeof(float) * MmaShape<BM>::smem_floats;                                               \
    allow_dynamic_smem((const void*)k_local_factor_mma<BM>);                                                   \
    k_local_factor_mma<BM><<<blocks, 32 * kLocalWarps, sm, h.stream>>>(nsub, k, sptr, h.sub_dofs, h.bandKf,     \
                                                                       h.bandMf, lam, rho, (float*)h.Lbuf,     \
                                                                       (float*)h.wpk, h.derr, h.wait_limit,    \
                                                                       rec_base);                              \
    if (mode == kLocalFull) {                                                                                  \
      const int nbuf = sweep_ring_buffers<BM>(bwd_blocks);                                                     \
      const size_t ssm = sizeof(float) * BlkShape<BM>::smem_floats(nbuf);                                      \
      allow_dynamic_smem((const void*)k_local_sweep_blk<BM, false>);                                           \
      k_local_sweep_blk<BM, false><<<bwd_blocks, 32 * BlkShape<BM>::WPB, ssm, h.stream>>>(                     \
          nsub, k, sptr, h.sub_dofs, rho, (const float*)h.Lbuf, (float*)h.wpk, h.derr, h.wait_limit, rec_base,  \
          nbuf);                                                                                               \
    }                                                                                                          \
    break;                                                                                                     \
  }
#define BPJD_LOCAL_WIDE(BM)                                                                                    \
  case BM: {                                                                                                   \
    k_local_factor_wide<BM><<<npairs_c, 32 * WideShape<BM>::NW, 0, h.stream>>>(                               \
        npairs_c, k, sptr, h.sub_dofs, h.bandKf, h.bandMf, lam, rho, (float*)h.Lbuf, (float*)h.wpk, h.derr,     \
        rec_base);                                                                                             \
    if (mode == kLocalFull) {                                                                                  \
      const size_t bsm = sizeof(float) * BwdShape<BM>::smem_floats;                                            \
      allow_dynamic_smem((const void*)k_local_backward<BM>);                                                   \
      k_local_backward<BM><<<bwd_blocks, 32 * BwdShape<BM>::WPB, bsm, h.stream>>>(                             \
          nsub, k, sptr, (const float*)h.Lbuf, (float*)h.wpk, h.derr, h.wait_limit, rec_base);                 \
    }                                                                                                          \
    break;                                                                                                     \
  }
        switch (h.Bpad) {
          BPJD_LOCAL_TILE(16)
          BPJD_LOCAL_TILE(24)
          BPJD_LOCAL_TILE(32)
          BPJD_LOCAL_TILE(40)
          BPJD_LOCAL_TILE(48)
          BPJD_LOCAL_WIDE(64)
          BPJD_LOCAL_WIDE(96)
          BPJD_LOCAL_WIDE(152)
          case 128:
            k_local_band_team<128><<<npairs_c, 128, 0, h.stream>>>(npairs_c, k, sptr, h.sub_dofs, h.bandKf,
                                                                   h.bandMf, lam, rho, (float*)h.Lbuf,
                                                                   (float*)h.wpk, h.derr, rec_base);
            break;
          default:
            return (int)cudaErrorInvalidValue;
        }
#undef BPJD_LOCAL_TILE
#undef BPJD_LOCAL_WIDE
      } else {
        const size_t esz = f32 ? sizeof(float) : sizeof(double);
        const size_t per_warp = (size_t)(B * B + 3 * B) * esz;
        int wpb = (int)std::max<size_t>(1, std::min<size_t>(4, (200 * 1024) / per_warp));
        size_t sm = per_warp * wpb;
        int blocks = (npairs_c + wpb - 1) / wpb;
        if (f32) {
          allow_dynamic_smem((const void*)k_local_band<float>);
          k_local_band<float><<<blocks, 32 * wpb, sm, h.stream>>>(npairs_c, k, sptr, h.sub_dofs, B, h.bandKf,
                                                                  h.bandMf, lam, rho, (float*)h.Lbuf,
                                                                  (float*)h.wpk, h.derr, rec_base);
        } else {
          allow_dynamic_smem((const void*)k_local_band<double>);
          k_local_band<double><<<blocks, 32 * wpb, sm, h.stream>>>(npairs_c, k, sptr, h.sub_dofs, B, h.bandK,
                                                                   h.bandM, lam, rho, (double*)h.Lbuf,
                                                                   (double*)h.wpk, h.derr, rec_base);
        }
      }
    }
  }
  return (int)cudaGetLastError();
}

int prime_kernel_attributes(Handle& h) {
  auto tier = [&](auto bm) {
    constexpr int BM = decltype(bm)::value;
    if constexpr (BM <= 48) {
      allow_dynamic_smem((const void*)k_local_sweep_blk<BM, true>);
      allow_dynamic_smem((const void*)k_local_sweep_blk<BM, false>);
    } else {
      allow_dynamic_smem((const void*)k_local_forward<BM>);
      allow_dynamic_smem((const void*)k_local_backward<BM>);
    }
  };
  switch (h.local_f32() ? h.Bpad : 0) {
    case 16: tier(std::integral_constant<int, 16>()); allow_dynamic_smem((const void*)k_local_factor_mma<16>); break;
    case 24: tier(std::integral_constant<int, 24>()); allow_dynamic_smem((const void*)k_local_factor_mma<24>); break;
    case 32: tier(std::integral_constant<int, 32>()); allow_dynamic_smem((const void*)k_local_factor_mma<32>); break;
    case 40: tier(std::integral_constant<int, 40>()); allow_dynamic_smem((const void*)k_local_factor_mma<40>); break;
    case 48: tier(std::integral_constant<int, 48>()); allow_dynamic_smem((const void*)k_local_factor_mma<48>); break;
    case 64: tier(std::integral_constant<int, 64>()); break;
    case 96: tier(std::integral_constant<int, 96>()); break;
    case 152: tier(std::integral_constant<int, 152>()); break;
    default: break;
  }
  allow_dynamic_smem((const void*)k_local_band<float>);
  allow_dynamic_smem((const void*)k_local_band<double>);
  return (int)cudaGetLastError();
}

int launch_precond(Handle& h, const double* rho, const double* lam, double* Z, int reuse) {
  const bool stored = reuse && can_reuse_factors(h);
  int e;
  if (h.batch && batch_eligible(h)) {
    // served handle: the local solves go into a launch shared with other requests
    e = batch_local(h.batch, h, rho, lam, !stored);
    if (e == 0) {
      h.launches += 2;
      if (stored)
        ++h.reuses;
      else
        ++h.refactorisations;
    }
  } else {
    e = launch_local(h, rho, lam, stored ? kLocalReuse : kLocalFull);
  }
  if (e) return e;
  return launch_coarse_prolong(h, rho, lam, Z);
}

int launch_local_grouped(Handle* const* hs, const double* const* rho, const double* const* lam,
                         const int* refactor, int n, cudaStream_t s) {
  if (n < 1 || n > kGroupedMax || n > kMaxSegs) return (int)cudaErrorInvalidValue;
  const int BM = hs[0]->Bpad;
  for (int j = 0; j < n; ++j)
    if (!can_reuse_factors(*hs[j]) || hs[j]->Bpad != BM) return (int)cudaErrorInvalidValue;
  auto run = [&](auto bm) -> int {
    constexpr int B = decltype(bm)::value;
    // segments: factorisations, forward sweeps on stored factors, backward sweeps
    LocalSegs gf{}, gr{}, gb{};
    int bf = 0, br = 0, bb = 0;
    for (int j = 0; j < n; ++j) {
      Handle& h = *hs[j];
      LocalSeg q{h.sub_ptr, h.sub_dofs, h.bandKf, h.bandMf, lam[j], rho[j], (float*)h.Lbuf, (float*)h.wpk,
                 h.derr, h.nsub, h.k, h.wait_limit, 0};
      const int sweep_blocks = (h.nsub * ((h.k + 3) / 4) + 1) / 2;
      if (refactor[j]) {
        q.blk0 = bf;
        gf.s[gf.n++] = q;
        bf += (B <= 48) ? h.nsub * ((h.k + kLocalWarps - 1) / kLocalWarps) : h.nsub * h.k;
      } else {
        q.blk0 = br;
        gr.s[gr.n++] = q;
        br += sweep_blocks;
      }
      q.blk0 = bb;
      gb.s[gb.n++] = q;
      bb += sweep_blocks;
    }
    if constexpr (B <= 48) {
      if (gf.n) {
        allow_dynamic_smem((const void*)k_local_factor_mma_grp<B>);
        k_local_factor_mma_grp<B><<<bf, 32 * kLocalWarps, sizeof(float) * MmaShape<B>::smem_floats, s>>>(gf);
      }
      if (gr.n) {
        const int nbuf = sweep_ring_buffers<B>(br);
        allow_dynamic_smem((const void*)k_local_sweep_blk_grp<B, true>);
        k_local_sweep_blk_grp<B, true><<<br, 32 * BlkShape<B>::WPB, sizeof(float) * BlkShape<B>::smem_floats(nbuf),
                                         s>>>(gr, nbuf);
      }
      const int nbuf = sweep_ring_buffers<B>(bb);
      allow_dynamic_smem((const void*)k_local_sweep_blk_grp<B, false>);
      k_local_sweep_blk_grp<B, false><<<bb, 32 * BlkShape<B>::WPB, sizeof(float) * BlkShape<B>::smem_floats(nbuf),
                                        s>>>(gb, nbuf);
    } else {
      const size_t bsm = sizeof(float) * BwdShape<B>::smem_floats;
      // wide tiers: each request's factorisation in a launch of its own (its register
      // allocation is tuned for one subdomain-shift pair per CTA), on the shared stream
      for (int j = 0; j < gf.n; ++j) {
        const LocalSeg& q = gf.s[j];
        k_local_factor_wide<B><<<q.nsub * q.k, 32 * WideShape<B>::NW, 0, s>>>(
            q.nsub * q.k, q.k, q.sub_ptr, q.sub_dofs, q.bandK, q.bandM, q.lam, q.rho, q.Lbuf, q.wpk, q.err, 0);
      }
      if (gr.n) {
        allow_dynamic_smem((const void*)k_local_forward_grp<B>);
        k_local_forward_grp<B><<<br, 32 * BwdShape<B>::WPB, bsm, s>>>(gr);
      }
      allow_dynamic_smem((const void*)k_local_backward_grp<B>);
      k_local_backward_grp<B><<<bb, 32 * BwdShape<B>::WPB, bsm, s>>>(gb);
    }
    return (int)cudaGetLastError();
  };
  switch (BM) {
    case 16: return run(std::integral_constant<int, 16>());
    case 24: return run(std::integral_constant<int, 24>());
    case 32: return run(std::integral_constant<int, 32>());
    case 40: return run(std::integral_constant<int, 40>());
    case 48: return run(std::integral_constant<int, 48>());
    case 64: return run(std::integral_constant<int, 64>());
    case 96: return run(std::integral_constant<int, 96>());
    case 152: return run(std::integral_constant<int, 152>());
    default: return (int)cudaErrorInvalidValue;
  }
}

int launch_coarse_prolong(Handle& h, const double* rho, const double* lam, double* Z) {
  const int k = h.k;
  // coarse solve
  {
    ProfScope ps(h, BPJD_PROF_COARSE);
    h.launches += 3;
    auto coarse = [&](auto kc) {
      constexpr int KC = decltype(kc)::value;
      k_coarse_restrict<KC><<<h.nH, 256, 0, h.stream>>>(h.nH, k, h.PT.row_ptr, h.PT.col, h.PT.val, rho, h.cH);
      k_coarse_spectral<KC><<<h.nH, 256, 0, h.stream>>>(h.nH, k, h.Phi, h.lamH, lam, h.cH, h.aH);
      k_coarse_expand<KC><<<h.nH, 256, 0, h.stream>>>(h.nH, k, h.Phi, h.aH, h.w0);
    };
    if (k <= 8)
      coarse(std::integral_constant<int, 8>());
    else if (k <= 16)
      coarse(std::integral_constant<int, 16>());
    else
      coarse(std::integral_constant<int, 32>());
  }
  // prolongation-add
  {
    ProfScope ps(h, BPJD_PROF_PROLONG);
    h.launches += 1;
    int64_t tot = (int64_t)h.n * k;
    const unsigned rblocks = (unsigned)(((int64_t)h.n + 255) / 256);
    if (h.local_f32() && h.Psplit) {
      if (k <= 8)
        k_prolong_add_f32<8><<<rblocks, 256, 0, h.stream>>>(h.n, k, h.P.row_ptr, h.P.col, h.Psplit, h.w0, h.rt_ptr,
                                                           h.rt_pos, (const float*)h.wpk, Z);
      else if (k <= 16)
        k_prolong_add_f32<16><<<rblocks, 256, 0, h.stream>>>(h.n, k, h.P.row_ptr, h.P.col, h.Psplit, h.w0,
                                                            h.rt_ptr, h.rt_pos, (const float*)h.wpk, Z);
      else
        k_prolong_add_f32<32><<<rblocks, 256, 0, h.stream>>>(h.n, k, h.P.row_ptr, h.P.col, h.Psplit, h.w0,
                                                            h.rt_ptr, h.rt_pos, (const float*)h.wpk, Z);
    } else if (h.local_f32())
      k_prolong_add<float><<<(unsigned)((tot + 255) / 256), 256, 0, h.stream>>>(
          h.n, k, h.P.row_ptr, h.P.col, h.P.val, h.w0, h.rt_ptr, h.rt_pos, (const float*)h.wpk, Z);
    else
      k_prolong_add<double><<<(unsigned)((tot + 255) / 256), 256, 0, h.stream>>>(
          h.n, k, h.P.row_ptr, h.P.col, h.P.val, h.w0, h.rt_ptr, h.rt_pos, (const double*)h.wpk, Z);
  }
  return (int)cudaGetLastError();
}


int launch_split_values(const double* v, int64_t nnz, float2* out, cudaStream_t s) {
  if (nnz <= 0) return 0;
  k_split_values<<<(unsigned)((nnz + 255) / 256), 256, 0, s>>>(nnz, v, out);
  return (int)cudaGetLastError();
}

int launch_band_fill(Handle& h, const CsrDev& c, const double* val2, double* out, double* out2, float* outf,
                     float* outf2) {
  const unsigned blocks = (unsigned)((h.sum_nl + 127) / 128);
  if (outf) {
    const int W = std::max(h.B, h.Bpad);
    k_band_fill<float><<<blocks, 128, 0, h.stream>>>(h.nsub, h.sum_nl, h.sub_ptr, h.sub_dofs, c.row_ptr, c.col, c.val,
                                                     val2, h.B, W, outf, outf2);
  } else {
    k_band_fill<double><<<blocks, 128, 0, h.stream>>>(h.nsub, h.sum_nl, h.sub_ptr, h.sub_dofs, c.row_ptr, c.col,
                                                      c.val, val2, h.B, h.B, out, out2);
  }
  return (int)cudaGetLastError();
}

int launch_validate_csr(const CsrDev& c, int32_t* flag, cudaStream_t s) {
  k_validate_csr<<<(c.n_rows + 256) / 256, 256, 0, s>>>(c.n_rows, c.n_cols, c.nnz, c.row_ptr, c.col, flag);
  return (int)cudaGetLastError();
}

int launch_same_pattern(const CsrDev& a, const CsrDev& m, int32_t* flag, cudaStream_t s) {
  const int64_t tot = std::max<int64_t>(a.nnz, (int64_t)a.n_rows + 1);
  k_same_pattern<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(a.n_rows, a.nnz, a.row_ptr, a.col, m.row_ptr, m.col,
                                                               flag);
  return (int)cudaGetLastError();
}

int launch_validate_part(Handle& h, int32_t* flag) {
  if (h.sum_nl <= 0) return 0;
  k_validate_part<<<(unsigned)((h.sum_nl + 255) / 256), 256, 0, h.stream>>>(h.nsub, h.n, h.sum_nl, h.sub_ptr,
                                                                           h.sub_dofs, flag);
  return (int)cudaGetLastError();
}

int launch_band_width(Handle& h, const CsrDev& c, int32_t* bw) {
  k_band_width<<<(unsigned)((h.sum_nl + 255) / 256), 256, 0, h.stream>>>(h.nsub, h.sum_nl, h.sub_ptr, h.sub_dofs,
                                                                         c.row_ptr, c.col, bw);
  return (int)cudaGetLastError();
}


int launch_galerkin(const CsrDev& A, const CsrDev& Msp, const CsrDev& P, const CsrDev& PT, double* KH,
                    double* MH, cudaStream_t s) {
  const int n = A.n_rows, nH = P.n_cols;
  const int wpb = (int)std::max<size_t>(1, std::min<size_t>(8, (200 * 1024) / (2 * (size_t)nH * sizeof(double))));
  const size_t sm = (size_t)wpb * 2 * nH * sizeof(double);
  int rc = (int)cudaErrorInvalidValue;
  for (int width = 32; width <= 128 && rc == (int)cudaErrorInvalidValue; width *= 2) {
    int32_t *kpc = nullptr, *cnt = nullptr, *ovf = nullptr;
    double *kpk = nullptr, *kpm = nullptr;
    int hov = 0;
    cudaError_t e = cudaSuccess;
    rc = 0;
    if ((e = cudaMalloc(&kpc, sizeof(int32_t) * (size_t)n * width)) != cudaSuccess) goto done;
    if ((e = cudaMalloc(&kpk, sizeof(double) * (size_t)n * width)) != cudaSuccess) goto done;
    if ((e = cudaMalloc(&kpm, sizeof(double) * (size_t)n * width)) != cudaSuccess) goto done;
    if ((e = cudaMalloc(&cnt, sizeof(int32_t) * (size_t)n)) != cudaSuccess) goto done;
    if ((e = cudaMalloc(&ovf, sizeof(int32_t))) != cudaSuccess) goto done;
    if ((e = cudaMemsetAsync(ovf, 0, sizeof(int32_t), s)) != cudaSuccess) goto done;
    k_kp_rows<<<(n + 127) / 128, 128, 0, s>>>(n, width, A.row_ptr, A.col, A.val, Msp.row_ptr, Msp.col, Msp.val,
                                              P.row_ptr, P.col, P.val, kpc, kpk, kpm, cnt, ovf);
    if ((e = cudaMemcpyAsync(&hov, ovf, sizeof(int32_t), cudaMemcpyDeviceToHost, s)) != cudaSuccess) goto done;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) goto done;
    if (hov) {
      rc = (int)cudaErrorInvalidValue;  // a row of K P holds more coarse columns: retry wider
      goto done;
    }
    allow_dynamic_smem((const void*)k_galerkin_rows);
    k_galerkin_rows<<<nH, 32 * wpb, sm, s>>>(nH, width, PT.row_ptr, PT.col, PT.val, kpc, kpk, kpm, cnt, KH, MH);
    if ((e = cudaGetLastError()) != cudaSuccess) goto done;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) goto done;
  done:
    cudaFree(kpc);
    cudaFree(kpk);
    cudaFree(kpm);
    cudaFree(cnt);
    cudaFree(ovf);
    if (e != cudaSuccess) return (int)e;
  }
  return rc;
}

}  // namespace bpjd
