// Setup-time device kernels that no iteration uses: the transpose of the
// coarse interpolation (Section 3: the coarse restriction applies P^T).

#include <algorithm>
#include <cstdint>

#include "bpjd_internal.h"

namespace bpjd {

namespace {

// ---------------------------------------------------------------------------
// Transpose of a validated CSR matrix on the device, deterministic: row j of the
// result lists the entries of column j in ascending original row (what a host
// counting sort gives).  The rows are taken in nch chunks of `chunk` rows:
// pass 1 counts every chunk's entries per column, pass 2 turns the counts into
// output offsets per (chunk, column) and the result's row pointers, pass 3 has
// one warp per chunk walk its rows in order, the chunk's running offsets in
// shared memory; the entries of one row lie in distinct columns and are placed
// in parallel.
// ---------------------------------------------------------------------------
__global__ void k_tr_count(int64_t nrows, int64_t chunk, int ncols, const int64_t* __restrict__ rp,
                           const int32_t* __restrict__ ci, unsigned long long* __restrict__ cnt) {
  const int64_t r0 = (int64_t)blockIdx.x * chunk, r1 = min(nrows, r0 + chunk);
  if (r0 >= r1) return;
  unsigned long long* out = cnt + (int64_t)blockIdx.x * ncols;
  for (int64_t e = rp[r0] + threadIdx.x; e < rp[r1]; e += blockDim.x) atomicAdd(&out[ci[e]], 1ull);
}

__global__ void __launch_bounds__(1024) k_tr_offsets(int nch, int ncols, unsigned long long* __restrict__ cnt,
                                                     int64_t* __restrict__ rpT) {
  __shared__ long long part[1024];
  const int per = (ncols + (int)blockDim.x - 1) / (int)blockDim.x;
  const int j0 = min(ncols, (int)threadIdx.x * per), j1 = min(ncols, j0 + per);
  long long mine = 0;
  for (int j = j0; j < j1; ++j)
    for (int c = 0; c < nch; ++c) mine += (long long)cnt[(int64_t)c * ncols + j];
  part[threadIdx.x] = mine;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long run = 0;
    for (int t = 0; t < (int)blockDim.x; ++t) {
      const long long v = part[t];
      part[t] = run;
      run += v;
    }
    rpT[ncols] = run;
  }
  __syncthreads();
  long long run = part[threadIdx.x];
  for (int j = j0; j < j1; ++j) {
    rpT[j] = run;
    for (int c = 0; c < nch; ++c) {
      const long long v = (long long)cnt[(int64_t)c * ncols + j];
      cnt[(int64_t)c * ncols + j] = (unsigned long long)run;
      run += v;
    }
  }
}

__global__ void __launch_bounds__(32) k_tr_fill(int64_t nrows, int64_t chunk, int ncols,
                                                const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                                const double* __restrict__ val,
                                                const unsigned long long* __restrict__ off, int32_t* __restrict__ ciT,
                                                double* __restrict__ valT) {
  extern __shared__ long long so[];  // this chunk's running offsets, one per column
  const int lane = threadIdx.x;
  const int64_t r0 = (int64_t)blockIdx.x * chunk, r1 = min(nrows, r0 + chunk);
  for (int j = lane; j < ncols; j += 32) so[j] = (long long)off[(int64_t)blockIdx.x * ncols + j];
  __syncwarp();
  for (int64_t r = r0; r < r1; ++r) {
    for (int64_t e = rp[r] + lane; e < rp[r + 1]; e += 32) {
      const int32_t j = ci[e];
      const long long pos = so[j]++;
      ciT[pos] = (int32_t)r;
      valT[pos] = val[e];
    }
    __syncwarp();
  }
}

}  // namespace

int launch_csr_transpose(const CsrDev& a, int64_t* rpT, int32_t* ciT, double* valT, cudaStream_t s) {
  const int ncols = a.n_cols;
  const int64_t nrows = a.n_rows;
  if (ncols > kTransposeMaxCols) return (int)cudaErrorInvalidValue;
  const int64_t chunk = std::max<int64_t>(1024, (nrows + 511) / 512);
  const int nch = (int)std::max<int64_t>(1, (nrows + chunk - 1) / chunk);
  unsigned long long* cnt = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&cnt, sizeof(unsigned long long) * (size_t)nch * ncols, s);
  if (e != cudaSuccess) return (int)e;
  cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * (size_t)nch * ncols, s);
  k_tr_count<<<nch, 256, 0, s>>>(nrows, chunk, ncols, a.row_ptr, a.col, cnt);
  k_tr_offsets<<<1, 1024, 0, s>>>(nch, ncols, cnt, rpT);
  const size_t sm = sizeof(long long) * (size_t)ncols;
  allow_dynamic_smem((const void*)k_tr_fill);
  k_tr_fill<<<nch, 32, sm, s>>>(nrows, chunk, ncols, a.row_ptr, a.col, a.val, cnt, ciT, valT);
  e = cudaGetLastError();
  cudaFreeAsync(cnt, s);
  return (int)e;
}

}  // namespace bpjd
