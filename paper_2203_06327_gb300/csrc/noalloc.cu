// Allocation-free variant of the double-word block inner product.
//
// bpjd_block_gram needs per-block partial sums in device scratch, which the
// handle allocates in bpjd_setup.  bpjd_block_gram_noalloc computes the same
// product without a handle and without allocating: its partial sums live in
// the file-scope device array below, reserved when the library is loaded on a
// device and held until the process exits.

#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "bpjd_internal.h"

namespace {

// 1 Mi doubles = 8 MiB of partial sums per device.
constexpr size_t kNoAllocScratchDoubles = (size_t)1024 * 1024;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

std::mutex g_scratch_mu;
double* g_scratch_ptr[64] = {};

// Device address of the scratch array on the current device.  In host code the
// symbol g_noalloc_scratch is only a host-side stand-in, so its device address
// is looked up once per device (with that device current) and cached.
int scratch_on_current_device(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return BPJD_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return BPJD_ERR_CUDA;
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return BPJD_OK;
}

}  // namespace

extern "C" int bpjd_block_gram_noalloc(int64_t n, int32_t k, int32_t nu, const double* const* U, int32_t nv,
                                       const double* const* V, int32_t symmetric, double* out, void* stream) {
  if (n < 1 || k < 1 || !U || !V || !out || nu < 1 || nv < 1 || nu > 6 || nv > 6) return BPJD_ERR_BAD_ARG;
  // the kernels index rows with 32-bit integers: larger blocks are refused before any launch
  if (n > (int64_t)INT32_MAX) return BPJD_ERR_TOO_LARGE;
  if (nu * k > 64 || nv * k > 64 || (symmetric && nu != nv)) return BPJD_ERR_BAD_ARG;
  for (int b = 0; b < nu; ++b)
    if (!U[b]) return BPJD_ERR_BAD_ARG;
  for (int b = 0; b < nv; ++b)
    if (!V[b]) return BPJD_ERR_BAD_ARG;
  if (bpjd::gram_partial_doubles(n, k, nu, nv, symmetric ? 1 : 0) > kNoAllocScratchDoubles)
    return BPJD_ERR_TOO_LARGE;
  double* scratch = nullptr;
  const int rc = scratch_on_current_device(&scratch);
  if (rc != BPJD_OK) return rc;
  // every partial sum the reduction reads is written earlier in the same call,
  // so the array needs no clearing between calls
  if (bpjd::launch_gram_raw(n, k, nu, U, nv, 1, V, nullptr, symmetric ? 1 : 0, out, nullptr, scratch,
                            kNoAllocScratchDoubles, static_cast<cudaStream_t>(stream)) != 0)
    return BPJD_ERR_CUDA;
  return BPJD_OK;
}
