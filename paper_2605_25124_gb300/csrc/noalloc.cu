// gini_stress_grad_noalloc: the stress/gradient entry point for callers that
// cannot allocate device memory.  Its scratch space is a fixed array compiled
// into the library instead of a caller workspace.
#include <mutex>

#include "common.cuh"

namespace gini {

// Largest scratch the variant offers: gini_workspace_size(GINI_OP_STRESS, n, 0,
// k, 0) must not exceed it (about 520,000 points at k = 2, 160,000 at k = 3).
constexpr size_t NOALLOC_SCRATCH_BYTES = (size_t)8 << 20;

// One copy per device that loads the library, held until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
static void* g_scratch_addr[MAX_DEVICES];
static std::mutex g_scratch_mu;

// Device address of the array on the current device.  In host code the symbol
// itself is only a host-side handle, so it must never be passed to a kernel.
static cudaError_t scratch_on_current_device(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

// Turns an error recorded by the kernels into a NaN stress.
__global__ void k_noalloc_error_to_nan(const unsigned* err, double* stress) {
  if (*err) *stress = __longlong_as_double(0x7ff8000000000000ll);
}

}  // namespace gini

using namespace gini;

extern "C" void gini_set_cuda_error(cudaError_t e);

extern "C" int gini_stress_grad_noalloc(const float* Y_dev, int64_t n, int k, double nu,
                                        const void* delta_dev, int layout, int dtype,
                                        int64_t ldd, const float* col_scale_dev,
                                        double sum_delta2, double* stress_dev, float* grad_dev,
                                        void* stream) {
  if (n < 2 || k < 2 || k > 8 || n > ((int64_t)1 << 31)) return GINI_EINVAL;
  if (gini_workspace_size(GINI_OP_STRESS, n, 0, k, 0) > NOALLOC_SCRATCH_BYTES) return GINI_ENOMEM;
  if (!Y_dev || !stress_dev || !delta_dev) return GINI_EINVAL;
  void* scratch = nullptr;
  cudaError_t e = scratch_on_current_device(&scratch);
  if (e != cudaSuccess) { gini_set_cuda_error(e); return GINI_ECUDA; }
  cudaStream_t s = (cudaStream_t)stream;
  // The array keeps the previous call's contents: clear the error word (the
  // accumulators are cleared by the stress path itself).
  e = cudaMemsetAsync(scratch, 0, WS_HEADER, s);
  if (e != cudaSuccess) { gini_set_cuda_error(e); return GINI_ECUDA; }
  const int st = gini_stress_grad(Y_dev, n, k, nu, delta_dev, layout, dtype, ldd, col_scale_dev,
                                  sum_delta2, stress_dev, grad_dev, scratch,
                                  NOALLOC_SCRATCH_BYTES, stream);
  if (st != GINI_OK) return st;
  gini_count_launch(1);
  k_noalloc_error_to_nan<<<1, 1, 0, s>>>(reinterpret_cast<const unsigned*>(scratch), stress_dev);
  e = cudaGetLastError();
  if (e != cudaSuccess) { gini_set_cuda_error(e); return GINI_ECUDA; }
  return GINI_OK;
}
