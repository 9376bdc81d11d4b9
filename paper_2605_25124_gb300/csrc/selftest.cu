// Diagnostics: the bounded wait that every pipelined kernel uses (an mbarrier
// phase that should be completed by a bulk copy), run on a barrier nothing
// arrives on.  The wait must give up after its limit, record ERR_TIMEOUT in
// the workspace and return, leaving the context usable.  The loop also stops
// after a fixed number of polls, so it ends even if the clock did not advance.
#include "common.cuh"
#include "pipe.cuh"

namespace gini {

__global__ void k_selftest_wait(unsigned* err, uint64_t limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_init_fence();
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  const uint64_t t0 = globaltimer_ns();
  bool done = false;
  for (uint64_t it = 0; it < (uint64_t)1 << 26; ++it) {
    if (mbar_try_wait(&bar, 0)) { done = true; break; }
    if (globaltimer_ns() - t0 > limit_ns) break;
  }
  if (!done) raise_error(err, ERR_TIMEOUT);
}

}  // namespace gini

using namespace gini;

extern "C" void gini_set_cuda_error(cudaError_t e);

extern "C" int gini_selftest_wait_timeout(uint64_t limit_ns, void* ws, size_t ws_bytes,
                                          void* stream) {
  if (!ws || ws_misaligned(ws) || ws_bytes < WS_HEADER) return GINI_EINVAL;
  if (limit_ns < 1000 || limit_ns > 1000000000ull) return GINI_EINVAL;
  gini_count_launch(1);
  k_selftest_wait<<<1, 32, 0, (cudaStream_t)stream>>>(reinterpret_cast<unsigned*>(ws), limit_ns);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { gini_set_cuda_error(e); return GINI_ECUDA; }
  return GINI_OK;
}
