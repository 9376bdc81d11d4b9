// Diagnostics.
//  - The bounded wait that every pipelined kernel uses (an mbarrier phase that
//    should be completed by a bulk copy), run on a barrier nothing arrives on.
//    The wait must give up after its limit, record ERR_TIMEOUT in the
//    workspace and return, leaving the context usable.  The loop also stops
//    after a fixed number of polls, so it ends even if the clock did not
//    advance.
//  - (debug builds) The index check, on a store whose index lies past the
//    bound it is checked against but inside the buffer it writes, so that the
//    store stays in bounds even if the check were broken.
#define GINI_FILE_ID 6  // site numbers of the debug index checks
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

// buf holds 64 floats; the checked bound is 32 and thread t stores at 8 + 4 t
// (8 .. 132 would leave the buffer, so only threads 0 .. 13 run: 8 .. 60).
// Threads 0 .. 5 pass the check (8 .. 28), threads 6 .. 13 fail it (32 .. 60).
__global__ void k_selftest_index(unsigned* err, float* buf) {
  const int t = threadIdx.x;
  if (t >= 14) return;
  const int idx = 8 + 4 * t;
  if (GINI_IDX_OK(err, idx, 32)) buf[idx] = (float)idx;
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

extern "C" int gini_debug_checks(void) {
#ifdef GINI_DEBUG_CHECKS
  return 1;
#else
  return 0;
#endif
}

extern "C" int gini_selftest_index_check(void* ws, size_t ws_bytes, void* stream) {
#ifdef GINI_DEBUG_CHECKS
  if (!ws || ws_misaligned(ws) || ws_bytes < WS_HEADER + 256) return GINI_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  float* buf = reinterpret_cast<float*>(reinterpret_cast<char*>(ws) + WS_HEADER);
  cudaError_t e = cudaMemsetAsync(buf, 0, 64 * sizeof(float), s);
  if (e == cudaSuccess) {
    gini_count_launch(1);
    k_selftest_index<<<1, 32, 0, s>>>(reinterpret_cast<unsigned*>(ws), buf);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) { gini_set_cuda_error(e); return GINI_ECUDA; }
  return GINI_OK;
#else
  (void)ws; (void)ws_bytes; (void)stream;
  return GINI_EINVAL;  // release build: there is no check to exercise
#endif
}

extern "C" int gini_debug_index_record(void* ws, uint32_t* site, int64_t* index, int64_t* bound,
                                       uint32_t* count) {
  if (!ws || ws_misaligned(ws)) return GINI_EINVAL;
  DebugRecord r{};
  char* rec = reinterpret_cast<char*>(ws) + DEBUG_RECORD_OFF;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&r, rec, sizeof(r), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(rec, 0, sizeof(r));
  if (e != cudaSuccess) { gini_set_cuda_error(e); return GINI_ECUDA; }
  if (site) *site = r.site;
  if (index) *index = r.index;
  if (bound) *bound = r.bound;
  if (count) *count = r.count;
  return GINI_OK;
}
