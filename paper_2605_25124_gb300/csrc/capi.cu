// Host-side C ABI helpers of libginimds and the FULL -> TILED pack kernels.
#include <math.h>
#include <string.h>

#include <atomic>

#define GINI_FILE_ID 5  // site numbers of the debug index checks
#include "common.cuh"

using namespace gini;

static thread_local char g_cuda_err[256] = "";
static std::atomic<uint64_t> g_launches{0};

extern "C" void gini_count_launch(unsigned n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

extern "C" uint64_t gini_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

extern "C" size_t gini_iter_ws_bytes(int64_t n, int k, int nacc, int det);

extern "C" void gini_set_cuda_error(cudaError_t e) {
  strncpy(g_cuda_err, cudaGetErrorString(e), sizeof(g_cuda_err) - 1);
  g_cuda_err[sizeof(g_cuda_err) - 1] = 0;
}

extern "C" const char* gini_last_cuda_error(void) { return g_cuda_err; }

extern "C" const char* gini_status_str(int status) {
  switch (status) {
    case GINI_OK: return "GINI_OK";
    case GINI_EINVAL: return "GINI_EINVAL: invalid argument";
    case GINI_ENONFINITE: return "GINI_ENONFINITE: NaN or Inf in the input";
    case GINI_EDEGENERATE: return "GINI_EDEGENERATE: sum of squared dissimilarities is zero";
    case GINI_ENOMEM: return "GINI_ENOMEM: workspace too small";
    case GINI_ECUDA: return "GINI_ECUDA: CUDA runtime error";
    case GINI_ETIMEOUT: return "GINI_ETIMEOUT: bounded device wait expired";
    case GINI_EINDEX: return "GINI_EINDEX: a device-side index check failed (debug build)";
    default: return "unknown gini status";
  }
}

extern "C" int gini_version(void) { return 2; }

// Deterministic mode of the calling host thread (see gini_set_deterministic).
static thread_local int g_deterministic = 0;

extern "C" void gini_set_deterministic(int on) { g_deterministic = on ? 1 : 0; }

extern "C" int gini_get_deterministic(void) { return g_deterministic; }

extern "C" int gini_tile_size(void) { return TILE; }

extern "C" int64_t gini_tiled_elems(int64_t n) {
  const int64_t T = tiles_1d(n);
  return T * (T + 1) / 2 * (int64_t)TILE * TILE;
}

extern "C" size_t gini_workspace_size(int op, int64_t n, int64_t m, int k, int iters) {
  switch (op) {
    case GINI_OP_RANK: return WS_HEADER;
    case GINI_OP_DIST: {
      const int64_t mm = m < 1 ? 1 : m;
      return WS_HEADER + 256 + (((size_t)8 * (size_t)(2 * mm - 1) * sizeof(float) + 255) & ~(size_t)255);
    }
    case GINI_OP_DIST_FP8: {
      // plus FP32 scratch for strips of columns of up to 8 matrices: all
      // columns if that fits in 128 MiB, else as many whole tile columns as
      // fit, at least one (a larger workspace gives wider strips)
      const size_t rows = n < 2 ? 2 : (size_t)n;
      const size_t per_col = sizeof(float) * rows * 8;
      const size_t all = per_col * (size_t)(tiles_1d((int64_t)rows) * TILE);
      size_t strip = all < ((size_t)128 << 20) ? all : ((size_t)128 << 20);
      if (strip < per_col * TILE) strip = per_col * TILE;
      return gini_workspace_size(GINI_OP_DIST, n, m, k, iters) + strip;
    }
    case GINI_OP_STRESS: return gini_iter_ws_bytes(n, k < 2 ? 2 : k, 1, 0);
    case GINI_OP_FIT: return gini_iter_ws_bytes(n, k < 2 ? 2 : k, (iters < 0 ? 0 : iters) + 1, 0);
    case GINI_OP_STRESS_DET: return gini_iter_ws_bytes(n, k < 2 ? 2 : k, 1, 1);
    case GINI_OP_FIT_DET:
      return gini_iter_ws_bytes(n, k < 2 ? 2 : k, (iters < 0 ? 0 : iters) + 1, 1);
    default: return 0;
  }
}

extern "C" int gini_check(void* ws, void* stream) {
  if (!ws) return GINI_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaStreamSynchronize(s);
  unsigned word = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&word, ws, sizeof(word), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && word) e = cudaMemset(ws, 0, sizeof(word));
  if (e != cudaSuccess) { gini_set_cuda_error(e); return GINI_ECUDA; }
  if (word & ERR_INDEX) return GINI_EINDEX;  // debug builds only
  if (word & ERR_TIMEOUT) return GINI_ETIMEOUT;
  if (word & ERR_DEGENERATE) return GINI_EDEGENERATE;
  if (word & ERR_NONFINITE) return GINI_ENONFINITE;
  return GINI_OK;
}

extern "C" double gini_default_step(int64_t n, int k, double nu, double sum_delta2, double eta0) {
  if (n < 2 || k < 2 || !(nu > 1.0)) return 0.0;
  const double wmax = pow((double)(k - 1) / (double)k, nu - 1.0);
  const double g = 0.5 * (double)k * wmax;
  return eta0 * sum_delta2 / (2.0 * (double)(n - 1) * (double)k * g * g);
}

// ----------------------------------------------------------------- pack ----

// Column maxima of |delta_ij| over i < j (as float bits: values are >= 0, so
// integer max of the bit patterns is the float max).
__global__ void k_colmax(const float* __restrict__ D, int64_t n, int64_t ldd,
                         unsigned* __restrict__ colmax) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int64_t i0 = (int64_t)blockIdx.y * 256;
  unsigned m = 0;
  for (int64_t i = i0; i < i0 + 256 && i < j; ++i) {
    const float v = fabsf(D[i * ldd + j]);
    m = max(m, __float_as_uint(v));
  }
  if (m) atomicMax(colmax + j, m);
}

__global__ void k_scale_from_max(unsigned* colmax_bits, int64_t n) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const float mx = __uint_as_float(colmax_bits[j]);
  const float sc = mx > 0.f ? mx / 448.f : 1.f;
  reinterpret_cast<float*>(colmax_bits)[j] = sc;
}

// Block (x = tile, y = 256-element slice of it); one thread per stored element.
template <int DT>
__global__ void k_pack(const float* __restrict__ D, int64_t n, int64_t ldd, int64_t T,
                       int64_t plane, void* __restrict__ out, const float* __restrict__ scale) {
  __shared__ int s_ij[2];
  const int64_t t = blockIdx.x;
  if (threadIdx.x == 0) tile_decode(t, T, s_ij[0], s_ij[1]);
  __syncthreads();
  const int I = s_ij[0], J = s_ij[1];
  const int rc = (int)blockIdx.y * blockDim.x + threadIdx.x;
  const int64_t e = t * (TILE * TILE) + rc;
  const int64_t i = (int64_t)I * TILE + rc / TILE, j = (int64_t)J * TILE + rc % TILE;
  const float v = (i < n && j < n && i < j) ? D[i * ldd + j] : 0.f;
  if (DT == GINI_F32) {
    reinterpret_cast<float*>(out)[e] = v;
  } else if (DT == GINI_BF16) {
    reinterpret_cast<__nv_bfloat16*>(out)[e] = __float2bfloat16_rn(v);
  } else if (DT == GINI_BF16X2) {
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    reinterpret_cast<__nv_bfloat16*>(out)[e] = hi;
    reinterpret_cast<__nv_bfloat16*>(out)[plane + e] = __float2bfloat16_rn(v - __bfloat162float(hi));
  } else {
    const float sc = (j < n) ? scale[j] : 1.f;
    reinterpret_cast<__nv_fp8_storage_t*>(out)[e] =
        __nv_cvt_float_to_fp8(v / sc, __NV_SATFINITE, __NV_E4M3);
  }
}

extern "C" int gini_pack(const float* delta_full_dev, int64_t n, int64_t ldd, int dtype,
                         void* packed_dev, float* col_scale_dev, void* stream) {
  NvtxRange nvtx_range("gini_pack");
  if (!delta_full_dev || !packed_dev || n < 2 || ldd < n || n > ((int64_t)1 << 31))
    return GINI_EINVAL;
  if (dtype < GINI_F32 || dtype > GINI_FP8E4M3) return GINI_EINVAL;
  if (dtype == GINI_FP8E4M3 && !col_scale_dev) return GINI_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t T = tiles_1d(n);
  const int64_t plane = gini_tiled_elems(n);
  cudaError_t e = cudaSuccess;
  if (dtype == GINI_FP8E4M3) {
    e = cudaMemsetAsync(col_scale_dev, 0, sizeof(float) * n, s);
    if (e == cudaSuccess) {
      dim3 g((unsigned)((n + 255) / 256), (unsigned)((n + 255) / 256));
      gini_count_launch(2);
      k_colmax<<<g, 256, 0, s>>>(delta_full_dev, n, ldd, reinterpret_cast<unsigned*>(col_scale_dev));
      k_scale_from_max<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(
          reinterpret_cast<unsigned*>(col_scale_dev), n);
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess) {
    const dim3 blocks((unsigned)(T * (T + 1) / 2), TILE * TILE / 256);
    gini_count_launch(1);
    switch (dtype) {
      case GINI_F32: k_pack<GINI_F32><<<blocks, 256, 0, s>>>(delta_full_dev, n, ldd, T, plane, packed_dev, col_scale_dev); break;
      case GINI_BF16: k_pack<GINI_BF16><<<blocks, 256, 0, s>>>(delta_full_dev, n, ldd, T, plane, packed_dev, col_scale_dev); break;
      case GINI_BF16X2: k_pack<GINI_BF16X2><<<blocks, 256, 0, s>>>(delta_full_dev, n, ldd, T, plane, packed_dev, col_scale_dev); break;
      default: k_pack<GINI_FP8E4M3><<<blocks, 256, 0, s>>>(delta_full_dev, n, ldd, T, plane, packed_dev, col_scale_dev); break;
    }
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) { gini_set_cuda_error(e); return GINI_ECUDA; }
  return GINI_OK;
}

// ---------------------------------------------------------- delta sums ----

// sum_{i<j} delta and delta^2 over a stored matrix; one thread per row of the
// FULL layout or per stored tile element of the TILED one.
template <int DT>
__device__ __forceinline__ float tiled_value(const void* D, int64_t e, int64_t plane,
                                             const float* scale, int64_t j) {
  if (DT == GINI_F32) return reinterpret_cast<const float*>(D)[e];
  if (DT == GINI_BF16) return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(D)[e]);
  if (DT == GINI_BF16X2)
    return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(D)[e]) +
           __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(D)[plane + e]);
  __half_raw hr = __nv_cvt_fp8_to_halfraw(reinterpret_cast<const __nv_fp8_storage_t*>(D)[e],
                                          __NV_E4M3);
  return __half2float(__half(hr)) * scale[j];
}

__device__ __forceinline__ void block_sums_add(double a, double b, double* out) {
  __shared__ double s[2][8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    a += __shfl_xor_sync(FULL_MASK, a, o);
    b += __shfl_xor_sync(FULL_MASK, b, o);
  }
  if (lane == 0) {
    s[0][warp] = a;
    s[1][warp] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double x = 0.0, y = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      x += s[0][w];
      y += s[1][w];
    }
    atomicAdd(out, x);
    atomicAdd(out + 1, y);
  }
}

__global__ void k_sums_full(const float* __restrict__ D, int64_t n, int64_t ldd, double* out) {
  double a = 0.0, b = 0.0;
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x)
    for (int64_t j = i + 1 + threadIdx.x; j < n; j += blockDim.x) {
      const double v = D[i * ldd + j];
      a += v;
      b += v * v;
    }
  block_sums_add(a, b, out);
}

template <int DT>
__global__ void k_sums_tiled(const void* D, int64_t n, int64_t T, int64_t plane,
                             const float* scale, double* out) {
  __shared__ int s_ij[2];
  const int64_t t = blockIdx.x;
  if (threadIdx.x == 0) tile_decode(t, T, s_ij[0], s_ij[1]);
  __syncthreads();
  double a = 0.0, b = 0.0;
  for (int rc = threadIdx.x; rc < TILE * TILE; rc += blockDim.x) {
    const int64_t i = (int64_t)s_ij[0] * TILE + rc / TILE, j = (int64_t)s_ij[1] * TILE + rc % TILE;
    if (i < j && j < n) {
      const double v = tiled_value<DT>(D, t * TILE * TILE + rc, plane, scale, j);
      a += v;
      b += v * v;
    }
  }
  block_sums_add(a, b, out);
}

extern "C" int gini_delta_sums(const void* delta_dev, int64_t n, int layout, int dtype,
                               int64_t ldd, const float* col_scale_dev, double* sums_dev,
                               void* stream) {
  if (!delta_dev || !sums_dev || n < 2 || n > ((int64_t)1 << 31)) return GINI_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(sums_dev, 0, 2 * sizeof(double), s);
  if (e != cudaSuccess) { gini_set_cuda_error(e); return GINI_ECUDA; }
  if (layout == GINI_LAYOUT_FULL) {
    if (dtype != GINI_F32 || ldd < n) return GINI_EINVAL;
    const unsigned g = (unsigned)(n < 4096 ? n : 4096);
    gini_count_launch(1);
    k_sums_full<<<g, 256, 0, s>>>((const float*)delta_dev, n, ldd, sums_dev);
  } else if (layout == GINI_LAYOUT_TILED) {
    if (dtype == GINI_FP8E4M3 && !col_scale_dev) return GINI_EINVAL;
    const int64_t T = tiles_1d(n), plane = gini_tiled_elems(n);
    const unsigned g = (unsigned)(T * (T + 1) / 2);
    gini_count_launch(1);
    switch (dtype) {
      case GINI_F32: k_sums_tiled<GINI_F32><<<g, 256, 0, s>>>(delta_dev, n, T, plane, col_scale_dev, sums_dev); break;
      case GINI_BF16: k_sums_tiled<GINI_BF16><<<g, 256, 0, s>>>(delta_dev, n, T, plane, col_scale_dev, sums_dev); break;
      case GINI_BF16X2: k_sums_tiled<GINI_BF16X2><<<g, 256, 0, s>>>(delta_dev, n, T, plane, col_scale_dev, sums_dev); break;
      case GINI_FP8E4M3: k_sums_tiled<GINI_FP8E4M3><<<g, 256, 0, s>>>(delta_dev, n, T, plane, col_scale_dev, sums_dev); break;
      default: return GINI_EINVAL;
    }
  } else {
    return GINI_EINVAL;
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) { gini_set_cuda_error(e); return GINI_ECUDA; }
  return GINI_OK;
}
