// Classical MDS of a dissimilarity matrix (Section IV-A): the Gram matrix
// B = -1/2 H D2 H (D2 the elementwise squares, H = I - 11'/n), its top k
// eigenpairs, and the embedding V_k Lambda_k^{1/2}.  Used as a starting point
// for the stress fits.
//
// B is never formed.  Block subspace iteration with an oversampled block of
// m = min(16, n) columns: each product streams the stored matrix once (squares
// on the fly, both halves of the symmetric matrix from the stored triangle);
// the block is re-orthonormalised twice per product through its FP64 Gram
// matrix (Cholesky QR, repeated to recover the orthogonality FP32 loses;
// columns whose residual vanishes -- B of low rank -- are set to zero).  After
// a few plain products a Rayleigh-Ritz step gives the most negative Ritz value
// theta_min, and the remaining products use B + max(0, -theta_min) I so that
// the largest algebraic eigenvalues, not the largest in magnitude, dominate
// (Gini dissimilarities are not Euclidean, so B has negative eigenvalues).  A
// final Rayleigh-Ritz step (Jacobi on the m x m projection) gives the top k.
#include <math.h>

#include <algorithm>

#include "common.cuh"

namespace gini {

constexpr int CMDS_KMAX = 8;   // embedding dimensions a caller may ask for
constexpr int CMDS_M = 16;     // columns of the iterated block
constexpr int CMDS_WARM = 4;   // plain products before the shift is estimated

struct CmdsParams {
  const void* delta;
  int64_t n, ldd, tiles, plane;
  const float* col_scale;
  int m;
};

template <int DT>
__device__ __forceinline__ float stored_value(const void* D, int64_t e, int64_t plane,
                                              const float* sc, int64_t j) {
  if (DT == GINI_F32) return reinterpret_cast<const float*>(D)[e];
  if (DT == GINI_BF16) return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(D)[e]);
  if (DT == GINI_BF16X2)
    return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(D)[e]) +
           __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(D)[plane + e]);
  __half_raw hr =
      __nv_cvt_fp8_to_halfraw(reinterpret_cast<const __nv_fp8_storage_t*>(D)[e], __NV_E4M3);
  return __half2float(__half(hr)) * sc[j];
}

// W += D2 V over the stored triangle: one CTA per tile (grid-stride); the tile's
// row block and column block of V sit in shared memory, the tile's squares are
// staged 32 rows at a time.  Each thread owns outputs o = threadIdx.x + q * 256
// (q < m) of the 2 * TILE * m outputs of the tile: (side, point l, column c),
// side 0 the tile's rows (sums over its columns), side 1 its columns.
template <int DT>
__global__ void __launch_bounds__(256) k_cmds_matvec_tiled(const CmdsParams P,
                                                           const float* __restrict__ V,
                                                           float* __restrict__ W) {
  __shared__ float s_v[2][TILE][CMDS_M];
  __shared__ float s_d[32][TILE + 1];
  __shared__ int s_ij[2];
  const int m = P.m;
  const int64_t ntiles = P.tiles * (P.tiles + 1) / 2;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    __syncthreads();
    if (threadIdx.x == 0) tile_decode(t, P.tiles, s_ij[0], s_ij[1]);
    __syncthreads();
    const int64_t i0 = (int64_t)s_ij[0] * TILE, j0 = (int64_t)s_ij[1] * TILE;
    for (int e = threadIdx.x; e < 2 * TILE * m; e += blockDim.x) {
      const int side = e / (TILE * m), l = (e / m) % TILE, c = e % m;
      const int64_t g = (side ? j0 : i0) + l;
      s_v[side][l][c] = g < P.n ? V[g * m + c] : 0.f;
    }
    float acc[CMDS_M];
#pragma unroll
    for (int q = 0; q < CMDS_M; ++q) acc[q] = 0.f;
    for (int rb = 0; rb < TILE; rb += 32) {
      __syncthreads();
      for (int e = threadIdx.x; e < 32 * TILE; e += blockDim.x) {
        const int r = e / TILE, c = e % TILE;
        const int64_t gi = i0 + rb + r, gj = j0 + c;
        float v = 0.f;
        if (gi < gj && gj < P.n) {
          v = stored_value<DT>(P.delta, t * TILE * TILE + (rb + r) * TILE + c, P.plane,
                               P.col_scale, gj);
          v *= v;
        }
        s_d[r][c] = v;
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < CMDS_M; ++q) {
        if (q < m) {
          const int o = threadIdx.x + q * 256;
          const int side = o / (TILE * m), l = (o / m) % TILE, c = o % m;
          float a = 0.f;
          if (side == 0) {
            if (l >= rb && l < rb + 32)
              for (int cc = 0; cc < TILE; ++cc) a = fmaf(s_d[l - rb][cc], s_v[1][cc][c], a);
          } else {
            for (int r = 0; r < 32; ++r) a = fmaf(s_d[r][l], s_v[0][rb + r][c], a);
          }
          acc[q] += a;
        }
      }
    }
#pragma unroll
    for (int q = 0; q < CMDS_M; ++q) {
      if (q < m) {
        const int o = threadIdx.x + q * 256;
        const int side = o / (TILE * m), l = (o / m) % TILE, c = o % m;
        const int64_t g = (side ? j0 : i0) + l;
        if (g < P.n && acc[q] != 0.f) atomicAdd(W + g * m + c, acc[q]);
      }
    }
  }
}

// FULL layout: warp per row, W[i] = sum_{j != i} D2_ij V[j].
__global__ void __launch_bounds__(256) k_cmds_matvec_full(const CmdsParams P,
                                                          const float* __restrict__ V,
                                                          float* __restrict__ W) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float* D = reinterpret_cast<const float*>(P.delta);
  const int m = P.m;
  for (int64_t i = (int64_t)blockIdx.x * 8 + warp; i < P.n; i += (int64_t)gridDim.x * 8) {
    float acc[CMDS_M];
#pragma unroll
    for (int c = 0; c < CMDS_M; ++c) acc[c] = 0.f;
    for (int64_t j = lane; j < P.n; j += 32) {
      float d = (j == i) ? 0.f : D[i * P.ldd + j];
      d *= d;
#pragma unroll
      for (int c = 0; c < CMDS_M; ++c)
        if (c < m) acc[c] = fmaf(d, V[j * m + c], acc[c]);
    }
#pragma unroll
    for (int c = 0; c < CMDS_M; ++c) {
      if (c < m) {
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) acc[c] += __shfl_xor_sync(FULL_MASK, acc[c], o);
        if (lane == 0) W[i * m + c] = acc[c];
      }
    }
  }
}

// Column sums of X (n x m) in FP64: thread c of each block sums column c over
// the block's rows (rows staged through shared memory), one atomic per block.
__global__ void __launch_bounds__(256) k_cmds_colsum(const float* __restrict__ X, int64_t n,
                                                     int m, double* sums) {
  __shared__ float s_x[256][CMDS_M + 1];
  double acc = 0.0;
  for (int64_t r0 = (int64_t)blockIdx.x * 256; r0 < n; r0 += (int64_t)gridDim.x * 256) {
    __syncthreads();
    for (int e = threadIdx.x; e < 256 * m; e += 256) {
      const int64_t r = r0 + e / m;
      s_x[e / m][e % m] = r < n ? X[r0 * m + e] : 0.f;
    }
    __syncthreads();
    if (threadIdx.x < m)
      for (int r = 0; r < 256; ++r) acc += s_x[r][threadIdx.x];
  }
  if (threadIdx.x < m) atomicAdd(sums + threadIdx.x, acc);
}

// The start block: uniform entries in [-1, 1) from SplitMix64 (Steele, Lea and
// Flood 2014) of seed + element index; any block that spans the wanted
// eigenvectors serves.
__global__ void k_cmds_start(float* V, int64_t count, uint64_t seed) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= count) return;
  uint64_t z = seed + 0x9e3779b97f4a7c15ull * (uint64_t)(e + 1);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  z ^= z >> 31;
  V[e] = (float)(z >> 40) * 0x1p-23f - 1.f;
}

// X <- scale * (X - mean(X)) + shift * V   (column means from `sums`)
__global__ void k_cmds_center(float* X, const float* V, int64_t n, int m, const double* sums,
                              float scale, const float* shift) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * m) return;
  const int c = (int)(e % m);
  const float mean = (float)(sums[c] / (double)n);
  float v = scale * (X[e] - mean);
  if (shift) v = fmaf(*shift, V[e], v);
  X[e] = v;
}

// G += A' B (m x m, FP64): rows staged 256 at a time in shared memory; thread
// t < m*m owns entry (t / m, t % m); one atomic per block and entry.
__global__ void __launch_bounds__(256) k_cmds_gram(const float* __restrict__ A,
                                                   const float* __restrict__ B, int64_t n, int m,
                                                   double* G) {
  __shared__ float s_a[256][CMDS_M];
  __shared__ float s_b[256][CMDS_M];
  const int a = threadIdx.x / m, b = threadIdx.x % m;
  const bool owner = threadIdx.x < m * m;
  double acc = 0.0;
  for (int64_t r0 = (int64_t)blockIdx.x * 256; r0 < n; r0 += (int64_t)gridDim.x * 256) {
    __syncthreads();
    for (int e = threadIdx.x; e < 256 * m; e += 256) {
      const bool in = r0 + e / m < n;
      s_a[e / m][e % m] = in ? A[r0 * m + e] : 0.f;
      s_b[e / m][e % m] = in ? B[r0 * m + e] : 0.f;
    }
    __syncthreads();
    if (owner)
      for (int r = 0; r < 256; ++r) acc += (double)s_a[r][a] * (double)s_b[r][b];
  }
  if (owner) atomicAdd(G + threadIdx.x, acc);
}

// From the Gram matrix G = W'W (m x m): R^-1 with G = R'R (Cholesky), row-major
// in `rinv`.  A column whose pivot falls to 1e-12 of the largest diagonal entry
// lies in the span of the earlier ones: its row and column of R^-1 are zero,
// so that column of W R^-1 is zero and stays zero.
__global__ void k_cmds_chol(const double* G, int m, float* rinv) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double R[CMDS_M][CMDS_M] = {};
  bool dead[CMDS_M];
  double mx = 0.0;
  for (int j = 0; j < m; ++j) mx = fmax(mx, G[j * m + j]);
  for (int j = 0; j < m; ++j) {
    double s = G[j * m + j];
    for (int p = 0; p < j; ++p) s -= R[p][j] * R[p][j];
    dead[j] = !(s > 1e-12 * mx);
    if (dead[j]) continue;
    R[j][j] = sqrt(s);
    for (int c = j + 1; c < m; ++c) {
      double t = G[j * m + c];
      for (int p = 0; p < j; ++p) t -= R[p][j] * R[p][c];
      R[j][c] = t / R[j][j];
    }
  }
  double X[CMDS_M][CMDS_M] = {};  // inverse of R on the live indices
  for (int c = 0; c < m; ++c) {
    if (dead[c]) continue;
    X[c][c] = 1.0 / R[c][c];
    for (int r = c - 1; r >= 0; --r) {
      if (dead[r]) continue;
      double t = 0.0;
      for (int p = r + 1; p <= c; ++p) t += R[r][p] * X[p][c];
      X[r][c] = -t / R[r][r];
    }
  }
  for (int a = 0; a < m; ++a)
    for (int b = 0; b < m; ++b) rinv[a * m + b] = (float)X[a][b];
}

// Y = W M with W n x m and M m x kout (row-major); in place when Y == W (each
// thread reads its whole row before writing).
__global__ void k_cmds_apply(const float* W, const float* M, int64_t n, int m, int kout,
                             float* Y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float w[CMDS_M];
#pragma unroll
  for (int c = 0; c < CMDS_M; ++c) w[c] = c < m ? W[i * m + c] : 0.f;
  for (int c = 0; c < kout; ++c) {
    float a = 0.f;
#pragma unroll
    for (int p = 0; p < CMDS_M; ++p)
      if (p < m) a = fmaf(w[p], M[p * kout + c], a);
    Y[i * kout + c] = a;
  }
}

// Rayleigh-Ritz: T = V'BV (G, symmetric m x m).  Cyclic Jacobi gives
// T = Q diag(theta) Q'.  With `M`, writes the top k (descending) as
// M = Q_k diag(sqrt(max(theta, 0))) (m x k, for Y = V M) and `lambda`; with
// `shift`, writes max(0, -min theta).
__global__ void k_cmds_ritz(const double* G, int m, int k, float* M, double* lambda,
                            float* shift) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double A[CMDS_M][CMDS_M], Q[CMDS_M][CMDS_M];
  double fro = 0.0;
  for (int a = 0; a < m; ++a)
    for (int b = 0; b < m; ++b) {
      A[a][b] = 0.5 * (G[a * m + b] + G[b * m + a]);
      Q[a][b] = a == b ? 1.0 : 0.0;
      fro += A[a][b] * A[a][b];
    }
  for (int sweep = 0; sweep < 50; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < m; ++p)
      for (int q = p + 1; q < m; ++q) off += A[p][q] * A[p][q];
    if (!(off > 1e-30 * fro)) break;
    for (int p = 0; p < m; ++p)
      for (int q = p + 1; q < m; ++q) {
        if (A[p][q] == 0.0) continue;
        // the angle that zeroes A[p][q]: tan(2 th) = 2 A_pq / (A_qq - A_pp)
        const double th = 0.5 * atan2(2.0 * A[p][q], A[q][q] - A[p][p]);
        const double c = cos(th), s = sin(th);
        for (int r = 0; r < m; ++r) {  // A <- A J
          const double ap = A[r][p], aq = A[r][q];
          A[r][p] = c * ap - s * aq;
          A[r][q] = s * ap + c * aq;
        }
        for (int r = 0; r < m; ++r) {  // A <- J' A
          const double ap = A[p][r], aq = A[q][r];
          A[p][r] = c * ap - s * aq;
          A[q][r] = s * ap + c * aq;
        }
        for (int r = 0; r < m; ++r) {  // Q <- Q J
          const double qp = Q[r][p], qq = Q[r][q];
          Q[r][p] = c * qp - s * qq;
          Q[r][q] = s * qp + c * qq;
        }
      }
  }
  if (shift) {
    double mn = 0.0;
    for (int a = 0; a < m; ++a) mn = fmin(mn, A[a][a]);
    *shift = (float)(-mn);
  }
  if (!M) return;
  int order[CMDS_M];
  for (int a = 0; a < m; ++a) order[a] = a;
  for (int a = 0; a < k; ++a)
    for (int b = a + 1; b < m; ++b)
      if (A[order[b]][order[b]] > A[order[a]][order[a]]) {
        const int t = order[a];
        order[a] = order[b];
        order[b] = t;
      }
  for (int c = 0; c < k; ++c) {
    const double lam = A[order[c]][order[c]];
    lambda[c] = lam;
    const double sc = lam > 0.0 ? sqrt(lam) : 0.0;
    for (int r = 0; r < m; ++r) M[r * k + c] = (float)(Q[r][order[c]] * sc);
  }
}

}  // namespace gini

using namespace gini;

extern "C" void gini_set_cuda_error(cudaError_t e);

static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

static int cmds_block(int64_t n) { return (int)std::min<int64_t>(CMDS_M, n); }

extern "C" size_t gini_cmds_workspace_size(int64_t n, int k) {
  if (n < 2 || k < 1) return 0;
  const size_t m = (size_t)cmds_block(n);
  return WS_HEADER + 2 * al256(sizeof(float) * (size_t)n * m) +
         al256(sizeof(double) * (CMDS_M * CMDS_M + CMDS_M)) +
         al256(sizeof(float) * (CMDS_M * CMDS_M + 1));
}

extern "C" int gini_classical_mds(const void* delta_dev, int64_t n, int layout, int dtype,
                                  int64_t ldd, const float* col_scale_dev, int k, int iters,
                                  uint64_t seed, float* Y_dev, double* eigvals_dev, void* ws,
                                  size_t ws_bytes, void* stream) {
  NvtxRange nvtx_range("gini_classical_mds");
  if (!delta_dev || !Y_dev || !eigvals_dev || !ws) return GINI_EINVAL;
  if (ws_misaligned(ws)) return GINI_EINVAL;
  if (n < 2 || n > ((int64_t)1 << 31) || k < 1 || k > CMDS_KMAX || k > n || iters < 1)
    return GINI_EINVAL;
  if (layout == GINI_LAYOUT_FULL) {
    if (dtype != GINI_F32 || ldd < n) return GINI_EINVAL;
  } else if (layout == GINI_LAYOUT_TILED) {
    if (dtype < GINI_F32 || dtype > GINI_FP8E4M3) return GINI_EINVAL;
    if (dtype == GINI_FP8E4M3 && !col_scale_dev) return GINI_EINVAL;
  } else {
    return GINI_EINVAL;
  }
  if (ws_bytes < gini_cmds_workspace_size(n, k)) return GINI_ENOMEM;
  const int m = cmds_block(n);
  cudaStream_t s = (cudaStream_t)stream;
  char* p = reinterpret_cast<char*>(ws) + WS_HEADER;
  float* V = reinterpret_cast<float*>(p);
  p += al256(sizeof(float) * (size_t)n * m);
  float* W = reinterpret_cast<float*>(p);
  p += al256(sizeof(float) * (size_t)n * m);
  double* G = reinterpret_cast<double*>(p);  // Gram (m x m) then column sums (m)
  double* sums = G + CMDS_M * CMDS_M;
  p += al256(sizeof(double) * (CMDS_M * CMDS_M + CMDS_M));
  float* small = reinterpret_cast<float*>(p);  // R^-1 or M, then the shift
  float* sigma = small + CMDS_M * CMDS_M;

  CmdsParams P{};
  P.delta = delta_dev;
  P.n = n;
  P.ldd = ldd;
  P.tiles = tiles_1d(n);
  P.plane = gini_tiled_elems(n);
  P.col_scale = col_scale_dev;
  P.m = m;
  const unsigned gb = (unsigned)((n + 255) / 256);
  const unsigned gnm = (unsigned)((n * m + 255) / 256);
  const unsigned gred = (unsigned)std::min<int64_t>((n + 255) / 256, 304);
  const int64_t ntiles = P.tiles * (P.tiles + 1) / 2;
  cudaError_t e = cudaSuccess;
  auto ok = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };

  gini_count_launch(1);
  k_cmds_start<<<gnm, 256, 0, s>>>(V, n * m, seed);
  ok(cudaMemsetAsync(sigma, 0, sizeof(float), s));

  // W = B V (+ shift V)
  auto apply_B = [&](bool shifted) {
    ok(cudaMemsetAsync(sums, 0, sizeof(double) * m, s));
    gini_count_launch(2);
    k_cmds_colsum<<<gred, 256, 0, s>>>(V, n, m, sums);
    k_cmds_center<<<gnm, 256, 0, s>>>(V, V, n, m, sums, 1.f, nullptr);  // V <- H V
    if (layout == GINI_LAYOUT_FULL) {
      gini_count_launch(1);
      k_cmds_matvec_full<<<(unsigned)std::min<int64_t>((n + 7) / 8, 65535), 256, 0, s>>>(P, V, W);
    } else {
      ok(cudaMemsetAsync(W, 0, sizeof(float) * n * m, s));
      const unsigned g = (unsigned)std::min<int64_t>(ntiles, 152 * 8);
      gini_count_launch(1);
      switch (dtype) {
        case GINI_F32: k_cmds_matvec_tiled<GINI_F32><<<g, 256, 0, s>>>(P, V, W); break;
        case GINI_BF16: k_cmds_matvec_tiled<GINI_BF16><<<g, 256, 0, s>>>(P, V, W); break;
        case GINI_BF16X2: k_cmds_matvec_tiled<GINI_BF16X2><<<g, 256, 0, s>>>(P, V, W); break;
        default: k_cmds_matvec_tiled<GINI_FP8E4M3><<<g, 256, 0, s>>>(P, V, W); break;
      }
    }
    ok(cudaMemsetAsync(sums, 0, sizeof(double) * m, s));
    gini_count_launch(2);
    k_cmds_colsum<<<gred, 256, 0, s>>>(W, n, m, sums);
    k_cmds_center<<<gnm, 256, 0, s>>>(W, V, n, m, sums, -0.5f, shifted ? sigma : nullptr);
  };
  auto gram = [&](const float* A, const float* B) {
    ok(cudaMemsetAsync(G, 0, sizeof(double) * m * m, s));
    gini_count_launch(1);
    k_cmds_gram<<<gred, 256, 0, s>>>(A, B, n, m, G);
  };
  // V <- orth(src) by Cholesky QR, twice
  auto orthonormalise = [&](const float* src) {
    gram(src, src);
    gini_count_launch(2);
    k_cmds_chol<<<1, 1, 0, s>>>(G, m, small);
    k_cmds_apply<<<gb, 256, 0, s>>>(src, small, n, m, m, V);
    gram(V, V);
    gini_count_launch(2);
    k_cmds_chol<<<1, 1, 0, s>>>(G, m, small);
    k_cmds_apply<<<gb, 256, 0, s>>>(V, small, n, m, m, V);
  };

  orthonormalise(V);
  for (int it = 0; it < iters; ++it) {
    apply_B(it > CMDS_WARM);
    if (it == CMDS_WARM) {  // W = B V: the Ritz values give the shift
      gram(V, W);
      gini_count_launch(1);
      k_cmds_ritz<<<1, 1, 0, s>>>(G, m, k, nullptr, nullptr, sigma);
    }
    orthonormalise(W);
  }
  // Rayleigh-Ritz on span(V): T = V'BV, Y = V Q_k diag(sqrt(theta_k))
  apply_B(false);
  gram(V, W);
  gini_count_launch(2);
  k_cmds_ritz<<<1, 1, 0, s>>>(G, m, k, small, eigvals_dev, nullptr);
  k_cmds_apply<<<gb, 256, 0, s>>>(V, small, n, m, k, Y_dev);
  ok(cudaGetLastError());
  if (e != cudaSuccess) { gini_set_cuda_error(e); return GINI_ECUDA; }
  return GINI_OK;
}
