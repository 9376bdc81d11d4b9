// The alternating nu update of the heavy-tail experiment (Algorithm 2): fit
// an embedding at the current nu (Sammon loss by default), then choose the nu
// of the grid whose dissimilarities the fixed embedding fits best (lowest
// Kruskal stress KS(nu)), and repeat.
//
// Delta is built once for the grid and the starting nu (one sort per pair per
// 8 values) and kept in HBM in the tiled layout; each round is one
// gini_mds_fit at the current nu plus one stress pass per grid value.  The host
// reads back the grid's stresses once per round to choose the next nu.
#include <math.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace gini {

// rowsum[i] += sum_{j != i, delta_ij > 0} 1 / delta_ij over a tiled F32 matrix
// (each stored pair adds to its row and its column).
__global__ void __launch_bounds__(256) k_inv_rowsum(const float* __restrict__ D, int64_t n,
                                                    int64_t tiles, double* __restrict__ rowsum) {
  __shared__ double s_row[TILE], s_col[TILE];
  __shared__ int s_ij[2];
  const int64_t ntiles = tiles * (tiles + 1) / 2;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    __syncthreads();
    if (threadIdx.x == 0) tile_decode(t, tiles, s_ij[0], s_ij[1]);
    if (threadIdx.x < TILE) s_row[threadIdx.x] = s_col[threadIdx.x] = 0.0;
    __syncthreads();
    const int64_t i0 = (int64_t)s_ij[0] * TILE, j0 = (int64_t)s_ij[1] * TILE;
    // thread -> column c = threadIdx.x % 128, rows r = threadIdx.x / 128 + 2 m
    const int c = threadIdx.x % TILE;
    double col = 0.0;
    for (int r = threadIdx.x / TILE; r < TILE; r += 2) {
      const int64_t gi = i0 + r, gj = j0 + c;
      double v = 0.0;
      if (gi < gj && gj < n) {
        const float d = D[t * TILE * TILE + r * TILE + c];
        if (d > 0.f) v = 1.0 / (double)d;
      }
      col += v;
      // row r: sum over the warp's 32 columns, then one shared atomic per warp
      double w = v;
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) w += __shfl_xor_sync(FULL_MASK, w, o);
      if ((threadIdx.x & 31) == 0 && w != 0.0) atomicAdd(&s_row[r], w);
    }
    atomicAdd(&s_col[c], col);
    __syncthreads();
    if (threadIdx.x < TILE) {
      const int64_t gi = i0 + threadIdx.x, gj = j0 + threadIdx.x;
      if (gi < n && s_row[threadIdx.x] != 0.0) atomicAdd(rowsum + gi, s_row[threadIdx.x]);
      if (gj < n && s_col[threadIdx.x] != 0.0) atomicAdd(rowsum + gj, s_col[threadIdx.x]);
    }
  }
}

__global__ void k_max_reduce(const double* __restrict__ v, int64_t n, double* out) {
  __shared__ double s[32];
  double m = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, v[i]);
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) m = fmax(m, __shfl_xor_sync(FULL_MASK, m, o));
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, s[w]);
    *out = fmax(m, s[0]);
  }
}

}  // namespace gini

using namespace gini;

extern "C" void gini_set_cuda_error(cudaError_t e);

namespace {

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

struct AltLayout {
  size_t inner = 0, off_delta = 0, off_sums = 0, off_rows = 0, off_stress = 0, total = 0;
};

AltLayout alt_layout(int64_t n, int64_t p, int k, int nvals, int iters) {
  AltLayout L;
  L.inner = std::max({gini_workspace_size(GINI_OP_FIT, n, 0, k, iters),
                      gini_workspace_size(GINI_OP_STRESS, n, 0, k, 0),
                      gini_workspace_size(GINI_OP_DIST, n, p, 0, 0)});
  size_t off = al256(L.inner);
  L.off_delta = off;  off += al256(sizeof(float) * (size_t)gini_tiled_elems(n) * nvals);
  L.off_sums = off;   off += al256(sizeof(double) * 2 * (size_t)nvals);
  L.off_rows = off;   off += al256(sizeof(double) * ((size_t)n + 1));
  L.off_stress = off; off += al256(sizeof(double) * ((size_t)nvals + 1));
  L.total = off;
  return L;
}

// Curvature constant of one pair's embedding distance: (d/dy)^2 summed over
// the k components is at most k ((k/2) w_max)^2 for the Gini metric
// (w_max = ((k-1)/k)^{nu-1}) and 1 for the Euclidean one.
double metric_curv(int metric, int k, double nu) {
  if (metric == GINI_METRIC_EUCLID) return 1.0;
  const double w = pow((k - 1.0) / k, nu - 1.0);
  return k * (0.5 * k * w) * (0.5 * k * w);
}

}  // namespace

extern "C" size_t gini_alternating_nu_workspace_size(int64_t n, int64_t p, int k, int n_nu,
                                                     int iters) {
  if (n < 2 || p < 1 || k < 1 || n_nu < 1 || iters < 0) return 0;
  return alt_layout(n, p, k, n_nu + 1, iters).total;
}

extern "C" int gini_alternating_nu(const float* X_dev, int64_t n, int64_t p, int64_t ldx, int k,
                                   const double* nu_host, int n_nu, double nu_start, int rounds,
                                   int iters, double eta0, int metric, int loss, float* Y_dev,
                                   double* nu_path_host, double* ks_host, void* ws,
                                   size_t ws_bytes, void* stream) {
  NvtxRange nvtx_range("gini_alternating_nu");
  if (!X_dev || !nu_host || !Y_dev || !nu_path_host || !ks_host || !ws) return GINI_EINVAL;
  if (ws_misaligned(ws)) return GINI_EINVAL;
  if (n < 2 || p < 1 || p > 8192 || ldx < p || k < 2 || k > 8 || n_nu < 1 || n_nu > 64 ||
      rounds < 1 || iters < 0)
    return GINI_EINVAL;
  if (metric != GINI_METRIC_GINI && metric != GINI_METRIC_EUCLID) return GINI_EINVAL;
  if (loss != GINI_LOSS_KRUSKAL && loss != GINI_LOSS_SAMMON) return GINI_EINVAL;
  if (!(eta0 > 0.0) || !std::isfinite(eta0)) return GINI_EINVAL;
  std::vector<double> nus(nu_host, nu_host + n_nu);
  nus.push_back(nu_start);
  for (double v : nus)
    if (!(v > 1.0) || !std::isfinite(v)) return GINI_EINVAL;
  const int nvals = n_nu + 1;
  const AltLayout L = alt_layout(n, p, k, nvals, iters);
  if (ws_bytes < L.total) return GINI_ENOMEM;
  char* base = reinterpret_cast<char*>(ws);
  float* delta = reinterpret_cast<float*>(base + L.off_delta);
  double* sums = reinterpret_cast<double*>(base + L.off_sums);
  double* rows = reinterpret_cast<double*>(base + L.off_rows);
  double* stress = reinterpret_cast<double*>(base + L.off_stress);
  const int64_t plane = gini_tiled_elems(n), tiles = tiles_1d(n);
  cudaStream_t s = (cudaStream_t)stream;

  // Delta for the grid and the start, 8 values per sort of each pair.
  for (int v0 = 0; v0 < nvals; v0 += 8) {
    const int nc = std::min(8, nvals - v0);
    int st = gini_dist(X_dev, n, p, ldx, nus.data() + v0, nc, GINI_LAYOUT_TILED, GINI_F32,
                       delta + (size_t)v0 * plane, 0, plane, nullptr, nullptr, ws, L.inner,
                       stream);
    if (st != GINI_OK) return st;
  }
  for (int v = 0; v < nvals; ++v) {
    int st = gini_delta_sums(delta + (size_t)v * plane, n, GINI_LAYOUT_TILED, GINI_F32, 0,
                             nullptr, sums + 2 * v, stream);
    if (st != GINI_OK) return st;
  }
  std::vector<double> hsums(2 * nvals), hstress(nvals);
  cudaError_t e = cudaMemcpyAsync(hsums.data(), sums, sizeof(double) * 2 * nvals,
                                  cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) { gini_set_cuda_error(e); return GINI_ECUDA; }
  int st = gini_check(ws, stream);
  if (st != GINI_OK) return st;
  for (int v = 0; v < nvals; ++v)
    if (!(hsums[2 * v + 1] > 0.0)) return GINI_EDEGENERATE;

  int cur = n_nu;  // index into nus of the current nu (the start)
  nu_path_host[0] = nu_start;
  for (int t = 0; t < rounds; ++t) {
    const double nu = nus[cur];
    const float* Dc = delta + (size_t)cur * plane;
    // step: eta0 over a Gershgorin bound on the Gauss-Newton curvature of S
    double eta;
    const double c = metric_curv(metric, k, nu);
    if (loss == GINI_LOSS_KRUSKAL) {
      eta = eta0 * hsums[2 * cur + 1] / (2.0 * (double)(n - 1) * c);
    } else {
      e = cudaMemsetAsync(rows, 0, sizeof(double) * (size_t)n, s);
      if (e != cudaSuccess) { gini_set_cuda_error(e); return GINI_ECUDA; }
      gini_count_launch(2);
      k_inv_rowsum<<<(unsigned)std::min<int64_t>(tiles * (tiles + 1) / 2, 152 * 8), 256, 0, s>>>(
          Dc, n, tiles, rows);
      k_max_reduce<<<1, 1024, 0, s>>>(rows, n, rows + n);
      double mx = 0.0;
      e = cudaMemcpyAsync(&mx, rows + n, sizeof(double), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) { gini_set_cuda_error(e); return GINI_ECUDA; }
      if (!(mx > 0.0)) return GINI_EDEGENERATE;
      eta = eta0 * hsums[2 * cur] / (2.0 * c * mx);
    }
    gini_fit_args a{};
    a.n = n;
    a.k = k;
    a.nu = nu;
    a.delta_dev = Dc;
    a.layout = GINI_LAYOUT_TILED;
    a.dtype = GINI_F32;
    a.sum_delta2 = loss == GINI_LOSS_SAMMON ? hsums[2 * cur] : hsums[2 * cur + 1];
    a.eta = eta;
    a.iters = iters;
    a.Y_dev = Y_dev;
    a.metric = metric;
    a.loss = loss;
    st = gini_mds_fit(&a, ws, L.inner, stream);
    if (st != GINI_OK) return st;
    // KS(nu) of the fixed embedding for every grid value
    for (int v = 0; v < n_nu; ++v) {
      st = gini_stress_grad_ex(Y_dev, n, k, nus[v], delta + (size_t)v * plane, GINI_LAYOUT_TILED,
                               GINI_F32, 0, nullptr, metric, GINI_LOSS_KRUSKAL,
                               hsums[2 * v + 1], stress + v, nullptr, ws, L.inner, stream);
      if (st != GINI_OK) return st;
    }
    e = cudaMemcpyAsync(hstress.data(), stress, sizeof(double) * n_nu, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { gini_set_cuda_error(e); return GINI_ECUDA; }
    st = gini_check(ws, stream);
    if (st != GINI_OK) return st;
    int best = 0;
    for (int v = 0; v < n_nu; ++v) {
      ks_host[(size_t)t * n_nu + v] = sqrt(hstress[v]);
      if (hstress[v] < hstress[best]) best = v;
    }
    cur = best;
    nu_path_host[t + 1] = nus[cur];
  }
  return GINI_OK;
}
