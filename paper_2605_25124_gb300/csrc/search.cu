// The nu search of Algorithm 1: for every nu of a grid and every fold of the
// points, build the fold's dissimilarities, fit an embedding, record the
// Kruskal stress KS = sqrt(S(Y_T)); nu* minimises the mean KS over folds.
//
// The folds are independent problems of one batched fit per chunk of up to 8
// nu values (gini_fit_batched builds each fold's Delta for the whole chunk from
// one sort per pair, so a fold's pairs are ranked once per chunk and the whole
// Delta of all n points is never formed: the folds hold n^2/(2K) pairs).  Rows
// of X and the starting points are gathered per fold on the device; the stress
// reduction, the choice of nu* and the scatter of the chosen embedding back to
// point order are kernels too, so nothing waits on the host.
#include <math.h>

#include <algorithm>
#include <vector>

#include "common.cuh"

namespace gini {

constexpr int SEARCH_KMAX = 64;     // folds
constexpr int SEARCH_NUMAX = 64;    // grid values
constexpr int SEARCH_CHUNK = 8;     // nu values per batched fit

struct FoldTable {
  int64_t off[SEARCH_KMAX + 1];  // fold q holds sorted positions off[q] .. off[q+1]-1
  int K;
};

__device__ __forceinline__ int fold_of(const FoldTable& F, int64_t s) {
  int lo = 0, hi = F.K - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (F.off[mid] <= s) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Xg[s] = X[perm[s]] (rows of p floats)
__global__ void k_gather_rows(const float* __restrict__ X, int64_t ldx, int64_t p,
                              const int64_t* __restrict__ perm, int64_t n,
                              float* __restrict__ Xg) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * p) return;
  const int64_t s = e / p, c = e % p;
  Xg[e] = X[perm[s] * ldx + c];
}

// Starting points per fold, as the batched fit wants them: fold q holds
// R x n_q x 2 floats at offset 2 R off[q]; source Y0 is R x n x 2 in point order.
__global__ void k_gather_starts(const float* __restrict__ Y0, int64_t n, int R,
                                const int64_t* __restrict__ perm, const FoldTable F,
                                float* __restrict__ Y0g) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 2 * (int64_t)R * n) return;
  // fold q covers [2 R off[q], 2 R off[q+1])
  const int q = fold_of(F, e / (2 * R));
  const int64_t nq = F.off[q + 1] - F.off[q];
  const int64_t w = e - 2 * (int64_t)R * F.off[q];
  const int64_t r = w / (2 * nq), l = (w / 2) % nq, c = w & 1;
  Y0g[e] = Y0[(r * n + perm[F.off[q] + l]) * 2 + c];
}

// One chunk's final stresses (fold, nu, restart)-major -> KS of the best
// restart per (nu, fold), stored at ks[(v0 + v) * K + q], and that restart.
__global__ void k_search_reduce(const double* __restrict__ fs, int K, int nc, int R, int v0,
                                double* __restrict__ ks, int* __restrict__ best_r) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= K * nc) return;
  const int q = e / nc, v = e % nc;
  double best = INFINITY;
  int br = 0;
  for (int r = 0; r < R; ++r) {
    const double S = fs[((int64_t)q * nc + v) * R + r];
    if (S < best) { best = S; br = r; }  // NaN never wins
  }
  ks[(int64_t)(v0 + v) * K + q] = sqrt(best);
  best_r[(v0 + v) * K + q] = br;
}

// mean KS over folds per nu; nu* = the first minimiser (NaN means never chosen)
__global__ void k_search_select(const double* __restrict__ ks, int n_nu, int K,
                                double* __restrict__ mean_ks, int* __restrict__ best) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double bm = INFINITY;
  int bv = 0;
  for (int v = 0; v < n_nu; ++v) {
    double m = 0.0;
    for (int q = 0; q < K; ++q) m += ks[(int64_t)v * K + q];
    m /= K;
    mean_ks[v] = m;
    if (m < bm) { bm = m; bv = v; }
  }
  *best = bv;
}

// Y[perm[s]] = the embedding of sorted position s from its fold's best restart
// at nu*.  Chunk c of the fit outputs starts at 2 R n * SEARCH_CHUNK * c; inside
// it fold q's block (nc nu values x R restarts x n_q points x 2) starts at
// 2 R nc off[q].
__global__ void k_search_scatter(const float* __restrict__ Ybuf, const int* __restrict__ best,
                                 const int* __restrict__ best_r, int n_nu, int R,
                                 const int64_t* __restrict__ perm, const FoldTable F, int64_t n,
                                 float* __restrict__ Y) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int v = *best;
  const int c = v / SEARCH_CHUNK, vl = v % SEARCH_CHUNK;
  const int nc = min(SEARCH_CHUNK, n_nu - c * SEARCH_CHUNK);
  const int q = fold_of(F, s);
  const int64_t nq = F.off[q + 1] - F.off[q], l = s - F.off[q];
  const int r = best_r[v * F.K + q];
  const float* src = Ybuf + 2 * (int64_t)R * n * SEARCH_CHUNK * c + 2 * (int64_t)R * nc * F.off[q] +
                     (((int64_t)vl * R + r) * nq + l) * 2;
  Y[perm[s] * 2] = src[0];
  Y[perm[s] * 2 + 1] = src[1];
}

}  // namespace gini

using namespace gini;

extern "C" void gini_set_cuda_error(cudaError_t e);
extern "C" int gini_get_deterministic(void);

namespace {

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

struct SearchPlan {
  std::vector<int64_t> perm;   // points sorted by fold (stable)
  FoldTable F{};
  std::vector<gini_problem> probs;
  size_t batch_ws = 0, off_xg = 0, off_y0 = 0, off_perm = 0, off_ybuf = 0, off_fs = 0,
         off_ks = 0, off_br = 0, total = 0;
};

// Validates the folds and lays out the workspace; X pointers filled later.
int plan_search(int64_t n, int64_t p, const int32_t* fold, int K, int n_nu, int R, int iters,
                SearchPlan& pl) {
  if (n < 2 || p < 1 || !fold || K < 1 || K > SEARCH_KMAX || n_nu < 1 || n_nu > SEARCH_NUMAX ||
      R < 1 || iters < 0)
    return GINI_EINVAL;
  std::vector<int64_t> cnt(K + 1, 0);
  for (int64_t i = 0; i < n; ++i) {
    if (fold[i] < 0 || fold[i] >= K) return GINI_EINVAL;
    ++cnt[fold[i] + 1];
  }
  for (int q = 0; q < K; ++q) {
    if (cnt[q + 1] < 2) return GINI_EINVAL;  // every fold needs a pair
    cnt[q + 1] += cnt[q];
  }
  pl.F.K = K;
  for (int q = 0; q <= K; ++q) pl.F.off[q] = cnt[q];
  pl.perm.assign(n, 0);
  std::vector<int64_t> pos(cnt.begin(), cnt.end() - 1);
  for (int64_t i = 0; i < n; ++i) pl.perm[pos[fold[i]]++] = i;
  pl.probs.resize(K);
  for (int q = 0; q < K; ++q)
    pl.probs[q] = gini_problem{nullptr, cnt[q + 1] - cnt[q], p, p};
  const int chunk = std::min(n_nu, SEARCH_CHUNK);
  pl.batch_ws = gini_batch_workspace_size(pl.probs.data(), K, chunk, R, iters, nullptr);
  if (!pl.batch_ws) return GINI_EINVAL;
  size_t off = al256(pl.batch_ws);
  pl.off_xg = off;   off += al256(sizeof(float) * (size_t)n * p);
  pl.off_y0 = off;   off += al256(sizeof(float) * 2 * (size_t)R * n);
  pl.off_perm = off; off += al256(sizeof(int64_t) * (size_t)n);
  pl.off_ybuf = off; off += al256(sizeof(float) * 2 * (size_t)R * n * n_nu);
  // one chunk's final stresses, then KS and best restarts for the grid
  pl.off_fs = off;   off += al256(sizeof(double) * (size_t)K * chunk * R);
  pl.off_ks = off;   off += al256(sizeof(double) * (size_t)K * n_nu);
  pl.off_br = off;   off += al256(sizeof(int) * (size_t)K * n_nu);
  pl.total = off;
  return GINI_OK;
}

}  // namespace

extern "C" size_t gini_nu_search_workspace_size(int64_t n, int64_t p, const int32_t* fold_host,
                                                int K, int n_nu, int restarts, int iters) {
  SearchPlan pl;
  if (plan_search(n, p, fold_host, K, n_nu, restarts, iters, pl) != GINI_OK) return 0;
  return pl.total;
}

extern "C" int gini_nu_search(const float* X_dev, int64_t n, int64_t p, int64_t ldx,
                              const int32_t* fold_host, int K, const double* nu_host, int n_nu,
                              int restarts, int iters, double eta0, const float* Y0_dev,
                              double* ks_dev, double* mean_ks_dev, int* best_dev, float* Y_dev,
                              void* ws, size_t ws_bytes, void* stream) {
  NvtxRange nvtx_range("gini_nu_search");
  if (!X_dev || !nu_host || !Y0_dev || !ks_dev || !mean_ks_dev || !best_dev || !Y_dev || !ws)
    return GINI_EINVAL;
  if (ldx < p) return GINI_EINVAL;
  if (ws_misaligned(ws)) return GINI_EINVAL;
  SearchPlan pl;
  int st = plan_search(n, p, fold_host, K, n_nu, restarts, iters, pl);
  if (st != GINI_OK) return st;
  if (ws_bytes < pl.total) return GINI_ENOMEM;
  char* base = reinterpret_cast<char*>(ws);
  float* Xg = reinterpret_cast<float*>(base + pl.off_xg);
  float* Y0g = reinterpret_cast<float*>(base + pl.off_y0);
  int64_t* perm = reinterpret_cast<int64_t*>(base + pl.off_perm);
  float* Ybuf = reinterpret_cast<float*>(base + pl.off_ybuf);
  double* fs = reinterpret_cast<double*>(base + pl.off_fs);
  double* ks_all = reinterpret_cast<double*>(base + pl.off_ks);
  int* best_r = reinterpret_cast<int*>(base + pl.off_br);
  cudaStream_t s = (cudaStream_t)stream;

  cudaError_t e = cudaMemcpyAsync(perm, pl.perm.data(), sizeof(int64_t) * n,
                                  cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) { gini_set_cuda_error(e); return GINI_ECUDA; }
  gini_count_launch(2);
  k_gather_rows<<<(unsigned)((n * p + 255) / 256), 256, 0, s>>>(X_dev, ldx, p, perm, n, Xg);
  k_gather_starts<<<(unsigned)((2 * restarts * n + 255) / 256), 256, 0, s>>>(
      Y0_dev, n, restarts, perm, pl.F, Y0g);
  for (int q = 0; q < K; ++q) pl.probs[q].X_dev = Xg + pl.F.off[q] * p;

  for (int v0 = 0; v0 < n_nu; v0 += SEARCH_CHUNK) {
    const int nc = std::min(SEARCH_CHUNK, n_nu - v0);
    st = gini_fit_batched(pl.probs.data(), K, nu_host + v0, nc, restarts, iters, eta0, Y0g,
                          Ybuf + 2 * (size_t)restarts * n * v0, nullptr, fs, nullptr, nullptr,
                          ws, pl.batch_ws, stream);
    if (st != GINI_OK) return st;
    gini_count_launch(1);
    k_search_reduce<<<(unsigned)((K * nc + 127) / 128), 128, 0, s>>>(fs, K, nc, restarts, v0,
                                                                      ks_all, best_r);
  }
  gini_count_launch(2);
  k_search_select<<<1, 32, 0, s>>>(ks_all, n_nu, K, mean_ks_dev, best_dev);
  k_search_scatter<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(Ybuf, best_dev, best_r, n_nu,
                                                                 restarts, perm, pl.F, n, Y_dev);
  e = cudaMemcpyAsync(ks_dev, ks_all, sizeof(double) * K * n_nu, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) { gini_set_cuda_error(e); return GINI_ECUDA; }
  return GINI_OK;
}
