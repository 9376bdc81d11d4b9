// Evaluation measures of an embedding (Section V): trustworthiness T(k) and
// the neighbour label agreement NN(k), the silhouette score, and the Pearson
// and Spearman correlations between the pairwise Euclidean distances of the
// data and of the embedding.
//
// Every decision that turns distances into integers (which points are the k
// nearest, the rank of a distance) is taken on FP64 squared distances of the
// FP32 inputs, products and sums rounded separately (no contraction), ties
// going to the smaller index.  Spearman's ranks come from a device-wide LSD
// radix sort of the n(n-1)/2 distances (FP64 bit patterns as keys), then
// midranks over runs of equal keys.
#include <math.h>

#include <algorithm>

#include "common.cuh"

namespace gini {

constexpr int EVAL_KMAX = 64;      // neighbours
constexpr int EVAL_CMAX = 64;      // labels
constexpr int SCAN_TILE = 2048;    // 256 threads x 8 items

__device__ __forceinline__ double sq_dist_f64(const float* a, const float* b, int k) {
  double s = 0.0;
  for (int c = 0; c < k; ++c) {
    const double d = (double)a[c] - (double)b[c];
    s = __dadd_rn(s, __dmul_rn(d, d));
  }
  return s;
}

// (d, l) < (bd, bl) lexicographically
__device__ __forceinline__ bool lex_less(double d, int64_t l, double bd, int64_t bl) {
  return d < bd || (d == bd && l < bl);
}

// ---------------------------------------------------------------- T(k), NN(k)
// One CTA per point i.  The K = max(kt, knn) nearest embedding neighbours come
// from K rounds of a block-wide lexicographic argmin above the previous pick;
// the rank of a neighbour j among the data-space distances from i is
// 1 + #{l != i : (dX(i,l), l) < (dX(i,j), j)}.  acc[0] += sum max(0, r - kt),
// acc[1] += label hits among the first knn.
__global__ void __launch_bounds__(256) k_nbr_scores(const float* __restrict__ X, int64_t n,
                                                    int64_t p, int64_t ldx,
                                                    const float* __restrict__ Y, int k,
                                                    const int* __restrict__ labels, int kt,
                                                    int knn, double* acc) {
  __shared__ double s_bd[8];
  __shared__ int64_t s_bl[8];
  __shared__ int64_t s_nb[EVAL_KMAX];
  __shared__ double s_nbdx[EVAL_KMAX];
  __shared__ unsigned s_cnt[EVAL_KMAX];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int K = kt > knn ? kt : knn;
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
    float yi[8];
    for (int c = 0; c < k; ++c) yi[c] = Y[i * k + c];
    double pd = -1.0;
    int64_t pl = -1;
    for (int r = 0; r < K; ++r) {
      double bd = INFINITY;
      int64_t bl = INT64_MAX;
      for (int64_t l = threadIdx.x; l < n; l += blockDim.x) {
        if (l == i) continue;
        const double d = sq_dist_f64(yi, Y + l * k, k);
        if (lex_less(pd, pl, d, l) && lex_less(d, l, bd, bl)) { bd = d; bl = l; }
      }
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) {
        const double od = __shfl_xor_sync(FULL_MASK, bd, o);
        const int64_t ol = __shfl_xor_sync(FULL_MASK, bl, o);
        if (lex_less(od, ol, bd, bl)) { bd = od; bl = ol; }
      }
      __syncthreads();
      if (lane == 0) { s_bd[warp] = bd; s_bl[warp] = bl; }
      __syncthreads();
      bd = s_bd[0];
      bl = s_bl[0];
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
        if (lex_less(s_bd[w], s_bl[w], bd, bl)) { bd = s_bd[w]; bl = s_bl[w]; }
      if (threadIdx.x == 0) s_nb[r] = bl;
      pd = bd;
      pl = bl;
    }
    __syncthreads();
    if (knn > 0 && labels && threadIdx.x == 0) {
      int hits = 0;
      for (int r = 0; r < knn; ++r) hits += labels[s_nb[r]] == labels[i] ? 1 : 0;
      atomicAdd(acc + 1, (double)hits);
    }
    if (kt > 0) {
      const float* xi = X + i * ldx;
      // the neighbours' data-space distances, each summed in feature order by
      // one thread exactly as the counting loop below sums every distance
      if (threadIdx.x < kt) {
        const float* xj = X + s_nb[threadIdx.x] * ldx;
        double s = 0.0;
        for (int64_t c = 0; c < p; ++c) {
          const double d = (double)xi[c] - (double)xj[c];
          s = __dadd_rn(s, __dmul_rn(d, d));
        }
        s_nbdx[threadIdx.x] = s;
        s_cnt[threadIdx.x] = 0;
      }
      __syncthreads();
      const int64_t lend = (n + 31) / 32 * 32;
      for (int64_t l = threadIdx.x; l < lend; l += blockDim.x) {
        const bool ok = l < n && l != i;
        double s = 0.0;
        if (ok) {
          const float* xl = X + l * ldx;
          for (int64_t c = 0; c < p; ++c) {
            const double d = (double)xi[c] - (double)xl[c];
            s = __dadd_rn(s, __dmul_rn(d, d));
          }
        }
        for (int r = 0; r < kt; ++r) {
          const unsigned b = __ballot_sync(FULL_MASK, ok && lex_less(s, l, s_nbdx[r], s_nb[r]));
          if (lane == 0 && b) atomicAdd(&s_cnt[r], (unsigned)__popc(b));
        }
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        double t = 0.0;
        for (int r = 0; r < kt; ++r) {
          const int64_t rank = (int64_t)s_cnt[r] + 1;
          if (rank > kt) t += (double)(rank - kt);
        }
        atomicAdd(acc, t);
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- silhouette
__global__ void k_label_counts(const int* __restrict__ labels, int64_t n, int C,
                               unsigned* cnt, unsigned* err) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int c = labels[i];
  if (c < 0 || c >= C) { raise_error(err, ERR_NONFINITE); return; }
  atomicAdd(cnt + c, 1u);
}

// One CTA per point: per-thread, per-label sums of embedding distances in
// shared memory (row = thread), then per-label totals; acc += s_i.
__global__ void __launch_bounds__(256) k_silhouette(const float* __restrict__ Y, int64_t n, int k,
                                                    const int* __restrict__ labels, int C,
                                                    const unsigned* __restrict__ cnt,
                                                    double* acc) {
  extern __shared__ double s_sum[];  // blockDim.x x C
  __shared__ double s_tot[EVAL_CMAX];
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
    float yi[8];
    for (int c = 0; c < k; ++c) yi[c] = Y[i * k + c];
    double* mine = s_sum + (size_t)threadIdx.x * C;
    for (int c = 0; c < C; ++c) mine[c] = 0.0;
    for (int64_t l = threadIdx.x; l < n; l += blockDim.x) {
      if (l == i) continue;
      const int c = labels[l];
      if (c < 0 || c >= C) continue;
      mine[c] += __dsqrt_rn(sq_dist_f64(yi, Y + l * k, k));
    }
    __syncthreads();
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
      double t = 0.0;
      for (int w = 0; w < (int)blockDim.x; ++w) t += s_sum[(size_t)w * C + c];
      s_tot[c] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      const int own = labels[i];
      double s = 0.0;
      if (own >= 0 && own < C && cnt[own] > 1) {
        const double a = s_tot[own] / (double)(cnt[own] - 1);
        double b = INFINITY;
        for (int c = 0; c < C; ++c)
          if (c != own && cnt[c] > 0) b = fmin(b, s_tot[c] / (double)cnt[c]);
        if (b < INFINITY) s = (b - a) / fmax(a, b);
      }
      atomicAdd(acc, s);
    }
    __syncthreads();
  }
}

// ------------------------------------------------------- distance correlations
struct PairSums {
  double* sums;          // 5 doubles: sum u, v, u^2, v^2, u v of shifted distances
  double shift_x, shift_y;
};

__device__ __forceinline__ int64_t pair_index(int64_t i, int64_t j, int64_t n) {
  return i * n - i * (i + 1) / 2 + (j - i - 1);
}

// 64 x 64 tiles of the upper triangle; each thread 4 x 4 pairs; features in
// chunks of 32 through shared memory; FP64 accumulation in feature order.
// Writes the FP64 distances' bit patterns (keys) and pair indices (values) for
// the rank pass when kx is given.
__global__ void __launch_bounds__(256) k_pair_dists(const float* __restrict__ X, int64_t n,
                                                    int64_t p, int64_t ldx,
                                                    const float* __restrict__ Y, int k,
                                                    int64_t T, const double* shifts,
                                                    double* sums, unsigned long long* kx,
                                                    unsigned long long* ky, unsigned* vx,
                                                    unsigned* vy) {
  __shared__ float s_a[64][33], s_b[64][33];
  __shared__ double s_red[5][8];
  const int tr = threadIdx.x / 16, tc = threadIdx.x % 16;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const double shx = shifts[0], shy = shifts[1];
  double part[5] = {0, 0, 0, 0, 0};
  const int64_t ntiles = T * (T + 1) / 2;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    int I, J;
    tile_decode(t, T, I, J);
    const int64_t i0 = (int64_t)I * 64, j0 = (int64_t)J * 64;
    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
    for (int64_t c0 = 0; c0 < p; c0 += 32) {
      __syncthreads();
      for (int e = threadIdx.x; e < 64 * 32; e += blockDim.x) {
        const int r = e / 32, c = e % 32;
        const int64_t gi = i0 + r, gj = j0 + r, gc = c0 + c;
        s_a[r][c] = (gi < n && gc < p) ? X[gi * ldx + gc] : 0.f;
        s_b[r][c] = (gj < n && gc < p) ? X[gj * ldx + gc] : 0.f;
      }
      __syncthreads();
      const int cend = (int)((p - c0) < 32 ? (p - c0) : 32);
      for (int c = 0; c < cend; ++c) {
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const double xa = (double)s_a[4 * tr + a][c];
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            const double d = xa - (double)s_b[4 * tc + b][c];
            acc[a][b] = __dadd_rn(acc[a][b], __dmul_rn(d, d));
          }
        }
      }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int64_t i = i0 + 4 * tr + a, j = j0 + 4 * tc + b;
        if (i < j && j < n) {
          const double dx = __dsqrt_rn(acc[a][b]);
          const double dy = __dsqrt_rn(sq_dist_f64(Y + i * k, Y + j * k, k));
          const double u = dx - shx, v = dy - shy;
          part[0] += u;
          part[1] += v;
          part[2] += u * u;
          part[3] += v * v;
          part[4] += u * v;
          if (kx) {
            const int64_t idx = pair_index(i, j, n);
            kx[idx] = (unsigned long long)__double_as_longlong(dx);
            ky[idx] = (unsigned long long)__double_as_longlong(dy);
            vx[idx] = (unsigned)idx;
            vy[idx] = (unsigned)idx;
          }
        }
      }
  }
#pragma unroll
  for (int q = 0; q < 5; ++q) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) part[q] += __shfl_xor_sync(FULL_MASK, part[q], o);
  }
  if (lane == 0)
    for (int q = 0; q < 5; ++q) s_red[q][warp] = part[q];
  __syncthreads();
  if (threadIdx.x < 5) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += s_red[threadIdx.x][w];
    atomicAdd(sums + threadIdx.x, s);
  }
}

// shifts = distances of pair (0, 1) in both spaces (keeps the sums centred
// near the data, so the variance is not lost to cancellation)
__global__ void k_pair_shift(const float* __restrict__ X, int64_t p, int64_t ldx,
                             const float* __restrict__ Y, int k, double* shifts) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0;
  for (int64_t c = 0; c < p; ++c) {
    const double d = (double)X[c] - (double)X[ldx + c];
    s = __dadd_rn(s, __dmul_rn(d, d));
  }
  shifts[0] = __dsqrt_rn(s);
  shifts[1] = __dsqrt_rn(sq_dist_f64(Y, Y + k, k));
}

// out[q] = Pearson correlation from 5 shifted sums over P pairs
__global__ void k_pearson_finish(const double* sums, double P, double* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double mu = sums[0] / P, mv = sums[1] / P;
  const double cuu = sums[2] / P - mu * mu, cvv = sums[3] / P - mv * mv;
  const double cuv = sums[4] / P - mu * mv;
  *out = cuv / sqrt(cuu * cvv);
}

// ---------------------------------------------------------- scan and radix sort
// Exclusive scan of unsigned values, tiles of 2048 (256 threads x 8 items,
// thread t owning items 8t .. 8t+7 of the tile).
__device__ __forceinline__ unsigned block_exclusive_scan(unsigned v, unsigned& total) {
  __shared__ unsigned s_w[8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_up_sync(FULL_MASK, x, o);
    if (lane >= o) x += y;
  }
  __syncthreads();
  if (lane == 31) s_w[warp] = x;
  __syncthreads();
  unsigned wpre = 0;
  total = 0;
  for (int w = 0; w < 8; ++w) {
    if (w < warp) wpre += s_w[w];
    total += s_w[w];
  }
  return wpre + x - v;
}

__global__ void __launch_bounds__(256) k_tile_sums(const unsigned* __restrict__ d, int64_t N,
                                                   unsigned* sums) {
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + threadIdx.x * 8;
  unsigned s = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q)
    if (base + q < N) s += d[base + q];
  unsigned total;
  block_exclusive_scan(s, total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(256) k_tile_scan(unsigned* d, int64_t N,
                                                   const unsigned* __restrict__ pre) {
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + threadIdx.x * 8;
  unsigned v[8], s = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    v[q] = base + q < N ? d[base + q] : 0u;
    s += v[q];
  }
  unsigned total;
  unsigned run = block_exclusive_scan(s, total) + (pre ? pre[blockIdx.x] : 0u);
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    if (base + q < N) d[base + q] = run;
    run += v[q];
  }
}

static int64_t scan_tmp_elems(int64_t N) {
  int64_t t = 0;
  while (N > SCAN_TILE) {
    N = (N + SCAN_TILE - 1) / SCAN_TILE;
    t += N;
  }
  return t + 1;
}

// exclusive scan in place; tmp holds scan_tmp_elems(N) values
static void exclusive_scan(unsigned* d, int64_t N, unsigned* tmp, cudaStream_t s) {
  const int64_t nb = (N + SCAN_TILE - 1) / SCAN_TILE;
  if (nb <= 1) {
    gini_count_launch(1);
    k_tile_scan<<<1, 256, 0, s>>>(d, N, nullptr);
    return;
  }
  gini_count_launch(1);
  k_tile_sums<<<(unsigned)nb, 256, 0, s>>>(d, N, tmp);
  exclusive_scan(tmp, nb, tmp + nb, s);
  gini_count_launch(1);
  k_tile_scan<<<(unsigned)nb, 256, 0, s>>>(d, N, tmp);
}

// LSD radix sort pass on 8-bit digits: histogram per tile (digit-major),
// then a stable scatter (tile items in index order, ranks inside a round of
// 256 from warp matches, across warps from shared counts).
__global__ void __launch_bounds__(256) k_radix_hist(const unsigned long long* __restrict__ key,
                                                    int64_t N, int shift, unsigned* hist,
                                                    int64_t nb) {
  __shared__ unsigned s_c[256];
  s_c[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  for (int r = 0; r < 8; ++r) {
    const int64_t e = base + r * 256 + threadIdx.x;
    if (e < N) atomicAdd(&s_c[(unsigned)(key[e] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * nb + blockIdx.x] = s_c[threadIdx.x];
}

__global__ void __launch_bounds__(256) k_radix_scatter(
    const unsigned long long* __restrict__ kin, const unsigned* __restrict__ vin, int64_t N,
    int shift, const unsigned* __restrict__ off, int64_t nb, unsigned long long* __restrict__ kout,
    unsigned* __restrict__ vout) {
  __shared__ unsigned s_run[256];
  __shared__ unsigned s_wc[8][256];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  s_run[threadIdx.x] = off[(int64_t)threadIdx.x * nb + blockIdx.x];
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  const unsigned lt = (1u << lane) - 1u;
  for (int r = 0; r < 8; ++r) {
    for (int w = 0; w < 8; ++w) s_wc[w][threadIdx.x] = 0;
    __syncthreads();
    const int64_t e = base + r * 256 + threadIdx.x;
    const bool ok = e < N;
    unsigned long long kv = 0;
    unsigned vv = 0, dig = 256;
    if (ok) {
      kv = kin[e];
      vv = vin[e];
      dig = (unsigned)(kv >> shift) & 255u;
    }
    const unsigned peers = __match_any_sync(FULL_MASK, dig);
    const unsigned before = __popc(peers & lt);
    if (ok && before == 0) s_wc[warp][dig] = __popc(peers);
    __syncthreads();
    if (ok) {
      unsigned pos = s_run[dig] + before;
      for (int w = 0; w < warp; ++w) pos += s_wc[w][dig];
      kout[pos] = kv;
      vout[pos] = vv;
    }
    __syncthreads();
    unsigned add = 0;
    for (int w = 0; w < 8; ++w) add += s_wc[w][threadIdx.x];
    s_run[threadIdx.x] += add;
    __syncthreads();
  }
}

// head flags of runs of equal keys (1 at the first of each run)
__global__ void k_run_heads(const unsigned long long* __restrict__ key, int64_t N,
                            unsigned* flag) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < N) flag[e] = (e == 0 || key[e] != key[e - 1]) ? 1u : 0u;
}

// after the exclusive scan of the head flags: id = scan + flag - 1 is the run
// of sorted position e; a head records its start
__global__ void k_run_starts(const unsigned long long* __restrict__ key, int64_t N,
                             const unsigned* __restrict__ scan, unsigned* start) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < N && (e == 0 || key[e] != key[e - 1])) start[scan[e]] = (unsigned)e;
}

// midrank of sorted position e, stored at its pair's index, minus (N + 1) / 2
__global__ void k_midranks(const unsigned long long* __restrict__ key, int64_t N,
                           const unsigned* __restrict__ scan, const unsigned* __restrict__ start,
                           const unsigned* __restrict__ val, double* rank) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N) return;
  const bool head = (e == 0 || key[e] != key[e - 1]);
  const unsigned id = scan[e] + (head ? 1u : 0u) - 1u;
  const unsigned long long last = scan[N - 1] + ((N == 1 || key[N - 1] != key[N - 2]) ? 1u : 0u);
  const int64_t a = start[id];
  const int64_t b = (id + 1 < last) ? (int64_t)start[id + 1] - 1 : N - 1;
  rank[val[e]] = 0.5 * (double)(a + b + 2) - 0.5 * (double)(N + 1);
}

__global__ void __launch_bounds__(256) k_rank_sums(const double* __restrict__ rx,
                                                   const double* __restrict__ ry, int64_t N,
                                                   double* sums) {
  __shared__ double s_red[3][8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double a = 0, b = 0, c = 0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N;
       e += (int64_t)gridDim.x * blockDim.x) {
    a += rx[e] * rx[e];
    b += ry[e] * ry[e];
    c += rx[e] * ry[e];
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    a += __shfl_xor_sync(FULL_MASK, a, o);
    b += __shfl_xor_sync(FULL_MASK, b, o);
    c += __shfl_xor_sync(FULL_MASK, c, o);
  }
  if (lane == 0) { s_red[0][warp] = a; s_red[1][warp] = b; s_red[2][warp] = c; }
  __syncthreads();
  if (threadIdx.x < 3) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += s_red[threadIdx.x][w];
    atomicAdd(sums + threadIdx.x, s);
  }
}

__global__ void k_spearman_finish(const double* sums, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *out = sums[2] / sqrt(sums[0] * sums[1]);
}

__global__ void k_scale(double* v, double a, double b) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *v = a * *v + b;
}

}  // namespace gini

using namespace gini;

extern "C" void gini_set_cuda_error(cudaError_t e);

namespace {

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

struct CorrLayout {
  size_t sums = 0, keys = 0, vals = 0, ranks = 0, flags = 0, starts = 0, hist = 0, tmp = 0,
         total = 0;
};

CorrLayout corr_layout(int64_t n, bool spearman) {
  CorrLayout L;
  size_t off = WS_HEADER;
  L.sums = off;  off += al256(sizeof(double) * 16);
  if (spearman) {
    const int64_t P = n * (n - 1) / 2, nb = (P + SCAN_TILE - 1) / SCAN_TILE;
    L.keys = off;   off += al256(sizeof(unsigned long long) * (size_t)P) * 4;  // x, y, 2 buffers
    L.vals = off;   off += al256(sizeof(unsigned) * (size_t)P) * 4;
    L.ranks = off;  off += al256(sizeof(double) * (size_t)P) * 2;
    L.flags = off;  off += al256(sizeof(unsigned) * (size_t)P);
    L.starts = off; off += al256(sizeof(unsigned) * (size_t)P);
    L.hist = off;   off += al256(sizeof(unsigned) * 256 * (size_t)nb);
    L.tmp = off;    off += al256(sizeof(unsigned) * (size_t)scan_tmp_elems(std::max<int64_t>(256 * nb, P)));
  }
  L.total = off;
  return L;
}

int check_xy(const float* X, int64_t n, int64_t p, int64_t ldx, const float* Y, int k) {
  if (!X || !Y || n < 2 || p < 1 || ldx < p || k < 1 || k > 8) return GINI_EINVAL;
  return GINI_OK;
}

}  // namespace

extern "C" size_t gini_eval_workspace_size(int64_t n, int n_labels, int spearman) {
  if (n < 2) return 0;
  size_t s = WS_HEADER + al256(sizeof(double) * 16) + al256(sizeof(unsigned) * (size_t)std::max(n_labels, 1));
  return std::max(s, corr_layout(n, spearman != 0).total);
}

extern "C" int gini_neighbour_scores(const float* X_dev, int64_t n, int64_t p, int64_t ldx,
                                     const float* Y_dev, int k, const int* labels_dev, int k_trust,
                                     int k_nn, double* out_dev, void* ws, size_t ws_bytes,
                                     void* stream) {
  int st = check_xy(X_dev, n, p, ldx, Y_dev, k);
  if (st != GINI_OK || !out_dev || !ws) return GINI_EINVAL;
  if (ws_misaligned(ws)) return GINI_EINVAL;
  if (k_trust < 0 || k_nn < 0 || k_trust > EVAL_KMAX || k_nn > EVAL_KMAX) return GINI_EINVAL;
  if (k_trust >= n || k_nn >= n || (k_nn > 0 && !labels_dev)) return GINI_EINVAL;
  if (k_trust > 0 && 2 * n - 3 * k_trust - 1 <= 0) return GINI_EINVAL;
  if (ws_bytes < gini_eval_workspace_size(n, 1, 0)) return GINI_ENOMEM;
  cudaStream_t s = (cudaStream_t)stream;
  double* acc = reinterpret_cast<double*>(reinterpret_cast<char*>(ws) + WS_HEADER);
  cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(double) * 2, s);
  if (e != cudaSuccess) { gini_set_cuda_error(e); return GINI_ECUDA; }
  gini_count_launch(1);
  k_nbr_scores<<<(unsigned)std::min<int64_t>(n, 152 * 16), 256, 0, s>>>(
      X_dev, n, p, ldx, Y_dev, k, labels_dev, k_trust, k_nn, acc);
  // T = 1 - 2 sum / (n k (2n - 3k - 1)); NN = hits / (n knn)
  const double nn = (double)n;
  gini_count_launch(2);
  if (k_trust > 0)
    k_scale<<<1, 32, 0, s>>>(acc, -2.0 / (nn * k_trust * (2.0 * nn - 3.0 * k_trust - 1.0)), 1.0);
  else
    k_scale<<<1, 32, 0, s>>>(acc, 0.0, NAN);
  if (k_nn > 0)
    k_scale<<<1, 32, 0, s>>>(acc + 1, 1.0 / (nn * k_nn), 0.0);
  else
    k_scale<<<1, 32, 0, s>>>(acc + 1, 0.0, NAN);
  e = cudaMemcpyAsync(out_dev, acc, sizeof(double) * 2, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) { gini_set_cuda_error(e); return GINI_ECUDA; }
  return GINI_OK;
}

extern "C" int gini_silhouette(const float* Y_dev, int64_t n, int k, const int* labels_dev,
                               int n_labels, double* out_dev, void* ws, size_t ws_bytes,
                               void* stream) {
  if (!Y_dev || !labels_dev || !out_dev || !ws || n < 2 || k < 1 || k > 8 || n_labels < 1 ||
      n_labels > EVAL_CMAX)
    return GINI_EINVAL;
  if (ws_misaligned(ws)) return GINI_EINVAL;
  if (ws_bytes < gini_eval_workspace_size(n, n_labels, 0)) return GINI_ENOMEM;
  cudaStream_t s = (cudaStream_t)stream;
  char* base = reinterpret_cast<char*>(ws);
  double* acc = reinterpret_cast<double*>(base + WS_HEADER);
  unsigned* cnt = reinterpret_cast<unsigned*>(base + WS_HEADER + al256(sizeof(double) * 16));
  cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(double), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, sizeof(unsigned) * n_labels, s);
  if (e != cudaSuccess) { gini_set_cuda_error(e); return GINI_ECUDA; }
  const size_t smem = (size_t)256 * n_labels * sizeof(double);
  e = cudaFuncSetAttribute(k_silhouette, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) { gini_set_cuda_error(e); return GINI_ECUDA; }
  gini_count_launch(3);
  k_label_counts<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(labels_dev, n, n_labels, cnt,
                                                              reinterpret_cast<unsigned*>(ws));
  k_silhouette<<<(unsigned)std::min<int64_t>(n, 152 * 8), 256, smem, s>>>(Y_dev, n, k, labels_dev,
                                                                         n_labels, cnt, acc);
  k_scale<<<1, 32, 0, s>>>(acc, 1.0 / (double)n, 0.0);
  e = cudaMemcpyAsync(out_dev, acc, sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) { gini_set_cuda_error(e); return GINI_ECUDA; }
  return GINI_OK;
}

extern "C" int gini_distance_correlations(const float* X_dev, int64_t n, int64_t p, int64_t ldx,
                                          const float* Y_dev, int k, int spearman,
                                          double* out_dev, void* ws, size_t ws_bytes,
                                          void* stream) {
  int st = check_xy(X_dev, n, p, ldx, Y_dev, k);
  if (st != GINI_OK || !out_dev || !ws) return GINI_EINVAL;
  if (ws_misaligned(ws)) return GINI_EINVAL;
  if (n > 65535) return GINI_EINVAL;  // pair indices and counts stay below 2^31
  const CorrLayout L = corr_layout(n, spearman != 0);
  if (ws_bytes < L.total) return GINI_ENOMEM;
  cudaStream_t s = (cudaStream_t)stream;
  char* base = reinterpret_cast<char*>(ws);
  double* sums = reinterpret_cast<double*>(base + L.sums);  // 5 Pearson, 2 shifts, 3 rank sums
  const int64_t P = n * (n - 1) / 2, T = (n + 63) / 64;
  cudaError_t e = cudaMemsetAsync(sums, 0, sizeof(double) * 16, s);
  if (e != cudaSuccess) { gini_set_cuda_error(e); return GINI_ECUDA; }
  unsigned long long *kx = nullptr, *ky = nullptr, *kx2 = nullptr, *ky2 = nullptr;
  unsigned *vx = nullptr, *vy = nullptr, *vx2 = nullptr, *vy2 = nullptr;
  if (spearman) {
    const size_t kb = al256(sizeof(unsigned long long) * (size_t)P), vb = al256(sizeof(unsigned) * (size_t)P);
    kx = reinterpret_cast<unsigned long long*>(base + L.keys);
    ky = reinterpret_cast<unsigned long long*>(base + L.keys + kb);
    kx2 = reinterpret_cast<unsigned long long*>(base + L.keys + 2 * kb);
    ky2 = reinterpret_cast<unsigned long long*>(base + L.keys + 3 * kb);
    vx = reinterpret_cast<unsigned*>(base + L.vals);
    vy = reinterpret_cast<unsigned*>(base + L.vals + vb);
    vx2 = reinterpret_cast<unsigned*>(base + L.vals + 2 * vb);
    vy2 = reinterpret_cast<unsigned*>(base + L.vals + 3 * vb);
  }
  gini_count_launch(3);
  k_pair_shift<<<1, 32, 0, s>>>(X_dev, p, ldx, Y_dev, k, sums + 5);
  k_pair_dists<<<(unsigned)std::min<int64_t>(T * (T + 1) / 2, 152 * 8), 256, 0, s>>>(
      X_dev, n, p, ldx, Y_dev, k, T, sums + 5, sums, kx, ky, vx, vy);
  k_pearson_finish<<<1, 32, 0, s>>>(sums, (double)P, out_dev);
  if (!spearman) {
    gini_count_launch(1);
    k_scale<<<1, 32, 0, s>>>(out_dev + 1, 0.0, NAN);
  } else {
    const int64_t nb = (P + SCAN_TILE - 1) / SCAN_TILE;
    const size_t rb = al256(sizeof(double) * (size_t)P);
    double* rank[2] = {reinterpret_cast<double*>(base + L.ranks),
                       reinterpret_cast<double*>(base + L.ranks + rb)};
    unsigned* flags = reinterpret_cast<unsigned*>(base + L.flags);
    unsigned* starts = reinterpret_cast<unsigned*>(base + L.starts);
    unsigned* hist = reinterpret_cast<unsigned*>(base + L.hist);
    unsigned* tmp = reinterpret_cast<unsigned*>(base + L.tmp);
    unsigned long long* ka[2] = {kx, ky};
    unsigned long long* kb2[2] = {kx2, ky2};
    unsigned* va[2] = {vx, vy};
    unsigned* vb2[2] = {vx2, vy2};
    const unsigned g = (unsigned)((P + 255) / 256);
    for (int side = 0; side < 2; ++side) {
      unsigned long long *kin = ka[side], *kout = kb2[side];
      unsigned *vin = va[side], *vout = vb2[side];
      for (int shift = 0; shift < 64; shift += 8) {
        gini_count_launch(2);
        k_radix_hist<<<(unsigned)nb, 256, 0, s>>>(kin, P, shift, hist, nb);
        exclusive_scan(hist, 256 * nb, tmp, s);
        k_radix_scatter<<<(unsigned)nb, 256, 0, s>>>(kin, vin, P, shift, hist, nb, kout, vout);
        std::swap(kin, kout);
        std::swap(vin, vout);
      }
      // 8 passes: the sorted keys are back in the first buffer
      gini_count_launch(1);
      k_run_heads<<<g, 256, 0, s>>>(kin, P, flags);
      exclusive_scan(flags, P, tmp, s);
      gini_count_launch(2);
      k_run_starts<<<g, 256, 0, s>>>(kin, P, flags, starts);
      k_midranks<<<g, 256, 0, s>>>(kin, P, flags, starts, vin, rank[side]);
    }
    gini_count_launch(2);
    k_rank_sums<<<(unsigned)std::min<int64_t>((P + 255) / 256, 152 * 8), 256, 0, s>>>(
        rank[0], rank[1], P, sums + 8);
    k_spearman_finish<<<1, 32, 0, s>>>(sums + 8, out_dev + 1);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) { gini_set_cuda_error(e); return GINI_ECUDA; }
  return GINI_OK;
}
