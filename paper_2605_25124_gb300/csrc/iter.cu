// Kruskal stress and its adjoint for an embedding Y (n x k) under the Gini
// pseudo-distance, and the fixed-step gradient-descent fit (Section IV-B;
// Algorithm 1, "Run MDS").
//
//   d_ij = Dbar_{G,nu}(y_i, y_j) = sum_c z_c T[2R_c - 2],  z = y_i - y_j,
//          T = (k/2) W_{k,nu}, R_c the midrank of z_c among the k components;
//   r_ij = d_ij - delta_ij,  S = sum_{i<j} r_ij^2 / sum_delta2;
//   dS/dy_i = 2/sum_delta2 * sum_{j != i} r_ij T[2R(y_i - y_j) - 2]  (ranks fixed).
//
// Ranks of z are decided exactly: z_a < z_b  <=>  (y_ia - y_ib) < (y_ja - y_jb),
// and each point carries its within-point differences y_ia - y_ib as exact
// TwoSum pairs (computed once per iteration), so the comparison of two points
// is exact.  For k = 2 this reduces to u_i = y_i0 - y_i1 and
//   d_ij = 2^{1-nu} |u_i - u_j|,  dd_ij/dy_i = 2^{1-nu} sign(u_i - u_j) (1, -1),
// with sign 0 at an exact tie (W(3/2) = 0 for k = 2).
//
// Two forms:
//   plain  (GINI_LAYOUT_FULL, F32): a forward kernel over i<j for S, then an
//          adjoint kernel over all ordered pairs for dS/dY (each recomputes d).
//   fused  (GINI_LAYOUT_TILED, any dtype): one pass over the stored triangle of
//          B x B tiles; each element feeds the stress, its row's gradient and
//          its column's gradient (d_ji = d_ij, antisymmetric derivative).
#include <math.h>

#include <algorithm>
#include <atomic>

#define GINI_FILE_ID 2  // site numbers of the debug index checks
#include "common.cuh"
#include "pipe.cuh"

namespace gini {

constexpr int KMAX = 8;
constexpr int FUSED_THREADS = 256;  // 8 warps; a warp owns 16 rows of a 128 x 128 tile
// Stress of one pass: every CTA stores its FP64 partial in its own slot, and
// the slots are summed in index order afterwards, so the stress does not
// depend on the order the CTAs finish in.  Grids are capped at this count.
constexpr int STRESS_SLOTS = 1024;

struct PairTab {
  float c2;               // k = 2: 2^{1-nu}
  float w[2 * KMAX - 1];  // (k/2) W_{k,nu}(R) at 2R - 2 = 0 .. 2k - 2
};

struct IterParams {
  int64_t n;
  const float2* P;  // per point: k = 2 -> u_i as (hi, lo); else the k(k-1)/2 pairs y_ia - y_ib
  const float* Y;   // n x k (generic-k kernels read coordinates)
  const float4* Y4; // k = 3: y as (y0, y1, y2, 0), padded to whole tiles with zeros (else null)
  const void* delta;
  int64_t ldd;
  const float* col_scale;
  int64_t tiles;
  int64_t plane;
  float* h;          // k = 2: n scalars sum_j r_ij sign; else n x k sums of r_ij T
  double* stress;    // STRESS_SLOTS FP64 slots of this pass (slot = CTA index)
  // Deterministic mode (else null): per-tile gradient partials instead of
  // atomics into h.  Tile t's row sums at part[(2t) 128 kp ..], its column sums
  // at part[(2t+1) 128 kp ..], kp = 1 on the scalar k = 2 path, else k
  // components per point; k_det_reduce sums them per point in a fixed order.
  float* part;
  PairTab tab;
  unsigned* err;
  int metric;        // GINI_METRIC_GINI or GINI_METRIC_EUCLID
  int loss;          // GINI_LOSS_KRUSKAL or GINI_LOSS_SAMMON
};

// Gini distance with Kruskal stress and k = 2 takes the scalar fast path
// (one accumulator per point, the gradient is c2 h_i (1, -1)).
__host__ __device__ __forceinline__ bool scalar2_path(int k, int metric, int loss) {
  return k == 2 && metric == GINI_METRIC_GINI && loss == GINI_LOSS_KRUSKAL;
}

// Euclidean embedding distance ||y_i - y_j|| and its derivative in y_i
// ((y_i - y_j)/d, taken as 0 at d = 0).
template <int K>
__device__ __forceinline__ float pair_euclid(const float* yi, const float* yj, float (&dw)[K]) {
  float s = 0.f;
#pragma unroll
  for (int a = 0; a < K; ++a) {
    dw[a] = yi[a] - yj[a];
    s = fmaf(dw[a], dw[a], s);
  }
  const float d = sqrtf(s);
  const float inv = d > 0.f ? 1.f / d : 0.f;
#pragma unroll
  for (int a = 0; a < K; ++a) dw[a] *= inv;
  return d;
}

// Loss terms for one pair: stress term and gradient weight of dd/dy.
//   Kruskal: (d - delta)^2 and (d - delta)
//   Sammon:  (d - delta)^2 / delta and (d - delta) / delta, pairs with delta = 0
//            excluded
__device__ __forceinline__ void loss_terms(int loss, float d, float delta, float& sterm,
                                           float& gw) {
  const float r = d - delta;
  if (loss == GINI_LOSS_SAMMON) {
    const float w = delta > 0.f ? 1.f / delta : 0.f;
    gw = r * w;
    sterm = r * gw;
  } else {
    gw = r;
    sterm = r * r;
  }
}

// ------------------------------------------------------------ point prep ---

template <int K>
__global__ void k_prep(const float* __restrict__ Y, int64_t n, int64_t npad,
                       float2* __restrict__ P, float4* __restrict__ Y4, unsigned* err) {
  constexpr int NP = K * (K - 1) / 2;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool bad = false;
  if (i >= n && i < npad) {
#pragma unroll
    for (int p = 0; p < NP; ++p) P[i * NP + p] = make_float2(0.f, 0.f);
    if (K == 3 && Y4) Y4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  if (i < n) {
    float y[K];
#pragma unroll
    for (int c = 0; c < K; ++c) {
      y[c] = Y[i * K + c];
      bad |= !isfinite(y[c]);
    }
    int p = 0;
#pragma unroll
    for (int a = 0; a < K; ++a)
#pragma unroll
      for (int b = a + 1; b < K; ++b) P[i * NP + (p++)] = point_pair(y[a], y[b]);
    if (K == 3 && Y4) Y4[i] = make_float4(y[0], y[1], y[K - 1], 0.f);
  }
  if (__any_sync(FULL_MASK, bad) && (threadIdx.x & 31) == 0) raise_error(err, ERR_NONFINITE);
}

// ------------------------------------------------------- pair functions ---

// k = 2: residual r = 2^{1-nu}|u_i - u_j| - delta and t = r * sign(u_i - u_j).
__device__ __forceinline__ void pair2(float2 ui, float2 uj, float c2, float delta, float& r,
                                      float& t) {
  const float dh = ui.x - uj.x, dl = ui.y - uj.y;  // dl scaled by 2^24
  r = fmaf(c2, fabsf(fmaf(dl, LO_UNSCALE, dh)), -delta);
  const float sg = (dh != 0.f) ? dh : dl;  // exact sign of u_i - u_j
  // r * sign(sg): flip r's sign bit by sg's; an exact tie contributes 0
  const float rs = __int_as_float(__float_as_int(r) ^ (__float_as_int(sg) & 0x80000000));
  t = (sg == 0.f) ? 0.f : rs;
}

// Generic k: distance and dd/dy_i (= T[2R_c - 2]) with exact rank comparisons.
template <int K>
__device__ __forceinline__ float pair_k(const float* yi, const float* yj, const float2* Pi,
                                        const float2* Pj, const float* w, float (&dw)[K]) {
  int r2[K];
#pragma unroll
  for (int a = 0; a < K; ++a) r2[a] = 2;
  int p = 0;
#pragma unroll
  for (int a = 0; a < K; ++a)
#pragma unroll
    for (int b = a + 1; b < K; ++b) {
      const int c = exact_cmp(Pi[p], Pj[p]);  // sign(z_a - z_b)
      r2[a] += 1 + c;
      r2[b] += 1 - c;
      ++p;
    }
  float d = 0.f;
#pragma unroll
  for (int a = 0; a < K; ++a) {
    dw[a] = w[r2[a] - 2];
    d = fmaf(yi[a] - yj[a], dw[a], d);
  }
  return d;
}

// Exact sign of (hi_i - hi_j) + (lo_i - lo_j) for point pairs (lo scaled by
// 2^24), as -1, 0 or 1 on the FMA pipe: a = fma(dh, 2^88, dl') has the sign
// that decides (dl cannot outweigh a non-zero dh; a = dl' when dh = 0), and
// 2^126 takes any non-zero a to >= 2 before the saturations.
__device__ __forceinline__ float exact_sign(float2 pi, float2 pj) {
  const float dh = pi.x - pj.x, dl = pi.y - pj.y;  // dl scaled by 2^24
  const float a = fmaf(dh, SIGN_HI, dl);
  return __saturatef(a * SIGN_SAT) - __saturatef(-a * SIGN_SAT);
}

// k = 3: with the midrank offsets x_c = R_c - 2 in {0, +-1/2, +-1} (from the
// three exact pairwise signs) the table value (3/2) W(R_c) is an odd function
// of x_c, so T(x) = x (A + B x^2) with T(1) = w[4] and T(1/2) = w[3] -- exact
// at ties too, and no table lookups.
template <>
__device__ __forceinline__ float pair_k<3>(const float* yi, const float* yj, const float2* Pi,
                                           const float2* Pj, const float* w, float (&dw)[3]) {
  const float s01 = exact_sign(Pi[0], Pj[0]);  // sign(z_0 - z_1)
  const float s02 = exact_sign(Pi[1], Pj[1]);
  const float s12 = exact_sign(Pi[2], Pj[2]);
  const float t1 = w[4], th = w[3];
  const float A = (8.f * th - t1) * (1.f / 3.f), B = (4.f * t1 - 8.f * th) * (1.f / 3.f);
  const float x[3] = {0.5f * (s01 + s02), 0.5f * (s12 - s01), -0.5f * (s02 + s12)};
  float d = 0.f;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    dw[c] = x[c] * fmaf(B, x[c] * x[c], A);
    d = fmaf(yi[c] - yj[c], dw[c], d);
  }
  return d;
}

// ------------------------------------------------------------ plain form ---

// One warp per row i.  FWD: S over j > i.  !FWD: h_i over all j != i.
template <int K, bool FWD>
__global__ void __launch_bounds__(256) k_full(const IterParams Q) {
  constexpr int NP = K * (K - 1) / 2;
  __shared__ float s_w[2 * KMAX - 1];
  __shared__ double s_red[8];
  if (threadIdx.x < 2 * KMAX - 1) s_w[threadIdx.x] = Q.tab.w[threadIdx.x];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float* D = reinterpret_cast<const float*>(Q.delta);
  double Sd = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * 8 + warp; i < Q.n; i += (int64_t)gridDim.x * 8) {
    if (!(GINI_IDX_OK(Q.err, Q.n - 1, Q.ldd))) break;  // (debug builds) rows of the n x ldd matrix
    float yi[K];
    float2 Pi[NP];
#pragma unroll
    for (int c = 0; c < K; ++c) yi[c] = Q.Y[i * K + c];
#pragma unroll
    for (int p = 0; p < NP; ++p) Pi[p] = Q.P[i * NP + p];
    float acc[K];
#pragma unroll
    for (int c = 0; c < K; ++c) acc[c] = 0.f;
    float S = 0.f, Sc = 0.f;  // compensated FP32 sum over the row
    const bool fast2 = scalar2_path(K, Q.metric, Q.loss);
    if (K == 2 && fast2) {
      // Gini metric, Kruskal loss, k = 2: its own loop, so the streaming loads
      // of several columns can be in flight at once
#pragma unroll 4
      for (int64_t j = (FWD ? i + 1 : 0) + lane; j < Q.n; j += 32) {
        const float dl = __ldcs(D + i * Q.ldd + j);
        float r, t;
        pair2(Pi[0], Q.P[j], Q.tab.c2, dl, r, t);
        if (FWD) {
          const float y = fmaf(r, r, -Sc);
          const float tsum = S + y;
          Sc = (tsum - S) - y;
          S = tsum;
        } else if (j != i) {
          acc[0] += t;
        }
      }
    } else {
      for (int64_t j = (FWD ? i + 1 : 0) + lane; j < Q.n; j += 32) {
        const float dl = __ldcs(D + i * Q.ldd + j);
        float yj[K], dw[K];
#pragma unroll
        for (int c = 0; c < K; ++c) yj[c] = Q.Y[j * K + c];
        float d;
        if (Q.metric == GINI_METRIC_EUCLID) {
          d = pair_euclid<K>(yi, yj, dw);
        } else {
          float2 Pj[NP];
#pragma unroll
          for (int p = 0; p < NP; ++p) Pj[p] = Q.P[j * NP + p];
          d = pair_k<K>(yi, yj, Pi, Pj, s_w, dw);
        }
        float sterm, gw;
        loss_terms(Q.loss, d, dl, sterm, gw);
        if (FWD) {
          const float y = sterm - Sc;
          const float tsum = S + y;
          Sc = (tsum - S) - y;
          S = tsum;
        } else if (j != i) {
#pragma unroll
          for (int c = 0; c < K; ++c) acc[c] = fmaf(gw, dw[c], acc[c]);
        }
      }
    }
    if (FWD) {
      Sd += (double)S - (double)Sc;
    } else {
#pragma unroll
      for (int c = 0; c < K; ++c) {
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) acc[c] += __shfl_xor_sync(FULL_MASK, acc[c], o);
      }
      if (lane == 0) {
        if (K == 2 && fast2) Q.h[i] = acc[0];
        else
#pragma unroll
          for (int c = 0; c < K; ++c) Q.h[i * K + c] = acc[c];
      }
    }
  }
  if (FWD) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) Sd += __shfl_xor_sync(FULL_MASK, Sd, o);
    if (lane == 0) s_red[warp] = Sd;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < 8; ++w) s += s_red[w];
      Q.stress[blockIdx.x] = s;
    }
  }
}

// ------------------------------------------------------------ fused form ---

// Loads 4 consecutive stored dissimilarities (columns 4*lane .. 4*lane+3 of a
// tile row) and widens them to float.
template <int DT>
__device__ __forceinline__ void load4(const IterParams& Q, int64_t off, float (&d)[4],
                                      const float (&sc)[4]) {
  if (!(GINI_IDX_OK(Q.err, off + 3, Q.plane))) {  // (debug builds) inside the plane
    d[0] = d[1] = d[2] = d[3] = 0.f;
    return;
  }
  if (DT == GINI_F32) {
    const float4 v = __ldcs(reinterpret_cast<const float4*>(reinterpret_cast<const float*>(Q.delta) + off));
    d[0] = v.x; d[1] = v.y; d[2] = v.z; d[3] = v.w;
  } else if (DT == GINI_BF16 || DT == GINI_BF16X2) {
    const uint16_t* base = reinterpret_cast<const uint16_t*>(Q.delta);
    const uint2 h = __ldcs(reinterpret_cast<const uint2*>(base + off));
    d[0] = bf16_bits_to_float(h.x & 0xffffu);
    d[1] = __uint_as_float(h.x & 0xffff0000u);
    d[2] = bf16_bits_to_float(h.y & 0xffffu);
    d[3] = __uint_as_float(h.y & 0xffff0000u);
    if (DT == GINI_BF16X2) {
      const uint2 l = __ldcs(reinterpret_cast<const uint2*>(base + Q.plane + off));
      d[0] += bf16_bits_to_float(l.x & 0xffffu);
      d[1] += __uint_as_float(l.x & 0xffff0000u);
      d[2] += bf16_bits_to_float(l.y & 0xffffu);
      d[3] += __uint_as_float(l.y & 0xffff0000u);
    }
  } else {  // GINI_FP8E4M3
    const uint32_t q = __ldcs(reinterpret_cast<const unsigned int*>(
        reinterpret_cast<const uint8_t*>(Q.delta) + off));
    const __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(q & 0xffffu), __NV_E4M3);
    const __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(q >> 16), __NV_E4M3);
    const float2 a = __half22float2(__half2(lo));
    const float2 b = __half22float2(__half2(hi));
    d[0] = a.x * sc[0]; d[1] = a.y * sc[1]; d[2] = b.x * sc[2]; d[3] = b.y * sc[3];
  }
}

// Sums v over the CTA in a fixed order and stores it in the CTA's stress slot.
__device__ __forceinline__ void block_store_stress(double v, double* slots) {
  __shared__ double s_red[FUSED_THREADS / 32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(FULL_MASK, v, o);
  if (lane == 0) s_red[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < FUSED_THREADS / 32; ++w) s += s_red[w];
    slots[blockIdx.x] = s;
  }
}

// k = 2 fused kernel, fed by a bulk-copy pipeline.
//
// CTA = 8 consumer warps + 1 producer warp.  A CTA owns a contiguous range of
// tiles (so consecutive tiles usually share the tile-row I).  Each tile is
// streamed as two chunks of 64 rows x 128 columns (one or two planes); the
// producer's elected lane keeps S chunks in flight with cp.async.bulk into a
// shared-memory ring (full/empty mbarriers, bounded waits).  Consumer warp w
// takes rows w*8 .. w*8+7 of each chunk, lane l columns 4l .. 4l+3.
//
// Per element: r = 2^{1-nu}|u_i - u_j| - delta, S += r^2, t = r sign(u_i - u_j)
// with the exact sign of the TwoSum pairs; t adds to row i and subtracts from
// column j.  Row sums stay in registers while the tile-row does not change;
// column sums of a tile meet in shared memory behind one named barrier.
constexpr int CONSUMER_WARPS = 8;
constexpr int PIPE_THREADS = (CONSUMER_WARPS + 1) * 32;
constexpr int CHUNK_ROWS = 64;

template <int DT>
struct PipeCfg {
  static constexpr int planes = DT == GINI_BF16X2 ? 2 : 1;
  static constexpr int esize = DT == GINI_F32 ? 4 : (DT == GINI_FP8E4M3 ? 1 : 2);
  static constexpr int plane_bytes = CHUNK_ROWS * TILE * esize;
  // after the planes: the chunk's 64 row points and the tile's 128 column
  // points (u_i as (hi, lo) pairs), copied with the dissimilarities
  static constexpr int urow_off = planes * plane_bytes;
  static constexpr int ucol_off = urow_off + CHUNK_ROWS * 8;
  static constexpr int stage_bytes = ucol_off + TILE * 8;
  // Several CTAs per SM (the consumers are latency-bound, so more warps help):
  //  - narrow forms (16-bit, 8-bit tiles): four, with ~40 KB of stages + 8.5 KB
  //    static each (BF16: two stages, FP8: four) at 56 registers;
  //  - wide forms (FP32, BF16 hi+lo): three, with two 33.5 KB stages + 4.4 KB
  //    static, the column slices single-buffered behind a second named
  //    barrier per tile.  Bytes in flight per SM stay at six 32 KB chunks.
  static constexpr bool wide = DT == GINI_F32 || DT == GINI_BF16X2;
  static constexpr int budget = 40 * 1024;
  static constexpr int stages_raw = budget / stage_bytes;
  static constexpr int stages = wide ? 2 : (stages_raw > 8 ? 8 : stages_raw);
  static constexpr int smem = stages * stage_bytes;
  static constexpr int colbufs = wide ? 1 : 2;  // column-slice buffers
  // held to in registers too: 65536 / (3 x 288) = 75 per thread (72 used),
  // 65536 / (4 x 288) = 56 (56 used, a 4-byte spill in the gradient body)
  static constexpr int min_ctas = wide ? 3 : 4;
};

// Sums a[0..7] over the 32 lanes; lane l returns the total of entry
// rev3(l & 7).
__device__ __forceinline__ float reduce8(float (&a)[8], int lane) {
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    const int h = 4 >> s, x = 1 << s;
    const bool upper = (lane & x) != 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (i < h) {
        const float send = upper ? a[i] : a[i + h];
        const float keep = upper ? a[i + h] : a[i];
        a[i] = keep + __shfl_xor_sync(FULL_MASK, send, x);
      }
    }
  }
  float v = a[0] + __shfl_xor_sync(FULL_MASK, a[0], 8);
  return v + __shfl_xor_sync(FULL_MASK, v, 16);
}

__device__ __forceinline__ int rev3(int l) { return ((l & 1) << 2) | (l & 2) | ((l & 4) >> 2); }

template <int DT>
__device__ __forceinline__ void load4_smem(const unsigned char* stage, int rr, int lane,
                                           float (&d)[4], const float (&sc)[4]) {
  using C = PipeCfg<DT>;
  const int off = rr * TILE + 4 * lane;  // element offset inside a plane
  if (DT == GINI_F32) {
    const float4 v = *reinterpret_cast<const float4*>(stage + off * 4);
    d[0] = v.x; d[1] = v.y; d[2] = v.z; d[3] = v.w;
  } else if (DT == GINI_BF16 || DT == GINI_BF16X2) {
    const uint2 h = *reinterpret_cast<const uint2*>(stage + off * 2);
    d[0] = bf16_bits_to_float(h.x & 0xffffu);
    d[1] = __uint_as_float(h.x & 0xffff0000u);
    d[2] = bf16_bits_to_float(h.y & 0xffffu);
    d[3] = __uint_as_float(h.y & 0xffff0000u);
    if (DT == GINI_BF16X2) {
      const uint2 l = *reinterpret_cast<const uint2*>(stage + C::plane_bytes + off * 2);
      d[0] += bf16_bits_to_float(l.x & 0xffffu);
      d[1] += __uint_as_float(l.x & 0xffff0000u);
      d[2] += bf16_bits_to_float(l.y & 0xffffu);
      d[3] += __uint_as_float(l.y & 0xffff0000u);
    }
  } else {
    const uint32_t q = *reinterpret_cast<const uint32_t*>(stage + off);
    const __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(q & 0xffffu), __NV_E4M3);
    const __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(q >> 16), __NV_E4M3);
    const float2 a = __half22float2(__half2(lo));
    const float2 b = __half22float2(__half2(hi));
    d[0] = a.x * sc[0]; d[1] = a.y * sc[1]; d[2] = b.x * sc[2]; d[3] = b.y * sc[3];
  }
}

// One chunk row block of a consumer warp: 8 rows x 4 columns per lane, two
// columns per packed f32x2 instruction.  With s = u_i - u_j and
// sigma = sign(s) in {-1, 0, 1} (exact, see below): |s| = s sigma, the
// residual r = c2 |s| - delta and t = r sigma.  The kernel carries
// r' = -r = delta - c2 |s| and t' = -t, so no negations are needed:
// S += r'^2, the row sum collects t' (negated when flushed) and the column
// sum, which needs -t, collects t' directly.
//   sigma: with the point pairs' lo parts scaled by 2^24 (point_pair),
//   a = fma(dh, 2^88, dl') has the sign of u_i - u_j (dl cannot outweigh a
//   non-zero dh; a = dl' exactly when dh = 0), and sat(a 2^126 + 1/2) maps it
//   to exactly 0, 1/2 or 1 = (sigma + 1) / 2.
//   |s|: s = fma(dl', 2^-24, dh) has the sign 0 or sigma, so |s| = s sigma;
//   it is taken with an AND on the ALU pipe.  The lo parts matter here: near
//   a converged fit the residual is orders of magnitude below delta, and
//   dropping them (an error up to 2^-24 |u| in d) moved the gradient by 5e-4.
//   t' = r' sigma is exact, so the row and column sums take it in one FMA.
template <int DT, bool GRAD, bool MASKED>
__device__ __forceinline__ void chunk_compute(const unsigned char* stage, int rbase, int lane,
                                              const float2 (&nuh)[2], const float2 (&nul)[2],
                                              const float2* urow, float c2, const float (&sc)[4],
                                              float2& S2, float2 (&col2)[2], float (&rowv)[8],
                                              int64_t gi0, int64_t gj0, int64_t n, bool diag,
                                              int rl0) {
  const float2 khi = make_float2(SIGN_HI, SIGN_HI);
  const float2 kun = make_float2(LO_UNSCALE, LO_UNSCALE);
  const float2 m1 = make_float2(-1.f, -1.f);
  const float2 k2 = make_float2(2.f, 2.f);
  const float2 nc2 = make_float2(-c2, -c2);
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const float2 ur = urow[rbase + q];  // same address in every lane: broadcast
    const float2 uh2 = make_float2(ur.x, ur.x), ul2 = make_float2(ur.y, ur.y);
    float dl[4];
    load4_smem<DT>(stage, rbase + q, lane, dl, sc);
    float2 row2 = make_float2(0.f, 0.f);
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      const float2 d2 = make_float2(dl[2 * p], dl[2 * p + 1]);
      const float2 dh = __fadd2_rn(uh2, nuh[p]);
      const float2 dlo = __fadd2_rn(ul2, nul[p]);  // scaled by 2^24
      const float2 s2 = __ffma2_rn(dlo, kun, dh);
      const float2 a2 = __ffma2_rn(dh, khi, dlo);
      // sp = (sigma + 1) / 2 in {0, 1/2, 1}: one saturating FMA per column
      const float2 sp = make_float2(__saturatef(fmaf(a2.x, SIGN_SAT, 0.5f)),
                                    __saturatef(fmaf(a2.y, SIGN_SAT, 0.5f)));
      const float2 sig = __ffma2_rn(sp, k2, m1);  // 2 sp - 1
      float2 rp = __ffma2_rn(nc2, abs2_alu(s2), d2);  // r' = delta - c2 |s|
      if (MASKED) {
        const int rl = rl0 + q, cl = 4 * lane + 2 * p;
        const bool ok0 = (gi0 + q < n) && (gj0 + 2 * p < n) && (!diag || rl < cl);
        const bool ok1 = (gi0 + q < n) && (gj0 + 2 * p + 1 < n) && (!diag || rl < cl + 1);
        rp.x = ok0 ? rp.x : 0.f;
        rp.y = ok1 ? rp.y : 0.f;
      }
      S2 = __ffma2_rn(rp, rp, S2);
      if (GRAD) {  // t' = r' sigma = -t
        row2 = __ffma2_rn(rp, sig, row2);
        col2[p] = __ffma2_rn(rp, sig, col2[p]);
      }
    }
    rowv[q] = -(row2.x + row2.y);
  }
}

template <int DT, bool GRAD>
__global__ void __launch_bounds__(PIPE_THREADS, PipeCfg<DT>::min_ctas)
k_fused2(const IterParams Q, int64_t ntiles) {
  using C = PipeCfg<DT>;
  constexpr int S = C::stages;
  extern __shared__ __align__(128) unsigned char s_stage[];
  __shared__ __align__(8) uint64_t bar_full[S];
  __shared__ __align__(8) uint64_t bar_empty[S];
  __shared__ float s_colw[C::colbufs][CONSUMER_WARPS][TILE];
  __shared__ double s_red[CONSUMER_WARPS];
  __shared__ int s_abort;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t t_begin = ntiles * blockIdx.x / gridDim.x;
  const int64_t t_end = ntiles * (blockIdx.x + 1) / gridDim.x;
  const int nchunks = (int)(t_end - t_begin) * 2;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&bar_full[s], 1);
      mbar_init(&bar_empty[s], CONSUMER_WARPS);
    }
    s_abort = 0;
    mbar_init_fence();
  }
  __syncthreads();
  volatile int* abort = &s_abort;

  if (warp == CONSUMER_WARPS) {
    // ---------------------------------------------------------- producer --
    if (lane == 0) {
      const unsigned char* base = reinterpret_cast<const unsigned char*>(Q.delta);
      int issued = 0;
      int I = 0, J = 0;
      if (nchunks) tile_decode(t_begin, Q.tiles, I, J);
      for (int c = 0; c < nchunks; ++c) {
        const int s = c % S, use = c / S;
        if (use > 0 && !mbar_wait_bounded(&bar_empty[s], (use - 1) & 1, abort)) {
          raise_error(Q.err, ERR_TIMEOUT);
          *abort = 1;
          break;
        }
        const int64_t t = t_begin + c / 2;
        const int h = c & 1;
        if (h == 0 && c > 0) tile_next(I, J, Q.tiles);
        const int64_t eoff = t * (int64_t)(TILE * TILE) + (int64_t)h * CHUNK_ROWS * TILE;
        unsigned char* dst = s_stage + s * C::stage_bytes;
        // (debug builds) the chunk inside the plane, the tile's points inside
        // the padded point array; a failed check completes the stage without
        // copies, so the consumers compute on stale data but never wait
        [[maybe_unused]] const int64_t padded = Q.tiles * TILE;
        if (GINI_IDX_OK(Q.err, eoff + CHUNK_ROWS * TILE - 1, ntiles * (TILE * TILE)) &&
            GINI_IDX_OK(Q.err, t, ntiles) &&
            GINI_IDX_OK(Q.err, (int64_t)I * TILE + h * CHUNK_ROWS + CHUNK_ROWS - 1, padded) &&
            GINI_IDX_OK(Q.err, (int64_t)J * TILE + TILE - 1, padded)) {
          mbar_arrive_expect_tx(&bar_full[s], C::stage_bytes);
          bulk_copy_g2s(dst, base + eoff * C::esize, C::plane_bytes, &bar_full[s]);
          if (C::planes == 2)
            bulk_copy_g2s(dst + C::plane_bytes, base + (Q.plane + eoff) * C::esize, C::plane_bytes,
                          &bar_full[s]);
          // point arrays are padded to whole tiles, so these stay in bounds
          bulk_copy_g2s(dst + C::urow_off, Q.P + (int64_t)I * TILE + h * CHUNK_ROWS,
                        CHUNK_ROWS * 8, &bar_full[s]);
          bulk_copy_g2s(dst + C::ucol_off, Q.P + (int64_t)J * TILE, TILE * 8, &bar_full[s]);
        } else {
          mbar_arrive(&bar_full[s]);
        }
        issued = c + 1;
      }
      // Copies still in flight must land before this CTA's shared memory can
      // be released (normally the consumers have waited for all of them).
      for (int c = (issued > S ? issued - S : 0); c < issued; ++c)
        mbar_wait_bounded(&bar_full[c % S], (c / S) & 1, nullptr);
    }
    return;
  }

  // ------------------------------------------------------------ consumers --
  const float c2 = Q.tab.c2;
  const int64_t n = Q.n;
  float Ssum = 0.f, Scomp = 0.f;  // compensated sum of the per-tile FP32 partials
  float rowacc0 = 0.f, rowacc1 = 0.f;  // lane l < 8: rows rev3(l) of chunk 0 and 1
  int curI = -1;
  float2 nuh[2], nul[2];               // -u of the lane's 4 columns, packed by pairs
  float sc[4] = {1.f, 1.f, 1.f, 1.f};
  float2 col2[2];
  float2 S2 = make_float2(0.f, 0.f);
  int I = 0, J = 0;
  if (nchunks) tile_decode(t_begin, Q.tiles, I, J);
  for (int c = 0; c < nchunks; ++c) {
    const int s = c % S, h = c & 1;
    if (h == 0) {
      if (c > 0) tile_next(I, J, Q.tiles);
      if (GRAD && I != curI) {
        if (!Q.part && curI >= 0 && lane < 8) {
          const int64_t gi = (int64_t)curI * TILE + warp * 8 + rev3(lane);
          if (gi < n) atomicAdd(Q.h + gi, rowacc0);
          if (gi + CHUNK_ROWS < n) atomicAdd(Q.h + gi + CHUNK_ROWS, rowacc1);
        }
        rowacc0 = rowacc1 = 0.f;
        curI = I;
      }
      if (DT == GINI_FP8E4M3) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int64_t gj = (int64_t)J * TILE + 4 * lane + q;
          sc[q] = Q.col_scale[gj < n ? gj : n - 1];
        }
      }
#pragma unroll
      for (int p = 0; p < 2; ++p) col2[p] = make_float2(0.f, 0.f);
    }
    const int rl0 = h * CHUNK_ROWS + warp * 8;
    const int64_t gi0 = (int64_t)I * TILE + rl0;
    const int64_t gj0 = (int64_t)J * TILE + 4 * lane;
    const bool masked = (I == J) || ((int64_t)I * TILE + TILE > n) || ((int64_t)J * TILE + TILE > n);

    if (!mbar_wait_bounded(&bar_full[s], (c / S) & 1, abort)) {
      raise_error(Q.err, ERR_TIMEOUT);
      *abort = 1;
    }
    const unsigned char* stage = s_stage + s * C::stage_bytes;
    const float2* urow = reinterpret_cast<const float2*>(stage + C::urow_off);
    {
      const float4* ucol = reinterpret_cast<const float4*>(stage + C::ucol_off) + 2 * lane;
      const float4 a = ucol[0], b = ucol[1];  // columns 4l, 4l+1 | 4l+2, 4l+3 as (hi, lo)
      nuh[0] = make_float2(-a.x, -a.z);
      nul[0] = make_float2(-a.y, -a.w);
      nuh[1] = make_float2(-b.x, -b.z);
      nul[1] = make_float2(-b.y, -b.w);
    }
    float rowv[8];
    if (masked)
      chunk_compute<DT, GRAD, true>(stage, warp * 8, lane, nuh, nul, urow, c2, sc, S2, col2,
                                    rowv, gi0, gj0, n, I == J, rl0);
    else
      chunk_compute<DT, GRAD, false>(stage, warp * 8, lane, nuh, nul, urow, c2, sc, S2, col2,
                                     rowv, gi0, gj0, n, false, rl0);
    __syncwarp();
    if (lane == 0) mbar_arrive(&bar_empty[s]);
    if (h == 1) {  // fold the FP32 partial of each tile (Kahan)
      const float y = (S2.x + S2.y) - Scomp;
      const float tsum = Ssum + y;
      Scomp = (tsum - Ssum) - y;
      Ssum = tsum;
      S2 = make_float2(0.f, 0.f);
    }
    if (GRAD) {
      const float rs = reduce8(rowv, lane);
      if (h) rowacc1 += rs;
      else rowacc0 += rs;
      if (h == 1) {
        const int64_t tcur = t_begin + (c >> 1);
        if (Q.part && lane < 8 &&  // deterministic: this tile's row sums
            GINI_IDX_OK(Q.err, (2 * tcur) * TILE + warp * 8 + rev3(lane) + CHUNK_ROWS,
                        2 * ntiles * TILE)) {
          float* rp = Q.part + (2 * tcur) * TILE + warp * 8 + rev3(lane);
          rp[0] = rowacc0;
          rp[CHUNK_ROWS] = rowacc1;
          rowacc0 = rowacc1 = 0.f;
        }
        const int cb = (c >> 1) % C::colbufs;
        float* cw = s_colw[cb][warp];
        *reinterpret_cast<float4*>(cw + 4 * lane) =
            make_float4(col2[0].x, col2[0].y, col2[1].x, col2[1].y);
        named_bar_sync(CONSUMER_WARPS * 32);
        if (threadIdx.x < TILE) {
          float v = 0.f;
#pragma unroll
          for (int w = 0; w < CONSUMER_WARPS; ++w) v += s_colw[cb][w][threadIdx.x];
          const int64_t gj = (int64_t)J * TILE + threadIdx.x;
          if (Q.part) {
            if (GINI_IDX_OK(Q.err, (2 * tcur + 1) * TILE + threadIdx.x, 2 * ntiles * TILE))
              Q.part[(2 * tcur + 1) * TILE + threadIdx.x] = v;
          } else if (gj < n) {
            atomicAdd(Q.h + gj, v);
          }
        }
        // one slice buffer: every consumer has read it before the next tile writes
        if (C::colbufs == 1) named_bar_sync(CONSUMER_WARPS * 32);
      }
    }
  }
  if (GRAD && !Q.part && curI >= 0 && lane < 8) {
    const int64_t gi = (int64_t)curI * TILE + warp * 8 + rev3(lane);
    if (gi < n) atomicAdd(Q.h + gi, rowacc0);
    if (gi + CHUNK_ROWS < n) atomicAdd(Q.h + gi + CHUNK_ROWS, rowacc1);
  }
  double Sd = (double)Ssum - (double)Scomp;
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) Sd += __shfl_xor_sync(FULL_MASK, Sd, o);
  if (lane == 0) s_red[warp] = Sd;
  named_bar_sync(CONSUMER_WARPS * 32);
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int w = 0; w < CONSUMER_WARPS; ++w) v += s_red[w];
    Q.stress[blockIdx.x] = v;
  }
}

// Generic k (3..8) fused kernel: the tile's row and column points are staged
// in shared memory; a lane takes 4 columns of each of its warp's 16 rows.
template <int K>
struct FusedKSmem {
  static constexpr int NP = K * (K - 1) / 2;
  float2 p[2][TILE][NP];
  float y[2][TILE][K];
  float colh[TILE][K];
};

// (k = 3 with the Gini metric and Kruskal's loss runs in k_fused3 below.)
template <int K, int DT, bool GRAD>
__global__ void __launch_bounds__(FUSED_THREADS, 2) k_fusedk(const IterParams Q, int64_t ntiles) {
  constexpr int NP = K * (K - 1) / 2;
  extern __shared__ __align__(16) unsigned char s_raw[];
  FusedKSmem<K>& sm = *reinterpret_cast<FusedKSmem<K>*>(s_raw);
  // deterministic mode: per-warp column sums (8 x 128 x K floats after sm)
  float* det_cols = reinterpret_cast<float*>(s_raw + sizeof(FusedKSmem<K>));
  auto& s_p = sm.p;
  auto& s_y = sm.y;
  auto& s_colh = sm.colh;
  __shared__ float s_w[2 * KMAX - 1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x < 2 * KMAX - 1) s_w[threadIdx.x] = Q.tab.w[threadIdx.x];
  for (int e = threadIdx.x; e < TILE * K; e += FUSED_THREADS) (&s_colh[0][0])[e] = 0.f;
  __shared__ int s_ij[2];
  double Sd = 0.0;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    __syncthreads();
    if (threadIdx.x == 0) {
      tile_decode(t, Q.tiles, s_ij[0], s_ij[1]);
      // this CTA's next tile is one contiguous block: have it in L2 by then
      const int64_t tn = t + gridDim.x;
      if (tn < ntiles) {
        constexpr unsigned esz = DT == GINI_F32 ? 4 : (DT == GINI_FP8E4M3 ? 1 : 2);
        const char* base = reinterpret_cast<const char*>(Q.delta) + tn * (int64_t)(TILE * TILE) * esz;
        bulk_prefetch_l2(base, TILE * TILE * esz);
        if (DT == GINI_BF16X2) bulk_prefetch_l2(base + Q.plane * esz, TILE * TILE * esz);
      }
    }
    __syncthreads();
    const int I = s_ij[0], J = s_ij[1];
    const int64_t i0 = (int64_t)I * TILE, j0 = (int64_t)J * TILE;
    for (int e = threadIdx.x; e < 2 * TILE; e += FUSED_THREADS) {
      const int side = e / TILE, l = e % TILE;
      int64_t g = (side ? j0 : i0) + l;
      g = g < Q.n ? g : Q.n - 1;
#pragma unroll
      for (int c = 0; c < K; ++c) s_y[side][l][c] = Q.Y[g * K + c];
#pragma unroll
      for (int p = 0; p < NP; ++p) s_p[side][l][p] = Q.P[g * NP + p];
    }
    __syncthreads();
    float sc[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int64_t gj = j0 + 4 * lane + c;
      sc[c] = (DT == GINI_FP8E4M3) ? Q.col_scale[gj < Q.n ? gj : Q.n - 1] : 1.f;
    }
    const int64_t tbase = t * (int64_t)(TILE * TILE);
    float colacc[4][K];
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int a = 0; a < K; ++a) colacc[c][a] = 0.f;
    float S = 0.f;
    // one pair of the tile: stress term, and dd/dy weighted by the loss into the
    // row accumulator (racc) and, negated, the column accumulator
    auto pair_terms = [&](int rl, int c, const float (&dl)[4], float (&racc)[K]) {
      const int cl = 4 * lane + c;
      const int64_t gi = i0 + rl;
      const bool ok = gi < Q.n && j0 + cl < Q.n && (I != J || rl < cl);
      float dw[K];
      const float d = (Q.metric == GINI_METRIC_EUCLID)
                          ? pair_euclid<K>(s_y[0][rl], s_y[1][cl], dw)
                          : pair_k<K>(s_y[0][rl], s_y[1][cl], s_p[0][rl], s_p[1][cl], s_w, dw);
      float sterm, gw;
      loss_terms(Q.loss, d, dl[c], sterm, gw);
      sterm = ok ? sterm : 0.f;
      gw = ok ? gw : 0.f;
      S += sterm;
#pragma unroll
      for (int a = 0; a < K; ++a) {
        const float tt = gw * dw[a];
        racc[a] += tt;
        colacc[c][a] -= tt;
      }
    };
    // the same with the row's and the column's points already in registers
    auto pair_terms_r = [&](int rl, int c, const float (&dl)[4], const float (&ry)[K],
                            const float2 (&rp)[NP], const float (&cy)[K],
                            const float2 (&cpp)[NP], float (&racc)[K]) {
      const int cl = 4 * lane + c;
      const int64_t gi = i0 + rl;
      const bool ok = gi < Q.n && j0 + cl < Q.n && (I != J || rl < cl);
      float dw[K];
      const float d = (Q.metric == GINI_METRIC_EUCLID) ? pair_euclid<K>(ry, cy, dw)
                                                              : pair_k<K>(ry, cy, rp, cpp, s_w, dw);
      float sterm, gw;
      loss_terms(Q.loss, d, dl[c], sterm, gw);
      sterm = ok ? sterm : 0.f;
      gw = ok ? gw : 0.f;
      S += sterm;
#pragma unroll
      for (int a = 0; a < K; ++a) {
        const float tt = gw * dw[a];
        racc[a] += tt;
        colacc[c][a] -= tt;
      }
    };
    if constexpr (K <= 4) {
      // the lane's 4 columns in registers for the whole tile, a row's points
      // once per row; rows in blocks of 8: per-row partials stay in registers
      // and one 3-stage transpose-reduction (reduce8) per component serves 8 rows
      float cy[4][K];
      float2 cp[4][NP];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
#pragma unroll
        for (int a = 0; a < K; ++a) cy[c][a] = s_y[1][4 * lane + c][a];
#pragma unroll
        for (int q = 0; q < NP; ++q) cp[c][q] = s_p[1][4 * lane + c][q];
      }
      for (int rb = 0; rb < 16; rb += 8) {
        float racc8[K][8];
#pragma unroll
        for (int a = 0; a < K; ++a)
#pragma unroll
          for (int q = 0; q < 8; ++q) racc8[a][q] = 0.f;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int rl = warp * 16 + rb + q;
          float dl[4];
          load4<DT>(Q, tbase + (int64_t)rl * TILE + 4 * lane, dl, sc);
          float racc[K], ry[K];
          float2 rp[NP];
#pragma unroll
          for (int a = 0; a < K; ++a) {
            racc[a] = 0.f;
            ry[a] = s_y[0][rl][a];
          }
#pragma unroll
          for (int qq = 0; qq < NP; ++qq) rp[qq] = s_p[0][rl][qq];
#pragma unroll
          for (int c = 0; c < 4; ++c) pair_terms_r(rl, c, dl, ry, rp, cy[c], cp[c], racc);
#pragma unroll
          for (int a = 0; a < K; ++a) racc8[a][q] = racc[a];
        }
        if (GRAD) {
#pragma unroll
          for (int a = 0; a < K; ++a) {
            const float v = reduce8(racc8[a], lane);
            const int rl = warp * 16 + rb + rev3(lane & 7);
            const int64_t gi = i0 + rl;
            if (lane < 8) {
              if (Q.part) {
                if (GINI_IDX_OK(Q.err, (2 * t * TILE + rl) * K + a, 2 * ntiles * TILE * K))
                  Q.part[(2 * t * TILE + rl) * K + a] = v;
              } else if (gi < Q.n) {
                atomicAdd(Q.h + gi * K + a, v);
              }
            }
          }
        }
      }
    } else {
      for (int rr = 0; rr < 16; ++rr) {
        const int rl = warp * 16 + rr;
        const int64_t gi = i0 + rl;
        float dl[4];
        load4<DT>(Q, tbase + (int64_t)rl * TILE + 4 * lane, dl, sc);
        float racc[K];
#pragma unroll
        for (int a = 0; a < K; ++a) racc[a] = 0.f;
#pragma unroll
        for (int c = 0; c < 4; ++c) pair_terms(rl, c, dl, racc);
        if (GRAD) {
#pragma unroll
          for (int a = 0; a < K; ++a) {
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) racc[a] += __shfl_xor_sync(FULL_MASK, racc[a], o);
          }
          if (lane == 0 && Q.part) {
            if (GINI_IDX_OK(Q.err, (2 * t * TILE + rl) * K + K - 1, 2 * ntiles * TILE * K)) {
#pragma unroll
              for (int a = 0; a < K; ++a) Q.part[(2 * t * TILE + rl) * K + a] = racc[a];
            }
          } else if (lane == 0 && gi < Q.n) {
#pragma unroll
            for (int a = 0; a < K; ++a) atomicAdd(Q.h + gi * K + a, racc[a]);
          }
        }
      }
    }
    Sd += (double)S;
    if (GRAD && Q.part) {
      // deterministic: every warp's column sums in its own slice, summed over
      // the warps in order
      float* cw = det_cols + warp * TILE * K;
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int a = 0; a < K; ++a) cw[(4 * lane + c) * K + a] = colacc[c][a];
      __syncthreads();
      for (int e = threadIdx.x; e < TILE * K; e += FUSED_THREADS) {
        float v = 0.f;
        for (int w = 0; w < FUSED_THREADS / 32; ++w) v += det_cols[w * TILE * K + e];
        if (GINI_IDX_OK(Q.err, (2 * t + 1) * TILE * K + e, 2 * ntiles * TILE * K))
          Q.part[(2 * t + 1) * TILE * K + e] = v;
      }
    } else if (GRAD) {
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int a = 0; a < K; ++a) atomicAdd(&s_colh[4 * lane + c][a], colacc[c][a]);
      __syncthreads();
      for (int e = threadIdx.x; e < TILE * K; e += FUSED_THREADS) {
        const int l = e / K, a = e % K;
        const int64_t gj = j0 + l;
        const float v = s_colh[l][a];
        s_colh[l][a] = 0.f;
        if (gj < Q.n) atomicAdd(Q.h + gj * K + a, v);
      }
    }
  }
  block_store_stress(Sd, Q.stress);
}

// k = 3, Gini metric, Kruskal loss: the fused iteration fed by bulk copies.
//
// The arithmetic per pair is k_fusedk's packed k = 3 body (two columns per
// f32x2 instruction; exact signs of the three coordinate-pair differences from
// the scaled point pairs; midrank offsets x_c affine in the signs; dw_c =
// x_c (A + B x_c^2), or A x_c when B = 0).  What changes is how the data
// arrive.  A CTA owns a contiguous range of tiles, streamed as chunks of 64
// rows x 128 columns; a stage of the shared-memory ring holds one chunk's
// dissimilarities, its 64 row points and the tile's 128 column points (padded
// coordinates Y4 and point pairs P, both padded to whole tiles), all brought
// by cp.async.bulk and completed on the stage's mbarrier.  There is no
// producer warp (its registers would cost the second CTA per SM at 128 per
// thread): each warp counts itself done with a stage in a shared counter, and
// the warp that completes the count issues the stage's next chunk.  Column
// sums of a tile meet in per-warp slices behind one named barrier (slices
// double-buffered by tile parity); row sums of the 8 rows a warp owns in a
// chunk meet by a transpose-reduction and stay in registers while the tile
// row does not change.
template <int DT>
struct Pipe3Cfg {
  static constexpr int planes = DT == GINI_BF16X2 ? 2 : 1;
  static constexpr int esize = DT == GINI_F32 ? 4 : (DT == GINI_FP8E4M3 ? 1 : 2);
  static constexpr int plane_bytes = CHUNK_ROWS * TILE * esize;
  static constexpr int yrow_off = planes * plane_bytes;          // 64 x float4
  static constexpr int prow_off = yrow_off + CHUNK_ROWS * 16;     // 64 x 3 float2
  static constexpr int ycol_off = prow_off + CHUNK_ROWS * 24;     // 128 x float4
  static constexpr int pcol_off = ycol_off + TILE * 16;           // 128 x 3 float2
  static constexpr int stage_bytes = pcol_off + TILE * 24;
  // ~86 KB of stages + 24.6 KB of column slices keeps two CTAs on an SM
  static constexpr int stages_raw = (86 * 1024) / stage_bytes;
  static constexpr int stages = stages_raw > 4 ? 4 : (stages_raw < 2 ? 2 : stages_raw);
  static constexpr int smem = stages * stage_bytes;
  static_assert(prow_off % 16 == 0 && ycol_off % 16 == 0 && pcol_off % 16 == 0 &&
                    stage_bytes % 16 == 0,
                "bulk-copy destinations must be 16-byte aligned");
};

// Issues chunk c (tile t = t_begin + c / 2, half h = c & 1, tile (I, J)) into
// its stage.  One thread.
template <int DT>
__device__ __forceinline__ void fused3_issue(const IterParams& Q, unsigned char* s_stage,
                                             uint64_t* bar_full, int S, int64_t t_begin,
                                             int64_t ntiles, int c, int I, int J) {
  using C = Pipe3Cfg<DT>;
  const int s = c % S, h = c & 1;
  const int64_t t = t_begin + c / 2;
  const int64_t eoff = t * (int64_t)(TILE * TILE) + (int64_t)h * CHUNK_ROWS * TILE;
  const int64_t ri = (int64_t)I * TILE + h * CHUNK_ROWS, cj = (int64_t)J * TILE;
  unsigned char* dst = s_stage + s * C::stage_bytes;
  const unsigned char* base = reinterpret_cast<const unsigned char*>(Q.delta);
  [[maybe_unused]] const int64_t padded = Q.tiles * TILE;
  // (debug builds) the chunk inside the plane, the points inside the padded
  // arrays; a failed check completes the stage without copies
  if (GINI_IDX_OK(Q.err, t, ntiles) &&
      GINI_IDX_OK(Q.err, eoff + CHUNK_ROWS * TILE - 1, ntiles * (TILE * TILE)) &&
      GINI_IDX_OK(Q.err, ri + CHUNK_ROWS - 1, padded) && GINI_IDX_OK(Q.err, cj + TILE - 1, padded)) {
    mbar_arrive_expect_tx(&bar_full[s], C::stage_bytes);
    bulk_copy_g2s(dst, base + eoff * C::esize, C::plane_bytes, &bar_full[s]);
    if (C::planes == 2)
      bulk_copy_g2s(dst + C::plane_bytes, base + (Q.plane + eoff) * C::esize, C::plane_bytes,
                    &bar_full[s]);
    bulk_copy_g2s(dst + C::yrow_off, Q.Y4 + ri, CHUNK_ROWS * 16, &bar_full[s]);
    bulk_copy_g2s(dst + C::prow_off, Q.P + ri * 3, CHUNK_ROWS * 24, &bar_full[s]);
    bulk_copy_g2s(dst + C::ycol_off, Q.Y4 + cj, TILE * 16, &bar_full[s]);
    bulk_copy_g2s(dst + C::pcol_off, Q.P + cj * 3, TILE * 24, &bar_full[s]);
  } else {
    mbar_arrive(&bar_full[s]);
  }
}

template <int DT, bool GRAD, bool AFF>
__global__ void __launch_bounds__(FUSED_THREADS, 2) k_fused3(const IterParams Q, int64_t ntiles) {
  using C = Pipe3Cfg<DT>;
  constexpr int S = C::stages;
  constexpr int WARPS = FUSED_THREADS / 32;
  extern __shared__ __align__(128) unsigned char s_stage[];
  __shared__ __align__(8) uint64_t bar_full[S];
  __shared__ unsigned s_done[S];  // warps finished with the chunk now in the stage
  __shared__ float s_colw[2][WARPS][TILE * 3];
  __shared__ int s_abort;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t n = Q.n;
  const int64_t t_begin = ntiles * blockIdx.x / gridDim.x;
  const int64_t t_end = ntiles * (blockIdx.x + 1) / gridDim.x;
  const int nchunks = (int)(t_end - t_begin) * 2;
  int I = 0, J = 0;
  if (nchunks) tile_decode(t_begin, Q.tiles, I, J);
  if (threadIdx.x == 0) {
    for (int st = 0; st < S; ++st) {
      mbar_init(&bar_full[st], 1);
      s_done[st] = 0;
    }
    s_abort = 0;
    mbar_init_fence();
  }
  __syncthreads();
  volatile int* abort = &s_abort;
  if (threadIdx.x == 0) {  // the first S chunks
    int i2 = I, j2 = J;
    for (int c = 0; c < S && c < nchunks; ++c) {
      if (c > 0 && (c & 1) == 0) tile_next(i2, j2, Q.tiles);
      fused3_issue<DT>(Q, s_stage, bar_full, S, t_begin, ntiles, c, i2, j2);
    }
  }

  const float t1 = Q.tab.w[4], th = Q.tab.w[3];
  const float A = (8.f * th - t1) * (1.f / 3.f), B = (4.f * t1 - 8.f * th) * (1.f / 3.f);
  const float2 A2 = make_float2(A, A), B2 = make_float2(B, B), nA2 = make_float2(-A, -A);
  const float2 khi = make_float2(SIGN_HI, SIGN_HI);
  const float2 m1 = make_float2(-1.f, -1.f), one2 = make_float2(1.f, 1.f);
  float Ssum = 0.f, Scomp = 0.f;  // compensated sum of the per-tile FP32 partials
  float2 S2 = make_float2(0.f, 0.f);
  float rowacc[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};  // lane < 8: rows rev3(lane)
  int curI = -1;
  float2 ncy[2][3], nch[2][3], ncl[2][3], cacc[2][3];
  float sc[4] = {1.f, 1.f, 1.f, 1.f};
  for (int c = 0; c < nchunks; ++c) {
    const int s = c % S, h = c & 1;
    if (h == 0 && c > 0) tile_next(I, J, Q.tiles);
    if (GRAD && h == 0 && I != curI) {
      if (!Q.part && curI >= 0 && lane < 8) {
        const int64_t gi = (int64_t)curI * TILE + warp * 8 + rev3(lane);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          if (gi < n) atomicAdd(Q.h + gi * 3 + a, rowacc[0][a]);
          if (gi + CHUNK_ROWS < n) atomicAdd(Q.h + (gi + CHUNK_ROWS) * 3 + a, rowacc[1][a]);
        }
      }
#pragma unroll
      for (int a = 0; a < 3; ++a) rowacc[0][a] = rowacc[1][a] = 0.f;
      curI = I;
    }
    if (!mbar_wait_bounded(&bar_full[s], (c / S) & 1, abort)) {
      raise_error(Q.err, ERR_TIMEOUT);
      *abort = 1;
    }
    const unsigned char* stage = s_stage + s * C::stage_bytes;
    if (h == 0) {
      // the lane's four columns (4 lane + 2p, 4 lane + 2p + 1), negated and packed
      const float4* yc = reinterpret_cast<const float4*>(stage + C::ycol_off);
      const float2* pc = reinterpret_cast<const float2*>(stage + C::pcol_off);
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        const int c0 = 4 * lane + 2 * p;
        const float4 ya = yc[c0], yb = yc[c0 + 1];
        ncy[p][0] = make_float2(-ya.x, -yb.x);
        ncy[p][1] = make_float2(-ya.y, -yb.y);
        ncy[p][2] = make_float2(-ya.z, -yb.z);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const float2 pa = pc[c0 * 3 + a], pb = pc[(c0 + 1) * 3 + a];
          nch[p][a] = make_float2(-pa.x, -pb.x);
          ncl[p][a] = make_float2(-pa.y, -pb.y);
          cacc[p][a] = make_float2(0.f, 0.f);
        }
      }
      if (DT == GINI_FP8E4M3) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int64_t gj = (int64_t)J * TILE + 4 * lane + q;
          sc[q] = Q.col_scale[gj < n ? gj : n - 1];
        }
      }
    }
    const bool masked = (I == J) || ((int64_t)I * TILE + TILE > n) || ((int64_t)J * TILE + TILE > n);
    const float4* yr = reinterpret_cast<const float4*>(stage + C::yrow_off);
    const float2* pr = reinterpret_cast<const float2*>(stage + C::prow_off);
    float racc8[3][8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int rr = warp * 8 + q;  // row within the chunk
      const int rl = h * CHUNK_ROWS + rr;
      float dl[4];
      load4_smem<DT>(stage, rr, lane, dl, sc);
      const float4 yv = yr[rr];
      const float yvs[3] = {yv.x, yv.y, yv.z};
      float2 ryy[3], rph[3], rpl[3], rn[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const float2 pv = pr[rr * 3 + a];
        ryy[a] = make_float2(yvs[a], yvs[a]);
        rph[a] = make_float2(pv.x, pv.x);
        rpl[a] = make_float2(pv.y, pv.y);
        rn[a] = make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        float2 sp[3];
#pragma unroll
        for (int qq = 0; qq < 3; ++qq) {
          const float2 dh = __fadd2_rn(rph[qq], nch[p][qq]);
          const float2 dlo = __fadd2_rn(rpl[qq], ncl[p][qq]);
          const float2 a2 = __ffma2_rn(dh, khi, dlo);  // dlo scaled by 2^24
          sp[qq] = make_float2(__saturatef(fmaf(a2.x, SIGN_SAT, 0.5f)),
                               __saturatef(fmaf(a2.y, SIGN_SAT, 0.5f)));
        }
        float2 dw[3];
        if constexpr (AFF) {
          dw[0] = __ffma2_rn(__fadd2_rn(sp[0], sp[1]), A2, nA2);  // A (sp0 + sp1 - 1)
          dw[1] = __fmul2_rn(__ffma2_rn(sp[0], m1, sp[2]), A2);   // A (sp2 - sp0)
          dw[2] = __ffma2_rn(__fadd2_rn(sp[1], sp[2]), nA2, A2);  // A (1 - sp1 - sp2)
        } else {
          float2 xs[3];
          xs[0] = __fadd2_rn(__fadd2_rn(sp[0], sp[1]), m1);
          xs[1] = __ffma2_rn(sp[0], m1, sp[2]);
          xs[2] = __ffma2_rn(__fadd2_rn(sp[1], sp[2]), m1, one2);
#pragma unroll
          for (int cc = 0; cc < 3; ++cc)
            dw[cc] = __fmul2_rn(xs[cc], __ffma2_rn(B2, __fmul2_rn(xs[cc], xs[cc]), A2));
        }
        float2 d = make_float2(0.f, 0.f);
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) d = __ffma2_rn(__fadd2_rn(ryy[cc], ncy[p][cc]), dw[cc], d);
        float2 nr = __ffma2_rn(d, m1, make_float2(dl[2 * p], dl[2 * p + 1]));
        if (masked) {
          const int cl = 4 * lane + 2 * p;
          const bool rok = (int64_t)I * TILE + rl < n;
          const bool ok0 = rok && ((int64_t)J * TILE + cl < n) && (I != J || rl < cl);
          const bool ok1 = rok && ((int64_t)J * TILE + cl + 1 < n) && (I != J || rl < cl + 1);
          nr.x = ok0 ? nr.x : 0.f;
          nr.y = ok1 ? nr.y : 0.f;
        }
        S2 = __ffma2_rn(nr, nr, S2);
        if (GRAD) {
#pragma unroll
          for (int cc = 0; cc < 3; ++cc) {
            rn[cc] = __ffma2_rn(nr, dw[cc], rn[cc]);
            cacc[p][cc] = __ffma2_rn(nr, dw[cc], cacc[p][cc]);
          }
        }
      }
#pragma unroll
      for (int a = 0; a < 3; ++a) racc8[a][q] = -(rn[a].x + rn[a].y);
    }
    // this warp is done with the stage; the last warp to finish refills it
    __syncwarp();
    if (lane == 0) {
      __threadfence_block();
      if (atomicAdd(&s_done[s], 1u) == WARPS - 1) {
        s_done[s] = 0;
        const int cn = c + S;
        if (cn < nchunks) {
          int i2 = I, j2 = J;
          for (int k2 = c / 2; k2 < cn / 2; ++k2) tile_next(i2, j2, Q.tiles);
          __threadfence_block();
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          fused3_issue<DT>(Q, s_stage, bar_full, S, t_begin, ntiles, cn, i2, j2);
        }
      }
    }
    if (GRAD) {
#pragma unroll
      for (int a = 0; a < 3; ++a) rowacc[h][a] += reduce8(racc8[a], lane);
    }
    if (h == 1) {
      const float y = (S2.x + S2.y) - Scomp;  // fold the tile's FP32 partial (Kahan)
      const float tsum = Ssum + y;
      Scomp = (tsum - Ssum) - y;
      Ssum = tsum;
      S2 = make_float2(0.f, 0.f);
      if (GRAD) {
        const int64_t tcur = t_begin + (c >> 1);
        if (Q.part && lane < 8) {  // deterministic: this tile's row sums
          const int rl = warp * 8 + rev3(lane);
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            if (GINI_IDX_OK(Q.err, (2 * tcur * TILE + rl + CHUNK_ROWS) * 3 + a,
                            2 * ntiles * TILE * 3)) {
              Q.part[(2 * tcur * TILE + rl) * 3 + a] = rowacc[0][a];
              Q.part[(2 * tcur * TILE + rl + CHUNK_ROWS) * 3 + a] = rowacc[1][a];
            }
            rowacc[0][a] = rowacc[1][a] = 0.f;
          }
        }
        float* cw = s_colw[(c >> 1) & 1][warp];
#pragma unroll
        for (int p = 0; p < 2; ++p)
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            cw[(4 * lane + 2 * p) * 3 + a] = cacc[p][a].x;
            cw[(4 * lane + 2 * p + 1) * 3 + a] = cacc[p][a].y;
          }
        named_bar_sync(FUSED_THREADS);
        for (int e = threadIdx.x; e < TILE * 3; e += FUSED_THREADS) {
          float v = 0.f;
#pragma unroll
          for (int w = 0; w < WARPS; ++w) v += s_colw[(c >> 1) & 1][w][e];
          const int64_t gj = (int64_t)J * TILE + e / 3;
          if (Q.part) {
            if (GINI_IDX_OK(Q.err, (2 * tcur + 1) * TILE * 3 + e, 2 * ntiles * TILE * 3))
              Q.part[(2 * tcur + 1) * TILE * 3 + e] = v;
          } else if (gj < n) {
            atomicAdd(Q.h + gj * 3 + e % 3, v);
          }
        }
      }
    }
  }
  if (GRAD && !Q.part && curI >= 0 && lane < 8) {
    const int64_t gi = (int64_t)curI * TILE + warp * 8 + rev3(lane);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (gi < n) atomicAdd(Q.h + gi * 3 + a, rowacc[0][a]);
      if (gi + CHUNK_ROWS < n) atomicAdd(Q.h + (gi + CHUNK_ROWS) * 3 + a, rowacc[1][a]);
    }
  }
  // Copies still in flight must land before this CTA's shared memory can be
  // released: normally every issued chunk has been waited for already.
  if (threadIdx.x == 0)
    for (int c = (nchunks > S ? nchunks - S : 0); c < nchunks; ++c)
      mbar_wait_bounded(&bar_full[c % S], (c / S) & 1, nullptr);
  block_store_stress((double)Ssum - (double)Scomp, Q.stress);
}

// ------------------------------------------------------ update, finalize ---

// Y <- Y - scale * h (scale = eta * 2 / sum_delta2; for k = 2 the gradient is
// c2 * h_i * (1, -1)), then refresh the point pairs and clear h.
template <int K>
__global__ void k_update(float* __restrict__ Y, int64_t n, float2* __restrict__ P,
                         float4* __restrict__ Y4, float* __restrict__ h, float scale, float c2,
                         bool scalar2, unsigned* err) {
  constexpr int NP = K * (K - 1) / 2;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool bad = false;
  if (i < n) {
    float y[K];
#pragma unroll
    for (int c = 0; c < K; ++c) y[c] = Y[i * K + c];
    if (K == 2 && scalar2) {
      const float g = scale * c2 * h[i];
      y[0] -= g;
      y[1] += g;
      h[i] = 0.f;
    } else {
#pragma unroll
      for (int c = 0; c < K; ++c) {
        y[c] -= scale * h[i * K + c];
        h[i * K + c] = 0.f;
      }
    }
    int p = 0;
#pragma unroll
    for (int c = 0; c < K; ++c) {
      Y[i * K + c] = y[c];
      bad |= !isfinite(y[c]);
    }
#pragma unroll
    for (int a = 0; a < K; ++a)
#pragma unroll
      for (int b = a + 1; b < K; ++b) P[i * NP + (p++)] = point_pair(y[a], y[b]);
    if (K == 3 && Y4) Y4[i] = make_float4(y[0], y[1], y[K - 1], 0.f);
  }
  if (__any_sync(FULL_MASK, bad) && (threadIdx.x & 31) == 0) raise_error(err, ERR_NONFINITE);
}

__global__ void k_finalize_grad(const float* __restrict__ h, int64_t n, int k, float scale,
                                float c2, bool scalar2, float* __restrict__ grad) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (k == 2 && scalar2) {
    const float g = scale * c2 * h[i];
    grad[i * 2] = g;
    grad[i * 2 + 1] = -g;
  } else {
    for (int c = 0; c < k; ++c) grad[i * k + c] = scale * h[i * k + c];
  }
}

// S of each of cnt passes: one warp per pass sums its STRESS_SLOTS slots in a
// fixed order (lane-strided, then a shuffle tree), times 1 / normaliser.
__global__ void k_finalize_stress(const double* slots, int cnt, double inv_sd2, double* hist,
                                  double* final_out) {
  const int t = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (t >= cnt) return;
  const double* sl = slots + (size_t)t * STRESS_SLOTS;
  double v = 0.0;
  for (int k = lane; k < STRESS_SLOTS; k += 32) v += sl[k];
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(FULL_MASK, v, o);
  if (lane == 0) {
    v *= inv_sd2;
    if (hist) hist[t] = v;
    if (final_out && t == cnt - 1) final_out[0] = v;
  }
}

// Deterministic mode: the gradient accumulators h from the per-tile partials
// (IterParams::part), every point's terms added in the same order on every
// run.  CTA = one tile row I (128 points) x 8 groups; group g takes the tiles
// (I, J) with J = I + g, I + g + 8, ... (row sums) and (J', I) with J' = g,
// g + 8, ... <= I (column sums); the 8 group sums are added in group order.
__global__ void __launch_bounds__(8 * TILE) k_det_reduce(const float* __restrict__ part,
                                                       int64_t n, int64_t T, int kp,
                                                       float* __restrict__ h, unsigned* err) {
  __shared__ float s_g[8][TILE * KMAX];
  const int64_t I = blockIdx.x;
  const int g = threadIdx.x / TILE, r = threadIdx.x % TILE;
  if (!(GINI_IDX_OK(err, kp - 1, KMAX) && GINI_IDX_OK(err, I, T))) return;  // (debug builds)
  [[maybe_unused]] const int64_t lim = T * (T + 1) * TILE * kp;  // the partials of all tiles
  for (int a = 0; a < kp; ++a) {
    float v = 0.f;
    for (int64_t J = I + g; J < T; J += 8) {
      const int64_t o = (2 * tile_offset(I, J, T) * TILE + r) * kp + a;
      if (GINI_IDX_OK(err, o, lim)) v += part[o];
    }
    for (int64_t J = g; J <= I; J += 8) {
      const int64_t o = ((2 * tile_offset(J, I, T) + 1) * TILE + r) * kp + a;
      if (GINI_IDX_OK(err, o, lim)) v += part[o];
    }
    s_g[g][r * kp + a] = v;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < TILE * kp; e += blockDim.x) {
    const int64_t i = I * TILE + e / kp;
    if (i < n) {
      float v = 0.f;
#pragma unroll
      for (int q = 0; q < 8; ++q) v += s_g[q][e];
      h[i * kp + e % kp] = v;
    }
  }
}

// ---------------------------------------------------------------- host -----

struct IterWs {
  float2* P;
  float4* Y4;    // k = 3 only
  float* h;
  double* acc;   // nacc x STRESS_SLOTS stress slots
  float* part;   // deterministic mode: per-tile gradient partials, else null
  unsigned* err;
};

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace gini

using namespace gini;

extern "C" void gini_set_cuda_error(cudaError_t e);
extern "C" int gini_get_deterministic(void);

// Workspace of the iteration ops: header | nacc x STRESS_SLOTS doubles | point
// pairs | h | (k = 3) padded coordinates | (deterministic mode) per-tile
// gradient partials.  Point pairs and padded coordinates are stored for
// ceil(n / B) * B points (whole tiles, the padding zero-filled) so that bulk
// copies of a tile's points never leave the arrays.
static int64_t padded_points(int64_t n) { return tiles_1d(n) * TILE; }

static size_t part_floats(int64_t n, int k) {
  const int64_t T = tiles_1d(n);
  return (size_t)(T * (T + 1) / 2) * 2 * TILE * (size_t)k;
}

extern "C" size_t gini_iter_ws_bytes(int64_t n, int k, int nacc, int det) {
  const int np = k * (k - 1) / 2;
  return WS_HEADER + align256(sizeof(double) * (size_t)nacc * STRESS_SLOTS) +
         align256(sizeof(float2) * (size_t)padded_points(n) * np) +
         align256(sizeof(float) * (size_t)n * k) +
         (k == 3 ? align256(sizeof(float4) * (size_t)padded_points(n)) : 0) +
         (det ? align256(sizeof(float) * part_floats(n, k)) : 0);
}

static IterWs carve(void* ws, int64_t n, int k, int nacc, bool det) {
  IterWs w;
  char* p = reinterpret_cast<char*>(ws);
  w.err = reinterpret_cast<unsigned*>(p);
  p += WS_HEADER;
  w.acc = reinterpret_cast<double*>(p);
  p += align256(sizeof(double) * (size_t)nacc * STRESS_SLOTS);
  w.P = reinterpret_cast<float2*>(p);
  p += align256(sizeof(float2) * (size_t)padded_points(n) * (k * (k - 1) / 2));
  w.h = reinterpret_cast<float*>(p);
  p += align256(sizeof(float) * (size_t)n * k);
  w.Y4 = nullptr;
  if (k == 3) {
    w.Y4 = reinterpret_cast<float4*>(p);
    p += align256(sizeof(float4) * (size_t)padded_points(n));
  }
  w.part = det ? reinterpret_cast<float*>(p) : nullptr;
  return w;
}

static PairTab make_tab(int k, double nu) {
  PairTab T{};
  T.c2 = (float)pow(2.0, 1.0 - nu);
  const double d = (double)k;
  for (int idx = 0; idx <= 2 * k - 2; ++idx) {
    const double R = (idx + 2) / 2.0;
    T.w[idx] = (float)(0.5 * d * (pow((R - 1.0) / d, nu - 1.0) - pow((d - R) / d, nu - 1.0)));
  }
  return T;
}

// Per-device caches: a process may drive several GPUs (one per thread).
constexpr int MAX_DEVICES = 64;

static int sm_count() {
  static std::atomic<int> cached[MAX_DEVICES];
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return 148;
  const int c = cached[dev].load(std::memory_order_relaxed);
  if (c > 0) return c;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0)
    return 148;
  cached[dev].store(v, std::memory_order_relaxed);
  return v;
}

// The dynamic shared-memory limit above 48 KB is an attribute of the kernel on
// each device: set it once per device (setting it twice is harmless).
template <typename Kern>
static void smem_attr_once(Kern* fn, int bytes, std::atomic<unsigned long long>& done) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  const unsigned long long bit = 1ull << (dev & 63);
  if (done.load(std::memory_order_acquire) & bit) return;
  cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  done.fetch_or(bit, std::memory_order_acq_rel);
}

static int check_common(int64_t n, int k, double nu, const void* delta, int layout, int dtype,
                        int64_t ldd, const float* col_scale, double sum_delta2) {
  if (!delta) return GINI_EINVAL;
  if (n < 2 || n > ((int64_t)1 << 31) || k < 2 || k > KMAX) return GINI_EINVAL;
  if (!(nu > 1.0) || !isfinite(nu)) return GINI_EINVAL;
  if (layout == GINI_LAYOUT_FULL) {
    if (dtype != GINI_F32 || ldd < n) return GINI_EINVAL;
  } else if (layout == GINI_LAYOUT_TILED) {
    if (dtype < GINI_F32 || dtype > GINI_FP8E4M3) return GINI_EINVAL;
    if (dtype == GINI_FP8E4M3 && !col_scale) return GINI_EINVAL;
    if ((reinterpret_cast<uintptr_t>(delta) & 15) != 0) return GINI_EINVAL;
  } else {
    return GINI_EINVAL;
  }
  if (!(sum_delta2 > 0.0) || !isfinite(sum_delta2)) return GINI_EDEGENERATE;
  return GINI_OK;
}

template <int K>
static void launch_prep(const float* Y, int64_t n, float2* P, float4* Y4, unsigned* err,
                        cudaStream_t s) {
  const int64_t npad = padded_points(n);
  gini_count_launch(1);
  k_prep<K><<<(unsigned)((npad + 255) / 256), 256, 0, s>>>(Y, n, npad, P, Y4, err);
}

static void prep(int k, const float* Y, int64_t n, float2* P, float4* Y4, unsigned* err,
                 cudaStream_t s) {
  switch (k) {
    case 2: launch_prep<2>(Y, n, P, Y4, err, s); break;
    case 3: launch_prep<3>(Y, n, P, Y4, err, s); break;
    case 4: launch_prep<4>(Y, n, P, Y4, err, s); break;
    case 5: launch_prep<5>(Y, n, P, Y4, err, s); break;
    case 6: launch_prep<6>(Y, n, P, Y4, err, s); break;
    case 7: launch_prep<7>(Y, n, P, Y4, err, s); break;
    default: launch_prep<8>(Y, n, P, Y4, err, s); break;
  }
}

template <int K>
static void launch_update(float* Y, int64_t n, float2* P, float4* Y4, float* h, float scale,
                          float c2, bool scalar2, unsigned* err, cudaStream_t s) {
  gini_count_launch(1);
  k_update<K><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(Y, n, P, Y4, h, scale, c2, scalar2,
                                                          err);
}

static void update(int k, float* Y, int64_t n, float2* P, float4* Y4, float* h, float scale,
                   float c2, bool scalar2, unsigned* err, cudaStream_t s) {
  switch (k) {
    case 2: launch_update<2>(Y, n, P, Y4, h, scale, c2, scalar2, err, s); break;
    case 3: launch_update<3>(Y, n, P, Y4, h, scale, c2, scalar2, err, s); break;
    case 4: launch_update<4>(Y, n, P, Y4, h, scale, c2, scalar2, err, s); break;
    case 5: launch_update<5>(Y, n, P, Y4, h, scale, c2, scalar2, err, s); break;
    case 6: launch_update<6>(Y, n, P, Y4, h, scale, c2, scalar2, err, s); break;
    case 7: launch_update<7>(Y, n, P, Y4, h, scale, c2, scalar2, err, s); break;
    default: launch_update<8>(Y, n, P, Y4, h, scale, c2, scalar2, err, s); break;
  }
}

template <int K, bool FWD>
static void launch_full(const IterParams& Q, cudaStream_t s) {
  const int64_t blocks = (Q.n + 7) / 8;  // a warp per row, rows grid-strided
  // only the forward pass writes a stress slot per CTA; the adjoint takes a
  // warp per row over the whole grid
  const unsigned g = (unsigned)(FWD && blocks > STRESS_SLOTS ? STRESS_SLOTS : blocks);
  gini_count_launch(1);
  k_full<K, FWD><<<g, 256, 0, s>>>(Q);
}

template <bool FWD>
static void full_k(int k, const IterParams& Q, cudaStream_t s) {
  switch (k) {
    case 2: launch_full<2, FWD>(Q, s); break;
    case 3: launch_full<3, FWD>(Q, s); break;
    case 4: launch_full<4, FWD>(Q, s); break;
    case 5: launch_full<5, FWD>(Q, s); break;
    case 6: launch_full<6, FWD>(Q, s); break;
    case 7: launch_full<7, FWD>(Q, s); break;
    default: launch_full<8, FWD>(Q, s); break;
  }
}

template <int K, int DT, bool GRAD>
static void launch_fusedk(unsigned g, const IterParams& Q, int64_t ntiles, cudaStream_t s) {
  // deterministic mode: per-warp column sums after the staged points
  const size_t smem = sizeof(FusedKSmem<K>) +
                      (GRAD && Q.part ? sizeof(float) * (FUSED_THREADS / 32) * TILE * K : 0);
  if (smem + 1024 > 48 * 1024)  // plus the kernel's static shared memory
    cudaFuncSetAttribute(k_fusedk<K, DT, GRAD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
  gini_count_launch(1);
  k_fusedk<K, DT, GRAD><<<g, FUSED_THREADS, smem, s>>>(Q, ntiles);
}

template <int DT, bool GRAD, bool AFF>
static void launch_fused3(const IterParams& Q, int64_t ntiles, cudaStream_t s) {
  using C = Pipe3Cfg<DT>;
  static std::atomic<unsigned long long> attr{0};
  smem_attr_once(k_fused3<DT, GRAD, AFF>, C::smem, attr);
  const int64_t cap = std::min<int64_t>((int64_t)sm_count() * 2, STRESS_SLOTS);
  const unsigned g = (unsigned)(ntiles < cap ? ntiles : cap);
  gini_count_launch(1);
  k_fused3<DT, GRAD, AFF><<<g, FUSED_THREADS, C::smem, s>>>(Q, ntiles);
}

template <int DT, bool GRAD>
static void launch_fused_dt(int k, const IterParams& Q, cudaStream_t s) {
  const int64_t ntiles = Q.tiles * (Q.tiles + 1) / 2;
  const int64_t cap = std::min<int64_t>((int64_t)sm_count() * 4, STRESS_SLOTS);
  const unsigned g = (unsigned)(ntiles < cap ? ntiles : cap);
  if (!scalar2_path(k, Q.metric, Q.loss)) {
    switch (k) {
      case 2: launch_fusedk<2, DT, GRAD>(g, Q, ntiles, s); return;
      case 3:
        if (Q.metric == GINI_METRIC_GINI && Q.loss == GINI_LOSS_KRUSKAL) {
          // the table's cubic term B = (4 T(1) - 8 T(1/2)) / 3 is exactly zero
          // when T(1) = 2 T(1/2) in FP32 (nu = 2 or 3)
          if (Q.tab.w[4] == 2.f * Q.tab.w[3])
            launch_fused3<DT, GRAD, true>(Q, ntiles, s);
          else
            launch_fused3<DT, GRAD, false>(Q, ntiles, s);
        } else
          launch_fusedk<3, DT, GRAD>(g, Q, ntiles, s);
        return;
      case 4: launch_fusedk<4, DT, GRAD>(g, Q, ntiles, s); return;
      case 5: launch_fusedk<5, DT, GRAD>(g, Q, ntiles, s); return;
      case 6: launch_fusedk<6, DT, GRAD>(g, Q, ntiles, s); return;
      case 7: launch_fusedk<7, DT, GRAD>(g, Q, ntiles, s); return;
      default: launch_fusedk<8, DT, GRAD>(g, Q, ntiles, s); return;
    }
  }
  switch (k) {
    case 2: {
      using C = PipeCfg<DT>;
      static std::atomic<unsigned long long> attr{0};
      smem_attr_once(k_fused2<DT, GRAD>, C::smem, attr);
      static std::atomic<int> per_sm_cached{0};  // resident CTAs per SM (same on every GB300)
      int per_sm = per_sm_cached.load(std::memory_order_relaxed);
      if (!per_sm) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fused2<DT, GRAD>,
                                                          PIPE_THREADS, C::smem) != cudaSuccess ||
            per_sm < 1)
          per_sm = 1;
        per_sm_cached.store(per_sm, std::memory_order_relaxed);
      }
      const int64_t cap2 = std::min<int64_t>((int64_t)sm_count() * per_sm, STRESS_SLOTS);
      const unsigned g2 = (unsigned)(ntiles < cap2 ? ntiles : cap2);
      gini_count_launch(1);
      k_fused2<DT, GRAD><<<g2, PIPE_THREADS, C::smem, s>>>(Q, ntiles);
      break;
    }
    case 3: launch_fusedk<3, DT, GRAD>(g, Q, ntiles, s); break;
    case 4: launch_fusedk<4, DT, GRAD>(g, Q, ntiles, s); break;
    case 5: launch_fusedk<5, DT, GRAD>(g, Q, ntiles, s); break;
    case 6: launch_fusedk<6, DT, GRAD>(g, Q, ntiles, s); break;
    case 7: launch_fusedk<7, DT, GRAD>(g, Q, ntiles, s); break;
    default: launch_fusedk<8, DT, GRAD>(g, Q, ntiles, s); break;
  }
}

template <bool GRAD>
static void launch_fused(int k, int dtype, const IterParams& Q, cudaStream_t s) {
  switch (dtype) {
    case GINI_F32: launch_fused_dt<GINI_F32, GRAD>(k, Q, s); break;
    case GINI_BF16: launch_fused_dt<GINI_BF16, GRAD>(k, Q, s); break;
    case GINI_BF16X2: launch_fused_dt<GINI_BF16X2, GRAD>(k, Q, s); break;
    default: launch_fused_dt<GINI_FP8E4M3, GRAD>(k, Q, s); break;
  }
}

// One pass: stress into the slots at Q.stress (and h if grad).  dtype_eff lets a
// BF16X2 matrix be read through its hi plane only.  In deterministic mode the
// fused kernels write per-tile partials and k_det_reduce forms h from them;
// the plain form's adjoint writes each h_i from one warp already.
static void one_pass(int k, int layout, int dtype_eff, bool grad, const IterParams& Q,
                     cudaStream_t s) {
  if (layout == GINI_LAYOUT_FULL) {
    full_k<true>(k, Q, s);
    if (grad) full_k<false>(k, Q, s);
  } else if (grad) {
    launch_fused<true>(k, dtype_eff, Q, s);
    if (Q.part) {
      const int kp = scalar2_path(k, Q.metric, Q.loss) ? 1 : k;
      gini_count_launch(1);
      k_det_reduce<<<(unsigned)Q.tiles, 8 * TILE, 0, s>>>(Q.part, Q.n, Q.tiles, kp, Q.h, Q.err);
    }
  } else {
    launch_fused<false>(k, dtype_eff, Q, s);
  }
}

static IterParams make_params(int64_t n, int k, double nu, const float* Y, const void* delta,
                              int64_t ldd, const float* col_scale, const IterWs& w) {
  IterParams Q{};
  Q.n = n;
  Q.P = w.P;
  Q.Y = Y;
  Q.Y4 = w.Y4;
  Q.delta = delta;
  Q.ldd = ldd;
  Q.col_scale = col_scale;
  Q.tiles = tiles_1d(n);
  Q.plane = gini_tiled_elems(n);
  Q.h = w.h;
  Q.stress = w.acc;
  Q.part = w.part;
  Q.tab = make_tab(k, nu);
  Q.err = w.err;
  return Q;
}

extern "C" int gini_stress_grad_ex(const float* Y_dev, int64_t n, int k, double nu,
                                   const void* delta_dev, int layout, int dtype, int64_t ldd,
                                   const float* col_scale_dev, int metric, int loss, double norm,
                                   double* stress_dev, float* grad_dev, void* ws, size_t ws_bytes,
                                   void* stream) {
  NvtxRange nvtx_range("gini_stress_grad_ex");
  if (!Y_dev || !stress_dev || !ws) return GINI_EINVAL;
  if (ws_misaligned(ws)) return GINI_EINVAL;  // point pairs are bulk-copied from it
  if (metric != GINI_METRIC_GINI && metric != GINI_METRIC_EUCLID) return GINI_EINVAL;
  if (loss != GINI_LOSS_KRUSKAL && loss != GINI_LOSS_SAMMON) return GINI_EINVAL;
  int st = check_common(n, k, nu, delta_dev, layout, dtype, ldd, col_scale_dev, norm);
  if (st != GINI_OK) return st;
  const bool det = gini_get_deterministic() && layout == GINI_LAYOUT_TILED && grad_dev;
  if (ws_bytes < gini_workspace_size(det ? GINI_OP_STRESS_DET : GINI_OP_STRESS, n, 0, k, 0))
    return GINI_ENOMEM;
  cudaStream_t s = (cudaStream_t)stream;
  IterWs w = carve(ws, n, k, 1, det);
  IterParams Q = make_params(n, k, nu, Y_dev, delta_dev, ldd, col_scale_dev, w);
  Q.metric = metric;
  Q.loss = loss;
  cudaError_t e = cudaMemsetAsync(w.acc, 0, sizeof(double) * STRESS_SLOTS, s);
  if (e == cudaSuccess && grad_dev) e = cudaMemsetAsync(w.h, 0, sizeof(float) * n * k, s);
  if (e != cudaSuccess) { gini_set_cuda_error(e); return GINI_ECUDA; }
  prep(k, Y_dev, n, w.P, w.Y4, w.err, s);
  one_pass(k, layout, dtype, grad_dev != nullptr, Q, s);
  gini_count_launch(grad_dev ? 2 : 1);
  k_finalize_stress<<<1, 32, 0, s>>>(w.acc, 1, 1.0 / norm, nullptr, stress_dev);  // one warp
  if (grad_dev)
    k_finalize_grad<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(
        w.h, n, k, (float)(2.0 / norm), Q.tab.c2, scalar2_path(k, metric, loss), grad_dev);
  e = cudaGetLastError();
  if (e != cudaSuccess) { gini_set_cuda_error(e); return GINI_ECUDA; }
  return GINI_OK;
}

extern "C" int gini_stress_grad(const float* Y_dev, int64_t n, int k, double nu,
                                const void* delta_dev, int layout, int dtype, int64_t ldd,
                                const float* col_scale_dev, double sum_delta2, double* stress_dev,
                                float* grad_dev, void* ws, size_t ws_bytes, void* stream) {
  return gini_stress_grad_ex(Y_dev, n, k, nu, delta_dev, layout, dtype, ldd, col_scale_dev,
                             GINI_METRIC_GINI, GINI_LOSS_KRUSKAL, sum_delta2, stress_dev,
                             grad_dev, ws, ws_bytes, stream);
}

extern "C" int gini_mds_fit(const gini_fit_args* a, void* ws, size_t ws_bytes, void* stream) {
  NvtxRange nvtx_range("gini_mds_fit");
  if (!a || !ws || !a->Y_dev) return GINI_EINVAL;
  if (ws_misaligned(ws)) return GINI_EINVAL;
  int st = check_common(a->n, a->k, a->nu, a->delta_dev, a->layout, a->dtype, a->ldd,
                        a->col_scale_dev, a->sum_delta2);
  if (st != GINI_OK) return st;
  if (a->iters < 0 || !(a->eta > 0.0) || !isfinite(a->eta) || a->polish_iters < 0)
    return GINI_EINVAL;
  if (a->metric != GINI_METRIC_GINI && a->metric != GINI_METRIC_EUCLID) return GINI_EINVAL;
  if (a->loss != GINI_LOSS_KRUSKAL && a->loss != GINI_LOSS_SAMMON) return GINI_EINVAL;
  const bool det = (a->deterministic || gini_get_deterministic()) &&
                   a->layout == GINI_LAYOUT_TILED && a->iters > 0;
  if (ws_bytes < gini_workspace_size(det ? GINI_OP_FIT_DET : GINI_OP_FIT, a->n, 0, a->k, a->iters))
    return GINI_ENOMEM;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = a->n;
  const int k = a->k;
  const int T = a->iters;
  IterWs w = carve(ws, n, k, T + 1, det);
  IterParams Q = make_params(n, k, a->nu, a->Y_dev, a->delta_dev, a->ldd, a->col_scale_dev, w);
  Q.metric = a->metric;
  Q.loss = a->loss;
  const bool sc2 = scalar2_path(k, a->metric, a->loss);
  cudaError_t e = cudaMemsetAsync(w.acc, 0, sizeof(double) * (size_t)(T + 1) * STRESS_SLOTS, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(w.h, 0, sizeof(float) * n * k, s);
  if (e != cudaSuccess) { gini_set_cuda_error(e); return GINI_ECUDA; }
  prep(k, a->Y_dev, n, w.P, w.Y4, w.err, s);
  const float scale = (float)(a->eta * 2.0 / a->sum_delta2);
  const int polish_from = T - (a->polish_iters < T ? a->polish_iters : T);
  for (int t = 0; t < T; ++t) {
    int dt = a->dtype;
    if (dt == GINI_BF16X2 && a->layout == GINI_LAYOUT_TILED && t < polish_from) dt = GINI_BF16;
    Q.stress = w.acc + (size_t)t * STRESS_SLOTS;
    one_pass(k, a->layout, dt, true, Q, s);
    update(k, a->Y_dev, n, w.P, w.Y4, w.h, scale, Q.tab.c2, sc2, w.err, s);
  }
  Q.stress = w.acc + (size_t)T * STRESS_SLOTS;
  one_pass(k, a->layout, a->dtype, false, Q, s);
  gini_count_launch(1);
  k_finalize_stress<<<(unsigned)((T + 1 + 7) / 8), 256, 0, s>>>(
      w.acc, T + 1, 1.0 / a->sum_delta2, a->history_dev, a->final_stress_dev);
  e = cudaGetLastError();
  if (e != cudaSuccess) { gini_set_cuda_error(e); return GINI_ECUDA; }
  return GINI_OK;
}
