// Dissimilarity matrix build: Delta_q(i, j) = Dbar_{G,nu_q}(x_i, x_j)
// (Section III-B, symmetrized generalized Gini pseudo-distance; Algorithm 1).
//
// Per pair (i, j), i < j, one segment of L lanes:
//   z = x_i - x_j as the TwoSum pair (hi, lo)   (E registers per lane)
//   sort z ascending in its exact order          (register sorting network on
//                                                 64-bit (hi, lo) keys)
//   2R(pos) = first + last position of pos's tie run, + 2   (midranks)
//   delta_q = sum_pos hi(pos) * T_q[2R - 2],  T_q = (d/2) W_{d,nu_q}
// One sort serves every nu.  For a single nu = 2 the weight is affine in the
// rank, (d/2) W = R - (d+1)/2: a tie run's midrank weight equals the mean of its
// positional weights, and equal FP32 values give the same sum in any order, so
// that case sorts the FP32 values and skips the run bookkeeping.  So does a
// single nu = 3, whose weight is the same affine function times (d-1)/d.
//
// Work split: CTA = 8 warps = 8 consecutive rows i; blockIdx.x picks a block
// of CB columns j.  A warp keeps x_i in shared memory (in registers it would
// cost the 32 registers that let two CTAs share an SM) and walks its columns,
// each of the 32/L segments taking every (32/L)-th j.  X is read through L2 (a
// row is a few KB; the per-pair compute dwarfs the traffic).
#include <float.h>
#include <math.h>
#include <stdio.h>

#include <vector>

#include "common.cuh"
#include "sortnet.cuh"

namespace gini {

constexpr int DIST_WARPS = 8;
constexpr int NU_MAX = 8;

struct DistParams {
  const float* X;
  int64_t n, m, ldx;
  int n_nu;
  const float* wtab;  // n_nu x (2m - 1), T_q[idx], idx = first + last position
  int layout, dtype;
  void* out;
  int64_t ldd, nu_stride;
  int64_t tiles;      // tiles along one edge (TILED)
  int64_t plane;      // elements in one plane (TILED)
  double* sum_delta2;
  unsigned* err;
  int cb;             // columns per CTA
  float affine_scale; // affine path: (d/2) W / (R - (d+1)/2), 1 for nu = 2, (d-1)/d for nu = 3
};

__device__ __forceinline__ void store_delta(const DistParams& P, int q, int64_t i, int64_t j,
                                            float d) {
  if (P.layout == GINI_LAYOUT_FULL) {
    float* o = reinterpret_cast<float*>(P.out) + (int64_t)q * P.nu_stride;
    o[i * P.ldd + j] = d;
    o[j * P.ldd + i] = d;
    return;
  }
  const int64_t idx = (int64_t)q * P.nu_stride + tiled_index(i, j, P.tiles);
  if (P.dtype == GINI_F32) {
    reinterpret_cast<float*>(P.out)[idx] = d;
  } else if (P.dtype == GINI_BF16) {
    reinterpret_cast<__nv_bfloat16*>(P.out)[idx] = __float2bfloat16_rn(d);
  } else {  // GINI_BF16X2
    __nv_bfloat16 hi = __float2bfloat16_rn(d);
    __nv_bfloat16 lo = __float2bfloat16_rn(d - __bfloat162float(hi));
    reinterpret_cast<__nv_bfloat16*>(P.out)[idx] = hi;
    reinterpret_cast<__nv_bfloat16*>(P.out)[idx + P.plane] = lo;
  }
}

// Order-preserving 32-bit image of a float (ascending as unsigned integers)
// and its inverse.
__device__ __forceinline__ unsigned ord_bits(float f) {
  const unsigned b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float unord_bits(unsigned k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// a + c as the TwoSum pair (hi, lo), hi = fl(a + c), hi + lo = a + c exactly;
// -0 is replaced by +0 in both parts so equal values have equal bits.
__device__ __forceinline__ float2 two_sum_canonical(float a, float c) {
  const float hi = __fadd_rn(a, c);
  const float bb = __fsub_rn(hi, a);
  const float lo = __fadd_rn(__fsub_rn(a, __fsub_rn(hi, bb)), __fsub_rn(c, bb));
  return make_float2(__fadd_rn(hi, 0.f), __fadd_rn(lo, 0.f));
}

// Skewed shared-memory address of table entry idx: sorted positions of one
// lane are E apart, so idx ~ 2*E*ls + 2t; adding idx / (2E) spreads the lanes
// of a segment over distinct banks.
template <int E>
__device__ __forceinline__ int tab_addr(int idx) {
  return idx + (idx / (2 * E));
}

// TL, TR (affine path): registers t < TL hold a real element in every lane
// (t*L + ls < m), registers t >= TR none.
template <int E, int L, bool AFFINE, int TL, int TR>
__device__ __forceinline__ void dist_body(const DistParams& P) {
  constexpr int G = 32 / L;
  constexpr int NQ = AFFINE ? 1 : NU_MAX;  // nu slots carried in registers
  extern __shared__ float s_tab[];  // n_nu x tab_stride
  __shared__ double s_red[DIST_WARPS][NU_MAX];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int seg = lane / L, ls = lane % L;
  const int64_t row0 = (int64_t)blockIdx.y * DIST_WARPS;
  const int64_t col0 = (int64_t)blockIdx.x * P.cb;
  // Nothing above the diagonal in this block (uniform exit, before any barrier).
  if (col0 + P.cb - 1 <= row0 || row0 >= P.n - 1) return;

  const int m = (int)P.m;
  const int tab_n = 2 * m - 1;
  const int tab_stride = tab_addr<E>(tab_n - 1) + 1;
  if (!AFFINE) {
    for (int q = 0; q < P.n_nu; ++q)
      for (int idx = threadIdx.x; idx < tab_n; idx += blockDim.x)
        s_tab[q * tab_stride + tab_addr<E>(idx)] = P.wtab[(int64_t)q * tab_n + idx];
    __syncthreads();
  }

  // Affine path: sorted-position weights of the alternating layout, per
  // (segment lane, register), zero at padding; rows padded to E + 4 floats so
  // that the 16-byte reads of a quarter-warp fall in distinct banks.
  __shared__ __align__(16) float s_cw[AFFINE ? L : 1][AFFINE ? E + 4 : 4];
  if constexpr (AFFINE) {
    // padding of odd lanes (negated, so at the bottom of the sorted sequence)
    int n_lo = 0;
    if (L >= 2)
      for (int l = 1; l < L; l += 2) n_lo += E - min(E, m > l ? (m - l + L - 1) / L : 0);
    const float mid = 0.5f * (float)(m - 1);
    for (int idx = threadIdx.x; idx < L * E; idx += blockDim.x) {
      const int l = idx / E, t = idx % E;
      const bool odd = L >= 2 && (l & 1);
      const int pos = E * l + (odd ? E - 1 - t : t) - n_lo;  // rank among real elements
      s_cw[l][t] = (pos >= 0 && pos < m) ? (odd ? -1.f : 1.f) * ((float)pos - mid) : 0.f;
    }
  }

  const int64_t i = row0 + warp;
  const bool row_ok = i < P.n - 1;
  __shared__ float s_xi[DIST_WARPS][E * L];
#pragma unroll
  for (int t = 0; t < E; ++t) {
    const int e = t * L + ls;
    float x = (row_ok && e < m) ? __ldg(P.X + i * P.ldx + e) : 0.f;
    // affine path: stored with the sign of the lanes that read it (e and ls
    // have the same parity when L is even)
    if (AFFINE && L >= 2 && (e & 1)) x = -x;
    if (seg == 0) s_xi[warp][e] = x;
  }
  if constexpr (AFFINE) __syncthreads(); else __syncwarp();

  // sum of delta^2 per nu: in registers for the affine path (one nu); in
  // shared memory, one slot per segment, for the generic path, where eight
  // FP64 registers held across the sort would cost its occupancy
  constexpr int NR = AFFINE ? 1 : 0;
  double sd2[NR > 0 ? NR : 1];
  sd2[0] = 0.0;
  __shared__ double s_sd2[AFFINE ? 1 : DIST_WARPS][AFFINE ? 1 : G][NU_MAX];
  if constexpr (!AFFINE) {
    for (int idx = threadIdx.x; idx < DIST_WARPS * G * NU_MAX; idx += blockDim.x)
      (&s_sd2[0][0][0])[idx] = 0.0;
    __syncthreads();
  }

  for (int64_t jb = col0; jb < col0 + P.cb; jb += G) {
    const int64_t j = jb + seg;
    const bool active = row_ok && j > i && j < P.n;
    if (!__any_sync(FULL_MASK, active)) continue;
    float acc[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[q] = 0.f;
    const int pos0 = E * ls;
    if constexpr (AFFINE) {
      // nu = 2: (d/2) W(R) = R - (d+1)/2 is affine in the rank (nu = 3: the
      // same times (d-1)/d, applied to the sum), so the order of equal FP32
      // differences does not change the sum: FP32 keys suffice.
      // u = s0 (x_i - x_j) with the lane's sign s0 (alternating layout),
      // padded with FLT_MAX (weight 0; a real difference equal to it would
      // carry the same value in whichever slot it lands).
      const float nsg = (L >= 2 && (ls & 1)) ? 1.f : -1.f;  // -s0
      float u[E];
#pragma unroll
      for (int t = 0; t < E; ++t) {
        const int e = t * L + ls;
        if (t < TR) {
          const bool real = t < TL || e < m;
          const float xj = (active && real) ? __ldg(P.X + j * P.ldx + e) : 0.f;
          u[t] = real ? fmaf(nsg, xj, s_xi[warp][e]) : FLT_MAX;
        } else {
          u[t] = FLT_MAX;
        }
      }
      seg_sort_alternating<E, L, TR>(u, ls);
      float2 acc2 = make_float2(0.f, 0.f);
#pragma unroll
      for (int t = 0; t < E; t += 4) {
        const float4 c = *reinterpret_cast<const float4*>(&s_cw[ls][t]);
        acc2 = __ffma2_rn(make_float2(u[t], u[t + 1]), make_float2(c.x, c.y), acc2);
        acc2 = __ffma2_rn(make_float2(u[t + 2], u[t + 3]), make_float2(c.z, c.w), acc2);
      }
      acc[0] = (acc2.x + acc2.y) * P.affine_scale;
    } else {
      // Weights that are not affine in the rank: the order must be that of the
      // exact differences.  Each difference is the TwoSum pair (hi, lo),
      // hi + lo = x_i - x_j exactly, ordered lexicographically through one
      // 64-bit key; distinct differences that round to the same FP32 value stay
      // distinct, equal keys are exact ties.  The sum uses hi.
      unsigned long long kv[E];
#pragma unroll
      for (int t = 0; t < E; ++t) {
        const int e = t * L + ls;
        if (e < m) {
          const float a = s_xi[warp][e];
          const float c = active ? -__ldg(P.X + j * P.ldx + e) : 0.f;
          const float2 hl = two_sum_canonical(a, c);
          kv[t] = ((unsigned long long)ord_bits(hl.x) << 32) | ord_bits(hl.y);
        } else {
          kv[t] = ~0ull;  // padding above every real key
        }
      }
      seg_bitonic_sort<E, L>(kv, ls);
      // A tie run holds equal keys, so one hi: its members' terms sum to
      // count * hi * T_q[first + last], added once at the run's last entry
      // (in the lane that holds it; s is the run's first position).
      bool cont_right;
      int s = seg_first_run_start<E, L>(
          kv, ls, [](unsigned long long a, unsigned long long b) { return a == b; }, cont_right);
#pragma unroll
      for (int t = 0; t < E; ++t) {
        if (t > 0 && kv[t] != kv[t - 1]) s = pos0 + t;
        const bool last = (t < E - 1) ? (kv[t] != kv[t + 1]) : !cont_right;
        const int pos = pos0 + t;
        if (last && pos < m) {  // padding (positions >= m) forms runs of its own
          const float hi = unord_bits((unsigned)(kv[t] >> 32));
          const float w = hi * (float)(pos - s + 1);
          const int a = tab_addr<E>(s + pos);
#pragma unroll
          for (int q = 0; q < NQ; ++q)
            if (q < P.n_nu) acc[q] = fmaf(w, s_tab[q * tab_stride + a], acc[q]);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      if (q < P.n_nu) {
#pragma unroll
        for (int o = L / 2; o >= 1; o >>= 1) acc[q] += __shfl_xor_sync(FULL_MASK, acc[q], o);
      }
    }
    if (active && ls == 0) {
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        if (q < P.n_nu) {
          store_delta(P, q, i, j, acc[q]);
          const double d2 = (double)acc[q] * (double)acc[q];
          if constexpr (AFFINE) sd2[0] += d2;
          else s_sd2[warp][seg][q] += d2;
        }
      }
    }
  }

  // sum_{i<j} delta^2: warp (or segment slots), then CTA, then one FP64
  // atomic per nu.
  if constexpr (AFFINE) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) sd2[0] += __shfl_xor_sync(FULL_MASK, sd2[0], o);
    if (lane == 0) s_red[warp][0] = sd2[0];
  }
  __syncthreads();
  if (threadIdx.x < P.n_nu && P.sum_delta2) {
    double s = 0.0;
    for (int w = 0; w < DIST_WARPS; ++w) {
      if constexpr (AFFINE) s += s_red[w][threadIdx.x];
      else
        for (int g = 0; g < G; ++g) s += s_sd2[w][g][threadIdx.x];
    }
    if (s != 0.0) atomicAdd(P.sum_delta2 + threadIdx.x, s);
  }
}

// Entry points.  The affine kernel fits three CTAs per SM as compiled; the
// generic one is bounded to two (128 registers, a few spilled) instead of the
// one CTA its 64-bit network would otherwise take.
template <int E, int L, int TL, int TR>
__global__ void __launch_bounds__(DIST_WARPS * 32) k_dist(const DistParams P) {
  dist_body<E, L, true, TL, TR>(P);
}

template <int E, int L>
__global__ void __launch_bounds__(DIST_WARPS * 32, 2) k_dist_exact(const DistParams P) {
  dist_body<E, L, false, E, E>(P);
}

__global__ void k_check_finite(const float* X, int64_t n, int64_t m, int64_t ld, unsigned* err) {
  bool bad = false;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * m;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / m, c = e % m;
    bad |= !isfinite(X[r * ld + c]);
  }
  if (__any_sync(FULL_MASK, bad) && (threadIdx.x & 31) == 0) raise_error(err, ERR_NONFINITE);
}

__global__ void k_zero_diag(float* D, int64_t n, int64_t ldd, int64_t nu_stride, int n_nu) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n)
    for (int q = 0; q < n_nu; ++q) D[(int64_t)q * nu_stride + i * ldd + i] = 0.f;
}

template <int E, int L, bool AFFINE, int TL, int TR>
static auto dist_kernel() {
  if constexpr (AFFINE) return k_dist<E, L, TL, TR>;
  else return k_dist_exact<E, L>;
}

template <int E, int L, bool AFFINE, int TL = E, int TR = E>
static cudaError_t launch_dist(const DistParams& P, cudaStream_t s) {
  void (*kern)(const DistParams) = dist_kernel<E, L, AFFINE, TL, TR>();
  const int m = (int)P.m;
  const int tab_n = 2 * m - 1;
  const int tab_stride = tab_n - 1 + (tab_n - 1) / (2 * E) + 1;
  const size_t smem = AFFINE ? 0 : (size_t)P.n_nu * tab_stride * sizeof(float);
  // static (x_i rows) + dynamic (weight tables) may pass the 48 KB default
  if (smem > 0) {
    cudaError_t e = cudaFuncSetAttribute(kern,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  DistParams Q = P;
  constexpr int G = 32 / L;
  // Columns per CTA (several passes per warp): more of them amortise the CTA's
  // setup (weight table, x_i rows) where the grid stays many waves deep --
  // large n, or narrow segments with many pairs per warp.
  const bool wide = P.n >= 8192 || L < 8;
  Q.cb = G * (L >= 8 ? (wide ? 64 : 16) : (wide ? 16 : 4));
  dim3 grid((unsigned)((P.n + Q.cb - 1) / Q.cb), (unsigned)((P.n + DIST_WARPS - 1) / DIST_WARPS));
  gini_count_launch(1);
  kern<<<grid, DIST_WARPS * 32, smem, s>>>(Q);
  return cudaGetLastError();
}

// Generic keys (nu != 2): one instantiation per power-of-two segment size.
static cudaError_t dispatch_dist_exact(const DistParams& P, cudaStream_t s) {
  const int64_t m = P.m;
  if (m <= 4) return launch_dist<4, 1, false>(P, s);
  if (m <= 8) return launch_dist<8, 1, false>(P, s);
  if (m <= 16) return launch_dist<16, 1, false>(P, s);
  if (m <= 32) return launch_dist<32, 1, false>(P, s);
  if (m <= 64) return launch_dist<32, 2, false>(P, s);
  if (m <= 128) return launch_dist<32, 4, false>(P, s);
  if (m <= 256) return launch_dist<32, 8, false>(P, s);
  if (m <= 512) return launch_dist<32, 16, false>(P, s);
  return launch_dist<32, 32, false>(P, s);
}

// Affine (nu = 2): as above, with the bounds TL, TR on the real registers of
// each segment size (m in (E*L/2, E*L] fills every register below E/2), and
// the 32-lane segments split further by m so that the in-lane sort skips the
// comparators of registers that only ever hold padding (m = 784: 25 of 32).
static cudaError_t dispatch_dist_affine(const DistParams& P, cudaStream_t s) {
  const int64_t m = P.m;
  if (m <= 4) return launch_dist<4, 1, true, 1, 4>(P, s);
  if (m <= 8) return launch_dist<8, 1, true, 4, 8>(P, s);
  if (m <= 16) return launch_dist<16, 1, true, 8, 16>(P, s);
  if (m <= 32) return launch_dist<32, 1, true, 16, 32>(P, s);
  if (m <= 64) return launch_dist<32, 2, true, 16, 32>(P, s);
  if (m <= 128) return launch_dist<32, 4, true, 16, 32>(P, s);
  if (m <= 256) return launch_dist<32, 8, true, 16, 32>(P, s);
  if (m <= 512) return launch_dist<32, 16, true, 16, 32>(P, s);
  if (m <= 640) return launch_dist<32, 32, true, 16, 20>(P, s);
  if (m <= 800) return launch_dist<32, 32, true, 20, 25>(P, s);
  if (m <= 896) return launch_dist<32, 32, true, 25, 28>(P, s);
  return launch_dist<32, 32, true, 28, 32>(P, s);
}

}  // namespace gini

using namespace gini;

extern "C" void gini_set_cuda_error(cudaError_t e);

extern "C" int gini_dist(const float* X_dev, int64_t n, int64_t p, int64_t ldx,
                         const double* nu_host, int n_nu, int layout, int dtype, void* delta_dev,
                         int64_t ldd, int64_t nu_stride, double* sum_delta2_dev, void* ws,
                         size_t ws_bytes, void* stream) {
  if (!X_dev || !delta_dev || !nu_host || !ws) return GINI_EINVAL;
  if (ws_misaligned(ws)) return GINI_EINVAL;
  if (n < 2 || p < 1 || p > 1024 || ldx < p || n_nu < 1 || n_nu > NU_MAX) return GINI_EINVAL;
  if (n > (int64_t)65535 * DIST_WARPS) return GINI_EINVAL;  // grid.y = ceil(n / 8)
  for (int q = 0; q < n_nu; ++q)
    if (!(nu_host[q] > 1.0) || !isfinite(nu_host[q])) return GINI_EINVAL;
  if (layout == GINI_LAYOUT_FULL) {
    if (dtype != GINI_F32 || ldd < n) return GINI_EINVAL;
    if (n_nu > 1 && nu_stride < ldd * n) return GINI_EINVAL;
  } else if (layout == GINI_LAYOUT_TILED) {
    if (dtype != GINI_F32 && dtype != GINI_BF16 && dtype != GINI_BF16X2) return GINI_EINVAL;
    const int64_t plane = gini_tiled_elems(n);
    if (n_nu > 1 && nu_stride < plane * (dtype == GINI_BF16X2 ? 2 : 1)) return GINI_EINVAL;
  } else {
    return GINI_EINVAL;
  }
  if (ws_bytes < gini_workspace_size(GINI_OP_DIST, n, p, 0, 0)) return GINI_ENOMEM;

  cudaStream_t s = (cudaStream_t)stream;
  unsigned* err = reinterpret_cast<unsigned*>(ws);
  float* wtab = reinterpret_cast<float*>(reinterpret_cast<char*>(ws) + WS_HEADER);
  // W_{d,nu} is affine in the rank for nu = 2 and nu = 3:
  // (d/2) W_{d,3}(R) = ((d-1)/d) (R - (d+1)/2) = ((d-1)/d) (d/2) W_{d,2}(R)
  const bool affine = (n_nu == 1 && (nu_host[0] == 2.0 || nu_host[0] == 3.0));
  const int tab_n = (int)(2 * p - 1);
  if (!affine) {
    // T_q[idx] = (d/2) W_{d,nu_q}((idx + 2)/2), W(R) = ((R-1)/d)^{nu-1} - ((d-R)/d)^{nu-1}
    std::vector<float> tab((size_t)n_nu * tab_n);
    const double d = (double)p;
    for (int q = 0; q < n_nu; ++q)
      for (int idx = 0; idx < tab_n; ++idx) {
        const double R = (idx + 2) / 2.0;
        const double W = pow((R - 1.0) / d, nu_host[q] - 1.0) - pow((d - R) / d, nu_host[q] - 1.0);
        tab[(size_t)q * tab_n + idx] = (float)(0.5 * d * W);
      }
    // From pageable memory the copy is staged before cudaMemcpyAsync returns,
    // so `tab` may be released right after the call.
    cudaError_t e = cudaMemcpyAsync(wtab, tab.data(), tab.size() * sizeof(float),
                                    cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) { gini_set_cuda_error(e); return GINI_ECUDA; }
  }
  cudaError_t e = cudaSuccess;
  if (sum_delta2_dev) e = cudaMemsetAsync(sum_delta2_dev, 0, sizeof(double) * n_nu, s);
  if (e == cudaSuccess) {
    gini_count_launch(1);
    k_check_finite<<<296, 256, 0, s>>>(X_dev, n, p, ldx, err);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && layout == GINI_LAYOUT_FULL) {
    gini_count_launch(1);
    k_zero_diag<<<(unsigned)((n + 255) / 256), 256, 0, s>>>((float*)delta_dev, n, ldd,
                                                           nu_stride, n_nu);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    DistParams P{};
    P.X = X_dev; P.n = n; P.m = p; P.ldx = ldx; P.n_nu = n_nu; P.wtab = wtab;
    P.layout = layout; P.dtype = dtype; P.out = delta_dev; P.ldd = ldd; P.nu_stride = nu_stride;
    P.tiles = tiles_1d(n); P.plane = gini_tiled_elems(n);
    P.sum_delta2 = sum_delta2_dev; P.err = err;
    P.affine_scale = (affine && nu_host[0] == 3.0) ? (float)((double)(p - 1) / (double)p) : 1.f;
    e = affine ? dispatch_dist_affine(P, s) : dispatch_dist_exact(P, s);
  }
  if (e != cudaSuccess) { gini_set_cuda_error(e); return GINI_ECUDA; }
  return GINI_OK;
}
