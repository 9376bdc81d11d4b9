// Dissimilarity matrix build: Delta_q(i, j) = Dbar_{G,nu_q}(x_i, x_j)
// (Section III-B, symmetrized generalized Gini pseudo-distance; Algorithm 1).
//
// Per pair (i, j), i < j, one segment of L lanes (E registers per lane):
//   order the p differences z_a = x_ia - x_ja exactly (register sorting network)
//   2R(pos) = first + last position of pos's tie run, + 2   (midranks)
//   delta_q = sum_pos v(pos) * T_q[2R - 2],  T_q = (d/2) W_{d,nu_q}
// One sort serves every nu.  Three kernels share this structure:
//
//   k_dist        a single nu = 2 or 3.  The weight is affine in the rank
//                 ((d/2) W = R - (d+1)/2 for nu = 2, (d-1)/d times that for
//                 nu = 3), so a tie run's midrank weight is the mean of its
//                 positional weights and equal FP32 values give the same sum in
//                 any order: FP32 keys, positional weights, no run bookkeeping.
//   k_dist_keyed  every other nu.  Each difference becomes a 32-bit cell key:
//                 with RD and RU the FP32 roundings of z down and up, the key's
//                 magnitude is bits(|RD|) + bits(|RU|) -- twice the grid index
//                 of z when z is an FP32 value, the odd number between the two
//                 grid indices when z lies strictly between them -- and its sign
//                 is z's.  Read as a float it orders like z, so the FP32 network
//                 of k_dist sorts it.  Equal keys are exact ties, except for two
//                 inexact differences in one FP32 cell (an odd key); such runs
//                 (rare) are re-ordered by their TwoSum residuals in the same
//                 warp.  The sum uses the cell's end nearer zero (within one
//                 FP32 ulp of z).
//   k_dist_exact  the 64-bit (hi, lo) TwoSum key network, which runs instead
//                 of k_dist_keyed when the data's range would make the keys'
//                 scaling inexact (decided on the device by a pre-pass over X).
//
// Sum delta^2 is accumulated exactly: each CTA's FP64 partial, in units of a
// power of two fixed by the pre-pass, goes into a 128-bit integer with 64-bit
// atomics, so the result does not depend on the order the CTAs finish in.
//
// Work split: CTA = 8 warps = 8 consecutive rows i; blockIdx.x picks a block
// of CB columns j.  A warp keeps x_i in shared memory (in registers it would
// cost the 32 registers that let two CTAs share an SM) and walks its columns,
// each of the 32/L segments taking every (32/L)-th j.  X is read through L2 (a
// row is a few KB; the per-pair compute dwarfs the traffic).
#include <float.h>
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <vector>

#define GINI_FILE_ID 1  // site numbers of the debug index checks
#include "common.cuh"
#include "sortnet.cuh"

namespace gini {

constexpr int DIST_WARPS = 8;
constexpr int NU_MAX = 8;
// Internal layout of the FP8 output's column strips (see gini_dist).
constexpr int LAYOUT_STRIP = 2;

// Summary of X and the constants derived from it, kept in gini_dist's
// workspace right after the error word.  The three extrema are gathered with
// atomicMax on zero-filled words (minima as complements), so they are exact
// and independent of the order of the atomics.
struct DistState {
  unsigned max_ord;      // max over X of ord_bits(x)
  unsigned inv_min_ord;  // max over X of ~ord_bits(x): the minimum of X
  unsigned inv_min_nz;   // max over nonzero x of ~bits(|x|): the smallest nonzero |x|
  int fallback;          // 1: k_dist_keyed's scaled keys would be inexact; k_dist_exact runs
  float key_scale;       // 2^s, s <= 0, with (max X - min X) 2^s <= 1
  int sd2_q;             // Sum delta^2 is accumulated in units of 2^sd2_q
  int pad_[2];
  unsigned long long sd2[NU_MAX][2];  // (low, high) 64-bit words per nu
};
constexpr size_t DIST_STATE_BYTES = 256;
static_assert(sizeof(DistState) <= DIST_STATE_BYTES, "DistState must fit its region");

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
  DistState* st;
  int64_t col_begin, col_end;  // columns j built by this launch (a strip for FP8 output)
  int cb;             // columns per CTA
  float affine_scale; // affine path: (d/2) W / (R - (d+1)/2), 1 for nu = 2, (d-1)/d for nu = 3
};

// Adds v >= 0 exactly (up to truncation below 2^q, the same for every order)
// to the 128-bit integer acc[0] + 2^64 acc[1] counting units of 2^q.  With the
// pre-pass's q every CTA partial is below 2^(q + 126).  Integer addition is
// associative, so the total does not depend on the order of the atomics.
__device__ __forceinline__ void add_exact128(unsigned long long* acc, double v, int q) {
  if (!(v > 0.0)) return;                  // zero, or NaN from non-finite input
  const double x = ldexp(v, -q);           // exact scaling
  const double hi = floor(ldexp(x, -64));
  const double lo = x - ldexp(hi, 64);     // x mod 2^64: at most 53 significant bits, exact
  const unsigned long long l = __double2ull_rz(lo), h = __double2ull_rz(hi);
  const unsigned long long old = atomicAdd(acc, l);
  atomicAdd(acc + 1, h + ((old + l < old) ? 1ull : 0ull));
}

__device__ __forceinline__ void store_delta(const DistParams& P, int q, int64_t i, int64_t j,
                                            float d) {
  // (debug builds) matrix q of the call, 0 <= i < j < n
  if (!(GINI_IDX_OK(P.err, q, P.n_nu) && GINI_IDX_OK(P.err, j, P.n) && GINI_IDX_OK(P.err, i, j)))
    return;
  if (P.layout == GINI_LAYOUT_FULL) {
    float* o = reinterpret_cast<float*>(P.out) + (int64_t)q * P.nu_stride;
    if (!(GINI_IDX_OK(P.err, j, P.ldd))) return;
    o[i * P.ldd + j] = d;
    o[j * P.ldd + i] = d;
    return;
  }
  if (P.layout == LAYOUT_STRIP) {  // FP32 rows 0..n-1 of columns col_begin .. col_begin+ldd-1
    if (!(GINI_IDX_OK(P.err, j - P.col_begin, P.ldd))) return;
    reinterpret_cast<float*>(P.out)[(int64_t)q * P.nu_stride + i * P.ldd + (j - P.col_begin)] = d;
    return;
  }
  if (!(GINI_IDX_OK(P.err, tiled_index(i, j, P.tiles), P.plane))) return;
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
  const int64_t col0 = P.col_begin + (int64_t)blockIdx.x * P.cb;
  // Nothing above the diagonal in this block (uniform exit, before any barrier).
  if (col0 + P.cb - 1 <= row0 || row0 >= P.n - 1) return;
  // The 64-bit network runs only where the pre-pass flagged the keyed kernel.
  if (!AFFINE && !P.st->fallback) return;

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
  // (segment lane, register), zero at padding.  A row holds CWS >= E floats,
  // an odd multiple of 4 (20 for E = 20; 28 for 24, 25, 28; 36 for 32), so
  // that the rows of 8 consecutive lanes start in 8 distinct groups of 4 banks
  // and the 16-byte reads of a quarter-warp do not conflict.
  constexpr int CWS = ((E + 3) / 4) % 2 ? (E + 3) / 4 * 4 : (E + 3) / 4 * 4 + 4;
  __shared__ __align__(16) float s_cw[AFFINE ? L : 1][AFFINE ? CWS : 4];
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
    const bool active = row_ok && j > i && j < P.col_end && GINI_IDX_OK(P.err, j, P.n);
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
      for (int t = 0; t + 3 < E; t += 4) {
        const float4 c = *reinterpret_cast<const float4*>(&s_cw[ls][t]);
        acc2 = __ffma2_rn(make_float2(u[t], u[t + 1]), make_float2(c.x, c.y), acc2);
        acc2 = __ffma2_rn(make_float2(u[t + 2], u[t + 3]), make_float2(c.z, c.w), acc2);
      }
#pragma unroll
      for (int t = E / 4 * 4; t < E; ++t) acc2.x = fmaf(u[t], s_cw[ls][t], acc2.x);
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
          const bool tab_ok = GINI_IDX_OK(P.err, s + pos, 2 * P.m - 1);
#pragma unroll
          for (int q = 0; q < NQ; ++q)
            if (q < P.n_nu && tab_ok) acc[q] = fmaf(w, s_tab[q * tab_stride + a], acc[q]);
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

  // sum_{i<j} delta^2: warp (or segment slots), then CTA in a fixed order,
  // then the exact 128-bit accumulator of each nu.
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
    add_exact128(P.st->sd2[threadIdx.x], s, P.st->sd2_q);
  }
}

// Cell key of one difference for k_dist_keyed, as a float.  a = c x_i and
// b = -c x_j, c = +-2^s exact (the pre-pass guarantees no underflow), so
// RD and RU below are the roundings down and up of c (x_i - x_j).  The key's
// bits are bits(RD) + bits(RU) (mod 2^32) with the sign bit flipped when RD
// is negative:
//   z an FP32 value, z > 0:  2 bits(z);  z < 0: -(2 bits(|z|));  z = 0: +0
//   z strictly inside the cell (g, g+): 2 bits(|g|) + 1 with the sign of z,
//   g the cell end nearer zero
// so keys order like the exact z, equal keys are equal values unless the key
// is odd, and K(-z) = -K(z).  (|c z| <= 1 keeps the magnitude <= 2 bits(1.0) =
// 0x7F000000, a finite float below FLT_MAX, the padding value.)
__device__ __forceinline__ float cell_key(float c, float xi_scaled, float xj) {
  const float rd = __fmaf_rd(c, xj, xi_scaled), ru = __fmaf_ru(c, xj, xi_scaled);
  const unsigned b = __float_as_uint(rd);
  return __uint_as_float((b + __float_as_uint(ru)) ^ (b & 0x80000000u));
}

// The cell end nearer zero of a key's value (scaled by c), with its sign.
__device__ __forceinline__ float cell_value(float key) {
  const unsigned b = __float_as_uint(key);
  return __uint_as_float(((b & 0x7fffffffu) >> 1) | (b & 0x80000000u));
}

// Exact (hi, lo) order key of x_i - x_j (64-bit, lexicographic), for the rare
// runs whose cell keys tie although the differences do not.
__device__ __forceinline__ unsigned long long exact_key(float xi, float xj) {
  const float2 hl = two_sum_canonical(xi, -xj);
  return ((unsigned long long)ord_bits(hl.x) << 32) | ord_bits(hl.y);
}

// One ambiguous run of k_dist_keyed: the c >= 2 sorted entries at real
// positions f .. f+c-1 share the odd key K (inexact differences in one FP32
// cell), so they were weighted as one tie run.  Their exact order is that of
// the TwoSum pairs of x_i - x_j: each member m gets the midrank of its own tie
// group, first + last = 2 (f + lt_m) + eq_m - 1 (lt_m members below it, eq_m
// equal to it, itself included).  The difference to the tie-run weights is
// added to corr[q] (lane 0 of the segment).  Every lane of the warp calls this
// (shuffles); `have` is false in segments without a pending run.  The loops
// recompute the members from X, so nothing from the sort is kept; the work is
// O(c p) per run, and such runs are rare.
template <int E, int L>
__device__ __noinline__ void keyed_fix_run(const DistParams& P, const float* s_tab,
                                           int tab_stride, int64_t i, int64_t j, int ls,
                                           bool have, float K, int f, int c, float* corr) {
  const int m = (int)P.m;
  const float ksc = P.st->key_scale;
  const float val = cell_value(K);
  // member test and exact key of this lane's element e = t L + ls
  auto member = [&](int t, unsigned long long& key) {
    const int e = t * L + ls;
    if (!have || e >= m) return false;
    const float xi = __ldg(P.X + i * P.ldx + e), xj = __ldg(P.X + j * P.ldx + e);
    if (cell_key(-ksc, xi * ksc, xj) != K) return false;
    key = exact_key(xi, xj);
    return true;
  };
  const unsigned seg_bits = (L == 32) ? FULL_MASK : (((1u << L) - 1) << ((threadIdx.x & 31) & ~(L - 1)));
#pragma unroll 1
  for (int t1 = 0; t1 < E; ++t1) {
    unsigned long long k1 = 0;
    const bool m1 = member(t1, k1);
    unsigned mb = __ballot_sync(FULL_MASK, m1) & seg_bits;
    while (__any_sync(FULL_MASK, mb != 0)) {
      const bool h = mb != 0;
      const int ld = h ? (__ffs(mb) - 1) % L : 0;
      const unsigned lo32 = __shfl_sync(FULL_MASK, (unsigned)k1, ld, L);
      const unsigned hi32 = __shfl_sync(FULL_MASK, (unsigned)(k1 >> 32), ld, L);
      const unsigned long long kb = ((unsigned long long)hi32 << 32) | lo32;
      if (h) mb &= mb - 1;
      int lt = 0, eq = 0;
#pragma unroll 1
      for (int t2 = 0; t2 < E; ++t2) {
        unsigned long long k2 = 0;
        if (member(t2, k2)) {
          lt += (k2 < kb) ? 1 : 0;
          eq += (k2 == kb) ? 1 : 0;
        }
      }
#pragma unroll
      for (int o = L / 2; o >= 1; o >>= 1) {
        lt += __shfl_xor_sync(FULL_MASK, lt, o);
        eq += __shfl_xor_sync(FULL_MASK, eq, o);
      }
      if (h && ls == 0 && GINI_IDX_OK(P.err, 2 * (f + lt) + eq - 1, 2 * P.m - 1)) {
        const int a = tab_addr<E>(2 * (f + lt) + eq - 1);
        for (int q = 0; q < P.n_nu; ++q) corr[q] += val * s_tab[q * tab_stride + a];
      }
    }
  }
  if (have && ls == 0 && GINI_IDX_OK(P.err, 2 * f + c - 1, 2 * P.m - 1)) {
    const int a = tab_addr<E>(2 * f + c - 1);
    for (int q = 0; q < P.n_nu; ++q) corr[q] -= (float)c * val * s_tab[q * tab_stride + a];
  }
}

// k_dist_keyed: weights that are not affine in the rank (any nu but a single 2
// or 3).  Cell keys (cell_key) sorted by the FP32 network in the alternating
// layout, turned back into ascending order in every lane, then tie runs as
// in k_dist_exact: each run is added once, at its last entry, as
// count * value * T_q[first + last].  TL, TR as for k_dist; NQ >= n_nu nu
// slots are carried in registers (1, 4 or 8: fewer slots, less code).
template <int E, int L, int TL, int TR, int NQ>
__device__ __forceinline__ void dist_keyed_body(const DistParams& P) {
  constexpr int G = 32 / L;
  extern __shared__ float s_tab[];  // n_nu x tab_stride
  __shared__ double s_sd2[DIST_WARPS][G][NU_MAX];
  __shared__ float s_corr[DIST_WARPS][G][NU_MAX];
  __shared__ float s_xi[DIST_WARPS][E * L];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int seg = lane / L, ls = lane % L;
  const int64_t row0 = (int64_t)blockIdx.y * DIST_WARPS;
  const int64_t col0 = P.col_begin + (int64_t)blockIdx.x * P.cb;
  // Nothing above the diagonal in this block, or the 64-bit kernel's turn
  // (uniform exits, before any barrier).
  if (col0 + P.cb - 1 <= row0 || row0 >= P.n - 1) return;
  if (P.st->fallback) return;

  const int m = (int)P.m;
  const int tab_n = 2 * m - 1;
  const int tab_stride = tab_addr<E>(tab_n - 1) + 1;
  for (int q = 0; q < P.n_nu; ++q)
    for (int idx = threadIdx.x; idx < tab_n; idx += blockDim.x)
      s_tab[q * tab_stride + tab_addr<E>(idx)] = P.wtab[(int64_t)q * tab_n + idx];
  for (int idx = threadIdx.x; idx < DIST_WARPS * G * NU_MAX; idx += blockDim.x) {
    (&s_sd2[0][0][0])[idx] = 0.0;
    (&s_corr[0][0][0])[idx] = 0.f;
  }

  const float ksc = P.st->key_scale;
  const bool odd = L >= 2 && (ls & 1);
  // x_i scaled by 2^s and signed for the lanes that read it (e and ls have the
  // same parity when L is even): an odd lane's keys are those of -z, i.e. the
  // negated keys of z, which is the alternating layout's input
  const int64_t i = row0 + warp;
  const bool row_ok = i < P.n - 1;
#pragma unroll
  for (int t = 0; t < E; ++t) {
    const int e = t * L + ls;
    float x = (row_ok && e < m) ? __ldg(P.X + i * P.ldx + e) : 0.f;
    if (L >= 2 && (e & 1)) x = -x;
    if (seg == 0) s_xi[warp][e] = x * ksc;
  }
  // padding of odd lanes, which sorts to the bottom of the sequence
  int n_lo = 0;
  if (L >= 2)
    for (int l = 1; l < L; l += 2) n_lo += E - min(E, m > l ? (m - l + L - 1) / L : 0);
  __syncthreads();

  const float cj = odd ? ksc : -ksc;          // multiplier of x_j: -s0 2^s
  const int pos0 = E * ls;
  for (int64_t jb = col0; jb < col0 + P.cb; jb += G) {
    const int64_t j = jb + seg;
    const bool active = row_ok && j > i && j < P.col_end && GINI_IDX_OK(P.err, j, P.n);
    if (!__any_sync(FULL_MASK, active)) continue;
    float u[E];
#pragma unroll
    for (int t = 0; t < E; ++t) {
      const int e = t * L + ls;
      if (t < TR) {
        const bool real = t < TL || e < m;
        const float xj = (active && real) ? __ldg(P.X + j * P.ldx + e) : 0.f;
        u[t] = real ? cell_key(cj, s_xi[warp][e], xj) : FLT_MAX;
      } else {
        u[t] = FLT_MAX;
      }
    }
    // One nu: the merge levels as a loop (the unrolled network plus the
    // table-driven epilogue overflowed the instruction cache; 10.0 -> 9.35 ms
    // at n = 2000, p = 784).  Several nu: unrolled (looped measured 2 % slower).
    if constexpr (NQ == 1) seg_sort_alternating_looped<E, L, TR>(u, ls);
    else seg_sort_alternating<E, L, TR>(u, ls);
    // every lane in ascending position order: an odd lane holds -v in reverse
    // order, so it reverses its registers and keeps the sign (equality, and so
    // the runs, do not see it; it is taken out of the lane's sums below)
    float v[E];
#pragma unroll
    for (int t = 0; t < E; ++t) v[t] = odd ? u[E - 1 - t] : u[t];
    bool cont_right;
    // cross-lane equality compares values: adjacent lanes carry opposite signs
    int s = seg_first_run_start<E, L, true>(v, ls, [](float a, float b) { return a == b; },
                                            cont_right);
    float acc[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[q] = 0.f;
    unsigned amb = 0;  // bit t: register t ends a run of several entries with an odd key
#pragma unroll
    for (int t = 0; t < E; ++t) {
      if (t > 0 && v[t] != v[t - 1]) s = pos0 + t;
      const bool last = (t < E - 1) ? (v[t] != v[t + 1]) : !cont_right;
      // padding is +-FLT_MAX; a key's magnitude is at most 2^127
      if (last && fabsf(v[t]) < FLT_MAX) {
        const int pos = pos0 + t;
        const int cnt = pos - s + 1;
        const float fc = __int_as_float(0x4B000000 + cnt) - 8388608.f;  // (float)cnt
        const float w = cell_value(v[t]) * fc;
        const int a = tab_addr<E>(s + pos - 2 * n_lo);
        const bool tab_ok = GINI_IDX_OK(P.err, s + pos - 2 * n_lo, 2 * P.m - 1);
#pragma unroll
        for (int q = 0; q < NQ; ++q)
          if ((NQ == 1 || q < P.n_nu) && tab_ok) acc[q] = fmaf(w, s_tab[q * tab_stride + a], acc[q]);
        if (cnt > 1 && (__float_as_uint(v[t]) & 1u)) amb |= 1u << t;
      }
    }
    if (__any_sync(FULL_MASK, amb != 0)) {
      // Runs whose cell keys tie although the differences may not: fix each
      // one (segment by segment, lowest register first).
      const unsigned seg_bits = (L == 32) ? FULL_MASK : (((1u << L) - 1) << (seg * L));
      unsigned pend = amb;
      while (__any_sync(FULL_MASK, pend != 0)) {
        const unsigned sb = __ballot_sync(FULL_MASK, pend != 0) & seg_bits;
        const bool have = sb != 0;
        const int leader = have ? (__ffs(sb) - 1) % L : 0;
        const int tl = __shfl_sync(FULL_MASK, pend ? __ffs(pend) - 1 : 0, leader, L);
        float kl = 0.f;
#pragma unroll
        for (int t = 0; t < E; ++t) kl = (t == tl) ? v[t] : kl;
        const float K = __shfl_sync(FULL_MASK, odd ? -kl : kl, leader, L);  // the value
        if (have && ls == leader) pend &= pend - 1;
        const float Ks = odd ? -K : K;  // as this lane holds it
        int lt = 0, ceq = 0;
#pragma unroll
        for (int t = 0; t < E; ++t) {
          lt += (odd ? (v[t] > Ks) : (v[t] < Ks)) ? 1 : 0;
          ceq += (v[t] == Ks) ? 1 : 0;
        }
#pragma unroll
        for (int o = L / 2; o >= 1; o >>= 1) {
          lt += __shfl_xor_sync(FULL_MASK, lt, o);
          ceq += __shfl_xor_sync(FULL_MASK, ceq, o);
        }
        keyed_fix_run<E, L>(P, s_tab, tab_stride, i, active ? j : i + 1, ls, have && active, K,
                            lt - n_lo, ceq, s_corr[warp][seg]);
      }
      // lane 0 is even: its sums carry no sign
      if (ls == 0) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          acc[q] += s_corr[warp][seg][q];
          s_corr[warp][seg][q] = 0.f;
        }
      }
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      if (NQ == 1 || q < P.n_nu) {
        if (odd) acc[q] = -acc[q];
#pragma unroll
        for (int o = L / 2; o >= 1; o >>= 1) acc[q] += __shfl_xor_sync(FULL_MASK, acc[q], o);
      }
    }
    if (active && ls == 0) {
      const float inv = 1.f / ksc;  // a power of two: exact
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        if (NQ == 1 || q < P.n_nu) {
          const float d = acc[q] * inv;
          store_delta(P, q, i, j, d);
          s_sd2[warp][seg][q] += (double)d * (double)d;
        }
      }
    }
  }
  __syncthreads();
  if (threadIdx.x < P.n_nu && P.sum_delta2) {
    double sum = 0.0;
    for (int w = 0; w < DIST_WARPS; ++w)
      for (int g = 0; g < G; ++g) sum += s_sd2[w][g][threadIdx.x];
    add_exact128(P.st->sd2[threadIdx.x], sum, P.st->sd2_q);
  }
}

// Entry points.  The affine kernel fits three CTAs per SM as compiled; the
// 64-bit one is bounded to two (128 registers, a few spilled) instead of the
// one CTA its network would otherwise take.
template <int E, int L, int TL, int TR>
__global__ void __launch_bounds__(DIST_WARPS * 32) k_dist(const DistParams P) {
  dist_body<E, L, true, TL, TR>(P);
}

template <int E, int L, int TL, int TR, int NQ>
__global__ void __launch_bounds__(DIST_WARPS * 32, 3) k_dist_keyed(const DistParams P) {
  dist_keyed_body<E, L, TL, TR, NQ>(P);
}

template <int E, int L>
__global__ void __launch_bounds__(DIST_WARPS * 32, 2) k_dist_exact(const DistParams P) {
  dist_body<E, L, false, E, E>(P);
}

// Pre-pass over X: finiteness and the extrema of DistState (one warp-level
// reduction, then one atomicMax per warp and word).
__global__ void k_dist_stats(const float* X, int64_t n, int64_t m, int64_t ld, DistState* st,
                             unsigned* err) {
  unsigned mx = 0, imn = 0, inz = 0;
  bool bad = false;
  for (int64_t r = blockIdx.x; r < n; r += gridDim.x)
    for (int64_t c = threadIdx.x; c < m; c += blockDim.x) {
      const float x = X[r * ld + c];
      bad |= !isfinite(x);
      const unsigned o = ord_bits(x);
      mx = max(mx, o);
      imn = max(imn, ~o);
      if (x != 0.f) inz = max(inz, ~__float_as_uint(fabsf(x)));
    }
  mx = __reduce_max_sync(FULL_MASK, mx);
  imn = __reduce_max_sync(FULL_MASK, imn);
  inz = __reduce_max_sync(FULL_MASK, inz);
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&st->max_ord, mx);
    atomicMax(&st->inv_min_ord, imn);
    atomicMax(&st->inv_min_nz, inz);
  }
  if (__any_sync(FULL_MASK, bad) && (threadIdx.x & 31) == 0) raise_error(err, ERR_NONFINITE);
}

// One thread: the key scale, the fallback decision and the unit of Sum delta^2.
//   key scale 2^s: the smallest s <= 0 with R 2^s <= 1, R = max X - min X >=
//     |x_ia - x_ja|, so every cell key stays finite;
//   fallback: R not finite, or scaling would push some nonzero |x| below the
//     normal range (then x 2^s, and the keys, could be inexact);
//   unit 2^q: |delta| <= (d/2) sum_a |z_a| <= d^2 R / 2 (|W| <= 1), so
//     Sum delta^2 <= P (d^2 R / 2)^2 < 2^(q + 125).
__global__ void k_dist_setup(DistState* st, int64_t n, int64_t m) {
  const float mx = unord_bits(st->max_ord), mn = unord_bits(~st->inv_min_ord);
  const float R = __fsub_ru(mx, mn);
  int s = 0, fb = 0;
  if (!(R <= FLT_MAX)) {
    fb = 1;
  } else if (R > 1.f) {
    int e;
    frexpf(R, &e);  // R < 2^e
    s = -e;
    if (st->inv_min_nz != 0) {
      int e2;
      frexpf(__uint_as_float(~st->inv_min_nz), &e2);  // smallest nonzero |x| >= 2^(e2 - 1)
      if (e2 - 1 + s < -126) fb = 1;
    }
  }
  st->key_scale = ldexpf(1.f, s);
  st->fallback = fb;
  const double pairs = 0.5 * (double)n * (double)(n - 1);
  const double dmax = 0.5 * (double)m * (double)m * (double)R;
  const double bound = pairs * dmax * dmax;
  int q = 0;
  if (bound > 0.0 && bound <= DBL_MAX) {
    int eb;
    frexp(bound, &eb);  // bound < 2^eb
    q = eb - 125;
  }
  st->sd2_q = q;
}

// Sum delta^2 of each nu from its exact accumulator.
__global__ void k_dist_finalize(const DistState* st, int n_nu, double* out) {
  const int q = threadIdx.x;
  if (q < n_nu) {
    const double hi = (double)st->sd2[q][1], lo = (double)st->sd2[q][0];
    out[q] = ldexp(hi, 64 + st->sd2_q) + ldexp(lo, st->sd2_q);
  }
}

__global__ void k_zero_diag(float* D, int64_t n, int64_t ldd, int64_t nu_stride, int n_nu) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n)
    for (int q = 0; q < n_nu; ++q) D[(int64_t)q * nu_stride + i * ldd + i] = 0.f;
}

// FP8 e4m3 output, built one strip of columns [c0, c1) at a time: the strip's
// FP32 values (rows 0..n-1, entries i < j only) are in scratch; these kernels
// take each column's max |delta| over i < j, turn it into the column's scale
// max / 448 (1 for an all-zero column), and quantize the strip's tiles.
// Block (x: 256 columns, y: 256 rows of the strip); bits of |delta| >= 0
// order like the floats, so integer atomicMax gives the float maximum.
__global__ void k_strip_colmax(const float* __restrict__ strip, int64_t n, int64_t w,
                               int64_t c0, int64_t c1, unsigned* __restrict__ colmax) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c0 + c >= c1) return;
  const int64_t j = c0 + c;
  const int64_t i0 = (int64_t)blockIdx.y * 256;
  unsigned m = 0;
  for (int64_t i = i0; i < i0 + 256 && i < j; ++i)
    m = max(m, __float_as_uint(fabsf(strip[i * w + c])));
  if (m) atomicMax(colmax + j, m);
}

__global__ void k_strip_scale(unsigned* colmax_bits, int64_t c0, int64_t c1) {
  const int64_t j = c0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= c1) return;
  const float mx = __uint_as_float(colmax_bits[j]);
  reinterpret_cast<float*>(colmax_bits)[j] = mx > 0.f ? mx / 448.f : 1.f;
}

// Block (x: tile of the strip, in row-major (I, J) order over J in the strip's
// tile columns, y: 256-element slice of the tile); one thread per element.
__global__ void k_strip_quant(const float* __restrict__ strip, int64_t n, int64_t w, int64_t c0,
                              int64_t T, int64_t J0, int64_t nJ, const float* __restrict__ scale,
                              __nv_fp8_storage_t* __restrict__ out, unsigned* err) {
  // tiles (I, J), J0 <= J < J0 + nJ, I <= J: enumerate J-major (column of
  // tiles), I inside; t -> (I, J) by the running count (J + 1 tiles per column)
  int64_t t = blockIdx.x, J = J0;
  while (t > J) {
    t -= J + 1;
    ++J;
  }
  const int64_t I = t;
  const int rc = (int)blockIdx.y * blockDim.x + threadIdx.x;
  const int64_t i = I * TILE + rc / TILE, j = J * TILE + rc % TILE;
  // (debug builds) the tile is in the triangle and the strip holds column j
  if (!(GINI_IDX_OK(err, tile_offset(I, J, T), T * (T + 1) / 2) &&
        GINI_IDX_OK(err, I, J + 1) && (j >= n || GINI_IDX_OK(err, j - c0, w))))
    return;
  const float v = (i < n && j < n && i < j) ? strip[i * w + (j - c0)] : 0.f;
  const float sc = (j < n) ? scale[j] : 1.f;
  out[tile_offset(I, J, T) * (TILE * TILE) + rc] =
      __nv_cvt_float_to_fp8(v / sc, __NV_SATFINITE, __NV_E4M3);
}

// Vectors longer than one warp's registers (1024 < p <= 8192): one warp per
// pair sorts the exact (hi, lo) keys of x_i - x_j chunk by chunk into shared
// memory; every element's midrank then comes from binary searches in all
// chunks (lt below, eq equal, itself included: first + last = 2 lt + eq - 1),
// and it adds hi * T_q[first + last] for every nu (tables read from the
// workspace through the cache).  Exact for every nu; the work per pair is
// O(p log^2 1024 + p C log 1024) for C chunks.  CTA = LONG_WARPS pairs of one
// row i: j = max(i + 1, col_begin) + LONG_WARPS x + warp.
constexpr int LONG_WARPS = 2;

__global__ void __launch_bounds__(LONG_WARPS * 32) k_dist_long(const DistParams P, int nchunk) {
  extern __shared__ unsigned long long s_long[];  // [LONG_WARPS][nchunk][LONG_CHUNK_SLOTS]
  __shared__ double s_sd2[LONG_WARPS][NU_MAX];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m = (int)P.m, tab_n = 2 * m - 1;
  const int64_t i = blockIdx.y;
  const int64_t j = std::max(i + 1, P.col_begin) + (int64_t)blockIdx.x * LONG_WARPS + warp;
  const bool active = i < P.n - 1 && j < P.col_end && GINI_IDX_OK(P.err, j, P.n);
  unsigned long long* K = s_long + (size_t)warp * nchunk * LONG_CHUNK_SLOTS;
  const float* xi = P.X + i * P.ldx;
  const float* xj = P.X + (active ? j : i) * P.ldx;
  if (active) {  // warp-uniform
    for (int c = 0; c < nchunk; ++c) {
      unsigned long long kv[32];
#pragma unroll
      for (int t = 0; t < 32; ++t) {
        const int e = c * LONG_CHUNK + t * 32 + lane;
        kv[t] = e < m ? exact_key(__ldg(xi + e), __ldg(xj + e)) : ~0ull;
      }
      long_sort_chunk(kv, lane, K + (size_t)c * LONG_CHUNK_SLOTS);
    }
    __syncwarp();
    float acc[NU_MAX];
#pragma unroll
    for (int q = 0; q < NU_MAX; ++q) acc[q] = 0.f;
    for (int e = lane; e < m; e += 32) {
      const float a = __ldg(xi + e), b = __ldg(xj + e);
      const unsigned long long k = exact_key(a, b);
      int lt = 0, eq = 0;
      for (int c = 0; c < nchunk; ++c)
        long_count(K + (size_t)c * LONG_CHUNK_SLOTS, min(LONG_CHUNK, m - c * LONG_CHUNK), k, lt,
                   eq);
      const float hi = two_sum_canonical(a, -b).x;
      const int idx = 2 * lt + eq - 1;
      const bool tab_ok = GINI_IDX_OK(P.err, idx, tab_n);
#pragma unroll
      for (int q = 0; q < NU_MAX; ++q)
        if (q < P.n_nu && tab_ok)
          acc[q] = fmaf(hi, __ldg(P.wtab + (int64_t)q * tab_n + idx), acc[q]);
    }
#pragma unroll
    for (int q = 0; q < NU_MAX; ++q) {
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) acc[q] += __shfl_xor_sync(FULL_MASK, acc[q], o);
    }
    if (lane == 0) {
      for (int q = 0; q < P.n_nu; ++q) {
        store_delta(P, q, i, j, acc[q]);
        s_sd2[warp][q] = (double)acc[q] * (double)acc[q];
      }
    }
  } else if (lane == 0) {
    for (int q = 0; q < NU_MAX; ++q) s_sd2[warp][q] = 0.0;
  }
  __syncthreads();
  if (threadIdx.x < P.n_nu && P.sum_delta2) {
    double sum = 0.0;
    for (int w = 0; w < LONG_WARPS; ++w) sum += s_sd2[w][threadIdx.x];
    add_exact128(P.st->sd2[threadIdx.x], sum, P.st->sd2_q);
  }
}

static cudaError_t launch_dist_long(const DistParams& P, cudaStream_t s) {
  const int nchunk = (int)((P.m + LONG_CHUNK - 1) / LONG_CHUNK);
  const size_t smem = sizeof(unsigned long long) * LONG_WARPS * nchunk * LONG_CHUNK_SLOTS;
  cudaError_t e = cudaFuncSetAttribute(k_dist_long, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t rows = std::min(P.n, P.col_end) - 1;
  const int64_t span = P.col_end - P.col_begin;
  dim3 grid((unsigned)((span + LONG_WARPS - 1) / LONG_WARPS), (unsigned)rows);
  gini_count_launch(1);
  k_dist_long<<<grid, LONG_WARPS * 32, smem, s>>>(P, nchunk);
  return cudaGetLastError();
}

// KIND_KEYED + NQ: the keyed kernel with NQ nu slots.
enum DistKind { KIND_AFFINE = 0, KIND_EXACT = 1, KIND_KEYED = 2 };

template <int E, int L, int KIND, int TL, int TR>
static auto dist_kernel() {
  if constexpr (KIND == KIND_AFFINE) return k_dist<E, L, TL, TR>;
  else if constexpr (KIND == KIND_EXACT) return k_dist_exact<E, L>;
  else return k_dist_keyed<E, L, TL, TR, KIND - KIND_KEYED>;
}

template <int E, int L, int KIND, int TL = E, int TR = E>
static cudaError_t launch_dist(const DistParams& P, cudaStream_t s) {
  void (*kern)(const DistParams) = dist_kernel<E, L, KIND, TL, TR>();
  const int m = (int)P.m;
  const int tab_n = 2 * m - 1;
  const int tab_stride = tab_n - 1 + (tab_n - 1) / (2 * E) + 1;
  const size_t smem = KIND == KIND_AFFINE ? 0 : (size_t)P.n_nu * tab_stride * sizeof(float);
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
  const int64_t ncols = P.col_end - P.col_begin;
  dim3 grid((unsigned)((ncols + Q.cb - 1) / Q.cb),
            (unsigned)((std::min(P.n, P.col_end) + DIST_WARPS - 1) / DIST_WARPS));
  gini_count_launch(1);
  kern<<<grid, DIST_WARPS * 32, smem, s>>>(Q);
  return cudaGetLastError();
}

// Segment shapes by vector length m: one instantiation per power-of-two
// segment size up to 16 lanes, with the bounds TL, TR on the real registers
// (m in (E*L/2, E*L] fills every register below E/2); 32-lane segments take
// 20, 24, 25, 28 or 32 registers per lane by m, so that no register holds
// padding in every lane.  The 64-bit network takes the plain power-of-two
// shapes.
template <int KIND>
static cudaError_t dispatch_dist(const DistParams& P, cudaStream_t s) {
  const int64_t m = P.m;
  if constexpr (KIND == KIND_EXACT) {
    if (m <= 4) return launch_dist<4, 1, KIND>(P, s);
    if (m <= 8) return launch_dist<8, 1, KIND>(P, s);
    if (m <= 16) return launch_dist<16, 1, KIND>(P, s);
    if (m <= 32) return launch_dist<32, 1, KIND>(P, s);
    if (m <= 64) return launch_dist<32, 2, KIND>(P, s);
    if (m <= 128) return launch_dist<32, 4, KIND>(P, s);
    if (m <= 256) return launch_dist<32, 8, KIND>(P, s);
    if (m <= 512) return launch_dist<32, 16, KIND>(P, s);
    return launch_dist<32, 32, KIND>(P, s);
  } else {
    if (m <= 4) return launch_dist<4, 1, KIND, 1, 4>(P, s);
    if (m <= 8) return launch_dist<8, 1, KIND, 4, 8>(P, s);
    if (m <= 16) return launch_dist<16, 1, KIND, 8, 16>(P, s);
    if (m <= 32) return launch_dist<32, 1, KIND, 16, 32>(P, s);
    if (m <= 64) return launch_dist<32, 2, KIND, 16, 32>(P, s);
    if (m <= 128) return launch_dist<32, 4, KIND, 16, 32>(P, s);
    if (m <= 256) return launch_dist<32, 8, KIND, 16, 32>(P, s);
    if (m <= 512) return launch_dist<32, 16, KIND, 16, 32>(P, s);
    // 32 lanes: each holds as many registers as the data need, rounded to a
    // length with a short in-lane merge (20, 24, 25, 28, 32), so that no
    // register is padding in every lane (784 = 28 x 28 images: 25)
    if (m <= 640) return launch_dist<20, 32, KIND, 16, 20>(P, s);
    if (m <= 768) return launch_dist<24, 32, KIND, 20, 24>(P, s);
    if (m <= 800) return launch_dist<25, 32, KIND, 24, 25>(P, s);
    if (m <= 896) return launch_dist<28, 32, KIND, 25, 28>(P, s);
    return launch_dist<32, 32, KIND, 28, 32>(P, s);
  }
}

}  // namespace gini

using namespace gini;

extern "C" void gini_set_cuda_error(cudaError_t e);

extern "C" int gini_dist(const float* X_dev, int64_t n, int64_t p, int64_t ldx,
                         const double* nu_host, int n_nu, int layout, int dtype, void* delta_dev,
                         int64_t ldd, int64_t nu_stride, float* col_scale_dev,
                         double* sum_delta2_dev, void* ws, size_t ws_bytes, void* stream) {
  NvtxRange nvtx_range("gini_dist");
  if (!X_dev || !delta_dev || !nu_host || !ws) return GINI_EINVAL;
  if (ws_misaligned(ws)) return GINI_EINVAL;
  if (n < 2 || p < 1 || p > (int64_t)LONG_CHUNK * LONG_MAX_CHUNKS || ldx < p || n_nu < 1 ||
      n_nu > NU_MAX)
    return GINI_EINVAL;
  if (n > (int64_t)65535 * DIST_WARPS) return GINI_EINVAL;  // grid.y = ceil(n / 8)
  if (p > LONG_CHUNK && n > 65536) return GINI_EINVAL;      // long vectors: grid.y = n - 1
  for (int q = 0; q < n_nu; ++q)
    if (!(nu_host[q] > 1.0) || !isfinite(nu_host[q])) return GINI_EINVAL;
  if (layout == GINI_LAYOUT_FULL) {
    if (dtype != GINI_F32 || ldd < n) return GINI_EINVAL;
    if (n_nu > 1 && nu_stride < ldd * n) return GINI_EINVAL;
  } else if (layout == GINI_LAYOUT_TILED) {
    if (dtype < GINI_F32 || dtype > GINI_FP8E4M3) return GINI_EINVAL;
    if (dtype == GINI_FP8E4M3 && !col_scale_dev) return GINI_EINVAL;
    const int64_t plane = gini_tiled_elems(n);
    if (n_nu > 1 && nu_stride < plane * (dtype == GINI_BF16X2 ? 2 : 1)) return GINI_EINVAL;
  } else {
    return GINI_EINVAL;
  }
  const bool fp8 = layout == GINI_LAYOUT_TILED && dtype == GINI_FP8E4M3;
  const size_t ws_base = gini_workspace_size(GINI_OP_DIST, n, p, 0, 0);
  // FP8 needs scratch for at least one tile column of every matrix
  if (ws_bytes < ws_base + (fp8 ? sizeof(float) * (size_t)n * TILE * n_nu : 0))
    return GINI_ENOMEM;

  cudaStream_t s = (cudaStream_t)stream;
  // workspace: error word | DistState | weight tables
  unsigned* err = reinterpret_cast<unsigned*>(ws);
  DistState* st = reinterpret_cast<DistState*>(reinterpret_cast<char*>(ws) + WS_HEADER);
  float* wtab = reinterpret_cast<float*>(reinterpret_cast<char*>(ws) + WS_HEADER +
                                         DIST_STATE_BYTES);
  // W_{d,nu} is affine in the rank for nu = 2 and nu = 3:
  // (d/2) W_{d,3}(R) = ((d-1)/d) (R - (d+1)/2) = ((d-1)/d) (d/2) W_{d,2}(R)
  const bool affine = (n_nu == 1 && (nu_host[0] == 2.0 || nu_host[0] == 3.0));
  const int tab_n = (int)(2 * p - 1);
  if (!affine || p > LONG_CHUNK) {  // long vectors always read the table
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
  cudaError_t e = cudaMemsetAsync(st, 0, sizeof(DistState), s);
  if (e == cudaSuccess) {
    gini_count_launch(2);
    const int64_t rows = n < 2048 ? n : 2048;
    k_dist_stats<<<(unsigned)rows, 256, 0, s>>>(X_dev, n, p, ldx, st, err);
    k_dist_setup<<<1, 1, 0, s>>>(st, n, p);
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
    P.sum_delta2 = sum_delta2_dev; P.err = err; P.st = st;
    P.col_begin = 0; P.col_end = n;
    P.affine_scale = (affine && nu_host[0] == 3.0) ? (float)((double)(p - 1) / (double)p) : 1.f;
    auto build = [&](const DistParams& Q) -> cudaError_t {
      if (p > LONG_CHUNK) return launch_dist_long(Q, s);
      if (affine) return dispatch_dist<KIND_AFFINE>(Q, s);
      // both launch; the pre-pass's flag lets exactly one of them do the work
      cudaError_t r = n_nu == 1   ? dispatch_dist<KIND_KEYED + 1>(Q, s)
                      : n_nu <= 4 ? dispatch_dist<KIND_KEYED + 4>(Q, s)
                                  : dispatch_dist<KIND_KEYED + 8>(Q, s);
      return r == cudaSuccess ? dispatch_dist<KIND_EXACT>(Q, s) : r;
    };
    if (!fp8) {
      e = build(P);
    } else {
      // FP8: strips of w columns (a multiple of the tile) built into FP32
      // scratch, then each strip's column scales and its tiles of the output
      float* strip = reinterpret_cast<float*>(reinterpret_cast<char*>(ws) + ws_base);
      const size_t budget = ws_bytes - ws_base;
      int64_t w = (int64_t)(budget / (sizeof(float) * (size_t)n * n_nu)) / TILE * TILE;
      w = std::min(w, tiles_1d(n) * TILE);
      if (w < TILE) return GINI_ENOMEM;
      e = cudaMemsetAsync(col_scale_dev, 0, sizeof(float) * (size_t)n * n_nu, s);
      const int64_t T = tiles_1d(n), plane = gini_tiled_elems(n);
      for (int64_t c0 = 0; c0 < n && e == cudaSuccess; c0 += w) {
        const int64_t c1 = std::min(n, c0 + w);
        DistParams Q = P;
        Q.layout = LAYOUT_STRIP; Q.out = strip; Q.ldd = w; Q.nu_stride = n * w;
        Q.col_begin = c0; Q.col_end = c1;
        e = build(Q);
        const int64_t J0 = c0 / TILE, nJ = tiles_1d(c1) - J0;
        int64_t ntile = 0;
        for (int64_t J = J0; J < J0 + nJ; ++J) ntile += J + 1;
        for (int q = 0; q < n_nu && e == cudaSuccess; ++q) {
          const float* sq = strip + (int64_t)q * n * w;
          unsigned* cm = reinterpret_cast<unsigned*>(col_scale_dev + (int64_t)q * n);
          gini_count_launch(3);
          k_strip_colmax<<<dim3((unsigned)((c1 - c0 + 255) / 256), (unsigned)((c1 + 255) / 256)),
                           256, 0, s>>>(sq, n, w, c0, c1, cm);
          k_strip_scale<<<(unsigned)((c1 - c0 + 255) / 256), 256, 0, s>>>(cm, c0, c1);
          k_strip_quant<<<dim3((unsigned)ntile, TILE * TILE / 256), 256, 0, s>>>(
              sq, n, w, c0, T, J0, nJ, col_scale_dev + (int64_t)q * n,
              reinterpret_cast<__nv_fp8_storage_t*>(delta_dev) + (int64_t)q * nu_stride, err);
          e = cudaGetLastError();
        }
        (void)plane;
      }
    }
  }
  if (e == cudaSuccess && sum_delta2_dev) {
    gini_count_launch(1);
    k_dist_finalize<<<1, 32, 0, s>>>(st, n_nu, sum_delta2_dev);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) { gini_set_cuda_error(e); return GINI_ECUDA; }
  return GINI_OK;
}
