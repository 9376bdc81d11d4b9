// Register-resident bitonic sort of one segment spread over L lanes x E
// registers, plus the tie-run (midrank) bookkeeping on the sorted segment.
//
// Layout: a segment is L consecutive lanes of a warp (L in 1..32, a power of
// two, aligned); lane ls of the segment holds registers v[0..E).  The network
// sorts the E*L values ascending so that afterwards position
// pos = E*ls + t holds v[t] ("blocked" layout).  The initial placement of the
// values is arbitrary: the caller loads them in whatever order is coalesced.
//
// Network (float keys): each lane first sorts its E registers with Batcher's
// odd-even merge sort (fewer compare-exchanges than the bitonic levels it
// replaces: 191 instead of 240 for E = 32); the levels across lanes follow.
// Network (generic keys): the bitonic sorter written without direction flags.  For block size
// kk = 2, 4, ..., E*L, element i is first compared with its mirror i ^ (kk-1)
// inside the block, then with i ^ jj for jj = kk/4, ..., 1; the lower index
// always keeps the minimum.  Partners closer than E positions sit in the same
// lane (register exchange); farther ones in lane ls ^ (distance / E), reached
// with a warp shuffle.
#pragma once

#include "common.cuh"

namespace gini {

__device__ __forceinline__ float kmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ float kmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ unsigned long long kmin(unsigned long long a, unsigned long long b) {
  return a < b ? a : b;
}
__device__ __forceinline__ unsigned long long kmax(unsigned long long a, unsigned long long b) {
  return a < b ? b : a;
}

template <typename T>
__device__ __forceinline__ void cas(T& a, T& b) {
  T lo = kmin(a, b), hi = kmax(a, b);
  a = lo;
  b = hi;
}

// Cross-lane exchange: the lower lane keeps min(v, o), the upper max(v, o).
// (Rewriting it as s * min(s*v, s*o), s = +-1, moves two of the three
// operations off the ALU pipe but raised register use and measured slower.)
__device__ __forceinline__ float keep_lo_hi(float v, float o, bool lower) {
  return lower ? fminf(v, o) : fmaxf(v, o);
}
__device__ __forceinline__ unsigned long long keep_lo_hi(unsigned long long v,
                                                         unsigned long long o, bool lower) {
  return lower ? kmin(v, o) : kmax(v, o);
}

// Float keys: the cross-lane stages keep, in every lane whose role in the
// stage is "upper" (keeps the maximum), the negated values.  Partners then have
// opposite signs and both keep fminf(u, -o): the lower lane min(v, o), the upper
// lane min(-v, -o) = -max(v, o).  One min per element on the ALU pipe instead of
// a min, a max and a select; the sign changes between stages (a lane's role
// depends on the stage's lane bit) are multiplications by +-1 on the FMA pipe.
// Batcher's odd-even merge sort of N keys as a comparator list (compile time).
template <int N>
struct OemNet {
  int n = 0;
  unsigned char a[N * N / 2] = {}, b[N * N / 2] = {};
  constexpr OemNet() {
    for (int p = 1; p < N; p <<= 1)
      for (int k = p; k >= 1; k >>= 1)
        for (int j = k % p; j < N - k; j += 2 * k)
          for (int i = 0; i < k && i + j + k < N; ++i)
            if ((i + j) / (2 * p) == (i + j + k) / (2 * p)) {
              a[n] = (unsigned char)(i + j);
              b[n] = (unsigned char)(i + j + k);
              ++n;
            }
  }
};

template <int E, int JJ>
__device__ __forceinline__ void inlane_half_cleaners(float (&v)[E]) {
  if constexpr (JJ >= 1) {
#pragma unroll
    for (int t = 0; t < E; ++t)
      if ((t ^ JJ) > t) cas(v[t], v[t ^ JJ]);
    inlane_half_cleaners<E, JJ / 2>(v);
  }
}

// Cross-lane half-cleaners at lane distances D, D/2, ..., 1; sg is the sign
// the lane's values carry on entry and on exit.
template <int E, int D>
__device__ __forceinline__ void crosslane_half_cleaners(float (&v)[E], int ls, float& sg) {
  if constexpr (D >= 1) {
    const float sn = (ls & D) == 0 ? 1.f : -1.f;
    const float f = sn * sg;
    sg = sn;
#pragma unroll
    for (int t = 0; t < E; ++t) {
      v[t] *= f;
      const float o = __shfl_xor_sync(FULL_MASK, v[t], D);
      v[t] = fminf(v[t], -o);
    }
    crosslane_half_cleaners<E, D / 2>(v, ls, sg);
  }
}

template <int E, int L, int KK>
__device__ __forceinline__ void bitonic_level(float (&v)[E], int ls) {
  if constexpr (KK <= E) {
    if constexpr (KK == 2) {
      constexpr OemNet<E> net{};
#pragma unroll
      for (int c = 0; c < net.n; ++c) cas(v[net.a[c]], v[net.b[c]]);
    }
  } else {
    // mirror stage across lanes ls and ls ^ (KK/E - 1): register t meets the
    // partner's register E-1-t
    float sg = (ls & (KK / (2 * E))) == 0 ? 1.f : -1.f;
#pragma unroll
    for (int t = 0; t < E; ++t) v[t] *= sg;
#pragma unroll
    for (int t = 0; t < E / 2; ++t) {
      const float a = __shfl_xor_sync(FULL_MASK, v[E - 1 - t], KK / E - 1);
      const float b = __shfl_xor_sync(FULL_MASK, v[t], KK / E - 1);
      v[t] = fminf(v[t], -a);
      v[E - 1 - t] = fminf(v[E - 1 - t], -b);
    }
    crosslane_half_cleaners<E, KK / (4 * E)>(v, ls, sg);
#pragma unroll
    for (int t = 0; t < E; ++t) v[t] *= sg;
    inlane_half_cleaners<E, E / 2>(v);
  }
  if constexpr (2 * KK <= E * L) bitonic_level<E, L, 2 * KK>(v, ls);
}

// Float keys: the cross-lane stages keep, in every lane whose role in the
// stage is "upper" (keeps the maximum), the negated values.  Partners then have
// opposite signs and both keep fminf(u, -o): the lower lane min(v, o), the upper
// lane min(-v, -o) = -max(v, o).  One min per element on the ALU pipe instead of
// a min, a max and a select; the sign changes between stages (a lane's role
// depends on the stage's lane bit) are multiplications by +-1 on the FMA pipe.
template <int E, int L>
__device__ __forceinline__ void seg_bitonic_sort(float (&v)[E], int ls) {
  static_assert((E & (E - 1)) == 0 && (L & (L - 1)) == 0 && L <= 32 && E >= 2, "powers of two");
  bitonic_level<E, L, 2>(v, ls);
}

template <int E, int L, typename T>
__device__ __forceinline__ void seg_bitonic_sort(T (&v)[E], int ls) {
  static_assert((E & (E - 1)) == 0 && (L & (L - 1)) == 0 && L <= 32 && E >= 2, "powers of two");
#pragma unroll
  for (int kk = 2; kk <= E * L; kk <<= 1) {
    // mirror stage: i <-> i ^ (kk - 1)
    if (kk <= E) {
#pragma unroll
      for (int t = 0; t < E; ++t) {
        const int p = t ^ (kk - 1);
        if (p > t) cas(v[t], v[p]);
      }
    } else {
      const int mask = kk / E - 1;
      const bool lower = (ls & (kk / (2 * E))) == 0;
#pragma unroll
      for (int t = 0; t < E / 2; ++t) {
        // partner lane's mirrored registers: E-1-t pairs with t
        T a = __shfl_xor_sync(FULL_MASK, v[E - 1 - t], mask);
        T b = __shfl_xor_sync(FULL_MASK, v[t], mask);
        v[t] = keep_lo_hi(v[t], a, lower);
        v[E - 1 - t] = keep_lo_hi(v[E - 1 - t], b, lower);
      }
    }
    // half-cleaners: i <-> i ^ jj
#pragma unroll
    for (int jj = kk / 4; jj >= 1; jj >>= 1) {
      if (jj >= E) {
        const int mask = jj / E;
        const bool lower = (ls & mask) == 0;
#pragma unroll
        for (int t = 0; t < E; ++t) {
          T o = __shfl_xor_sync(FULL_MASK, v[t], mask);
          v[t] = keep_lo_hi(v[t], o, lower);
        }
      } else {
#pragma unroll
        for (int t = 0; t < E; ++t) {
          const int p = t ^ jj;
          if (p > t) cas(v[t], v[p]);
        }
      }
    }
  }
}

// Tie runs of a sorted segment.  For every register t, run_lo[t] receives the
// first (0-based) position of the run of equal keys containing position
// E*ls + t.  The last position of each run is left to the caller's backward
// sweep, seeded with the two values returned here:
//   e(E-1) = cont_right ? carry_e : E*ls + E - 1,
//   e(t)   = key(t) == key(t+1) ? e(t+1) : E*ls + t.
// Runs crossing lane boundaries are resolved with two segmented scans (a
// "nearest valid value" propagation from the left for starts and from the
// right for ends).  KeyEq(a, b) decides equality of two sorted entries.
template <int E, int L, typename T, typename KeyEq>
__device__ __forceinline__ void seg_runs(const T (&v)[E], int ls, KeyEq eq, int (&run_lo)[E],
                                         int& carry_e, bool& cont_right) {
  const int pos0 = E * ls;
  // Neighbouring lanes' edge keys.  With width L the shuffles stay inside the
  // segment; edge lanes get their own value back, hence the explicit guards.
  T prev = __shfl_up_sync(FULL_MASK, v[E - 1], 1, L);
  T next = __shfl_down_sync(FULL_MASK, v[0], 1, L);
  const bool cont_left = (ls > 0) && eq(prev, v[0]);
  cont_right = (ls < L - 1) && eq(v[E - 1], next);
  int cnt_first = 0, cnt_last = 0;
#pragma unroll
  for (int t = 0; t < E; ++t) {
    cnt_first += eq(v[t], v[0]) ? 1 : 0;
    cnt_last += eq(v[t], v[E - 1]) ? 1 : 0;
  }
  const bool all_eq = (cnt_first == E);
  // start of the run holding the lane's last entry (-1: began in an earlier lane)
  int sl = (all_eq && cont_left) ? -1 : pos0 + E - cnt_last;
  // end of the run holding the lane's first entry (-1: ends in a later lane)
  int ef = (all_eq && cont_right) ? -1 : pos0 + cnt_first - 1;
#pragma unroll
  for (int d = 1; d < L; d <<= 1) {
    int o = __shfl_up_sync(FULL_MASK, sl, d, L);
    if (ls >= d && sl < 0) sl = o;
    int o2 = __shfl_down_sync(FULL_MASK, ef, d, L);
    if (ls + d < L && ef < 0) ef = o2;
  }
  const int carry_s = __shfl_up_sync(FULL_MASK, sl, 1, L);
  carry_e = __shfl_down_sync(FULL_MASK, ef, 1, L);
  run_lo[0] = cont_left ? carry_s : pos0;
#pragma unroll
  for (int t = 1; t < E; ++t) run_lo[t] = eq(v[t], v[t - 1]) ? run_lo[t - 1] : pos0 + t;
}

}  // namespace gini
