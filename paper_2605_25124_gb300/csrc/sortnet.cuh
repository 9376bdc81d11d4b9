// Register-resident sorting networks for one segment spread over L lanes x E
// registers, plus the tie-run (midrank) bookkeeping on the sorted segment.
//
// Layout: a segment is L consecutive lanes of a warp (L in 1..32, a power of
// two, aligned); lane ls of the segment holds registers v[0..E).  Each lane
// first sorts its own E registers; merge levels across lanes follow, each a
// bitonic merge (a mirror stage, then half-cleaners at halving distances).
// Partners closer than E positions sit in the same lane (register exchange);
// farther ones in another lane of the segment, reached with a warp shuffle.
//
// Generic keys (seg_bitonic_sort): the bitonic sorter written without
// direction flags.  For block size kk = 2, 4, ..., E*L, element i is first
// compared with its mirror i ^ (kk-1) inside the block, then with i ^ jj for
// jj = kk/4, ..., 1; the lower index always keeps the minimum.  Afterwards
// position E*ls + t holds v[t] ("blocked" layout).
//
// Float keys (seg_sort_alternating): the same merges on a layout in which
// odd lanes hold negated values in reverse order, so that every exchange is
// one minimum; the in-lane sort is Batcher's odd-even merge sort (191
// compare-exchanges instead of 240 bitonic ones for E = 32).  E need not be a
// power of two: the lanes then hold exactly as many registers as the data
// need (25 for 784 keys over 32 lanes), the cross-lane stages are
// half-cleaners on blocks of 2 D E positions, exact for any even length, and
// the in-lane merge recurses down to odd-length tables (inlane_bitonic).
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

// Cross-lane exchange of generic keys: the lower lane keeps min(v, o), the
// upper max(v, o).
__device__ __forceinline__ unsigned long long keep_lo_hi(unsigned long long v,
                                                         unsigned long long o, bool lower) {
  return lower ? kmin(v, o) : kmax(v, o);
}

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

template <int E, int JJ, typename T>
__device__ __forceinline__ void inlane_half_cleaners(T (&v)[E]) {
  if constexpr (JJ >= 1) {
#pragma unroll
    for (int t = 0; t < E; ++t)
      if ((t ^ JJ) > t) cas(v[t], v[t ^ JJ]);
    inlane_half_cleaners<E, JJ / 2, T>(v);
  }
}

// In-lane merge of a lane's registers once they hold a cyclic-bitonic
// sequence (a rotation of an ascending-then-descending run).  A half-cleaner
// (t against t + N/2) splits a cyclic-bitonic sequence of any even length N
// into two cyclic-bitonic halves, every key of the first no greater than any
// key of the second; so even lengths recurse on their halves, and the odd
// lengths at the end of the recursion take a table (BitonicLeaf).  Powers of
// two give the usual half-cleaners (80 steps for 32 registers); 20 registers
// take 52, 24 take 60, 25 take 72, 28 take 76.
//
// The tables sort every cyclic-bitonic sequence of their length.  They were
// found by a seeded greedy search over 0-1 inputs (search_bitonic_net.py): by
// the 0-1 principle a comparator network sorts every cyclic-bitonic sequence of
// length N if and only if it sorts the rotations of 1^k 0^(N-k), which the CPU
// tests re-check on these tables.  Step c orders registers (a[c], b[c]),
// a[c] < b[c].
template <int N>
struct BitonicLeaf;  // defined for the odd lengths that occur

template <>
struct BitonicLeaf<3> {
  int n = 3;
  unsigned char a[3] = {0, 0, 1};
  unsigned char b[3] = {1, 2, 2};
};

template <>
struct BitonicLeaf<5> {
  int n = 8;
  unsigned char a[8] = {2, 0, 0, 1, 1, 0, 2, 3};
  unsigned char b[8] = {4, 3, 2, 4, 2, 1, 3, 4};
};

template <>
struct BitonicLeaf<7> {
  int n = 12;
  unsigned char a[12] = {1, 2, 3, 1, 0, 5, 0, 3, 4, 4, 2, 0};
  unsigned char b[12] = {6, 5, 4, 3, 4, 6, 2, 5, 6, 5, 3, 1};
};

template <>
struct BitonicLeaf<25> {
  int n = 72;
  unsigned char a[72] = {
      13, 14, 12, 15, 0, 1, 2, 16, 17, 3, 4, 5, 4, 3, 2, 1, 0, 5, 6, 7, 8, 9, 10, 12, 20, 21, 11,
      10, 9, 8, 7, 6, 5, 4, 0, 1, 1, 2, 3, 0, 8, 9, 10, 11, 16, 17, 18, 19, 22, 19, 18, 15, 14, 11,
      10, 7, 6, 3, 2, 0, 13, 1, 21, 15, 9, 3, 11, 23, 7, 19, 5, 17};
  unsigned char b[72] = {
      23, 22, 24, 21, 11, 10, 9, 20, 19, 8, 7, 6, 18, 17, 16, 15, 14, 19, 20, 21, 22, 23, 24, 13,
      24, 23, 19, 18, 17, 16, 15, 14, 13, 12, 3, 2, 5, 6, 7, 4, 12, 13, 14, 15, 20, 21, 22, 23, 24,
      21, 20, 17, 16, 13, 12, 9, 8, 5, 4, 1, 14, 2, 22, 16, 10, 4, 12, 24, 8, 20, 6, 18};
};

// Sorts registers v[OFF .. OFF+N) holding a cyclic-bitonic sequence.
template <int OFF, int N, int E, typename T>
__device__ __forceinline__ void bitonic_window(T (&v)[E]) {
  if constexpr (N % 2 == 0 && N >= 2) {
#pragma unroll
    for (int t = 0; t < N / 2; ++t) cas(v[OFF + t], v[OFF + t + N / 2]);
    bitonic_window<OFF, N / 2, E, T>(v);
    bitonic_window<OFF + N / 2, N / 2, E, T>(v);
  } else if constexpr (N > 1) {
    constexpr BitonicLeaf<N> net{};
#pragma unroll
    for (int c = 0; c < net.n; ++c) cas(v[OFF + net.a[c]], v[OFF + net.b[c]]);
  }
}

template <int E, typename T>
__device__ __forceinline__ void inlane_bitonic(T (&v)[E]) {
  bitonic_window<0, E, E, T>(v);
}

// Multiplies every register by f (+-1) two at a time (packed f32x2, FMA pipe).
template <int E>
__device__ __forceinline__ void flip(float (&u)[E], float f) {
  const float2 f2 = make_float2(f, f);
#pragma unroll
  for (int t = 0; t + 1 < E; t += 2) {
    const float2 p = __fmul2_rn(make_float2(u[t], u[t + 1]), f2);
    u[t] = p.x;
    u[t + 1] = p.y;
  }
  if constexpr (E % 2) u[E - 1] *= f;
}

// Cross-lane half-cleaners of the alternating layout (below) at lane
// distances D, D/2, ..., 1; s is the sign the lane's values carry.  Lanes D
// apart (D >= 2) have the same orientation, so register t meets register t;
// lanes 1 apart have opposite orientations, so register t meets E-1-t.
template <int E, int D>
__device__ __forceinline__ void alt_half_cleaners(float (&u)[E], int ls, float& s) {
  if constexpr (D >= 1) {
    const float sn = (ls & D) == 0 ? 1.f : -1.f;
    flip(u, sn * s);
    s = sn;
    if constexpr (D >= 2) {
#pragma unroll
      for (int t = 0; t < E; ++t) {
        const float o = __shfl_xor_sync(FULL_MASK, u[t], D);
        u[t] = fminf(u[t], -o);
      }
    } else {
#pragma unroll
      for (int t = 0; t < E / 2; ++t) {
        const float a = __shfl_xor_sync(FULL_MASK, u[E - 1 - t], 1);
        const float b = __shfl_xor_sync(FULL_MASK, u[t], 1);
        u[t] = fminf(u[t], -a);
        u[E - 1 - t] = fminf(u[E - 1 - t], -b);
      }
      if constexpr (E % 2) {  // odd E: the middle register meets itself
        const float o = __shfl_xor_sync(FULL_MASK, u[E / 2], 1);
        u[E / 2] = fminf(u[E / 2], -o);
      }
    }
    alt_half_cleaners<E, D / 2>(u, ls, s);
  }
}

// Merge level of K lanes (two sorted runs of K/2 lanes each become one).
template <int E, int L, int K>
__device__ __forceinline__ void alt_level(float (&u)[E], int ls, float s0) {
  float s = s0;
  if constexpr (K >= 4) {
    // the lower run (lane bit K/2 clear) keeps the minima: it carries +v
    const float sn = (ls & (K / 2)) == 0 ? 1.f : -1.f;
    flip(u, sn * s);
    s = sn;
  }
  // First stage: position i of the block meets position K*E-1-i, which sits
  // in lane ls ^ (K-1) -- of the other orientation -- at the same register.
#pragma unroll
  for (int t = 0; t < E; ++t) {
    const float o = __shfl_xor_sync(FULL_MASK, u[t], K - 1);
    u[t] = fminf(u[t], -o);
  }
  alt_half_cleaners<E, K / 4>(u, ls, s);  // ends with s = s0
  inlane_bitonic(u);
  if constexpr (2 * K <= L) alt_level<E, L, 2 * K>(u, ls, s0);
}

// Float keys in the alternating layout.  Lane ls of a segment holds
// u = s0 * v, s0 = (-1)^(ls & 1), with its registers ascending in u: an even
// lane holds sorted positions E*ls + t in register t, an odd lane holds
// position E*ls + E-1-t in register t (negated values, reversed order).
// In a cross-lane stage the lane that keeps the minima carries +v and its
// partner -v, so both keep fminf(u, -o): min(v, o) in the first, and
// min(-v, -o) = -max(v, o) in the second -- one ALU operation per element.
// Within a lane a compare-exchange is a plain (min, max) on u.  A lane's sign
// changes only when its role in the next stage differs (a multiplication by
// -1 on the FMA pipe); the layout is the same at the end of every merge
// level, so no level ends with a flip.
//
// The caller loads u already signed and pads with a value above every real
// |u|, in registers TR..E-1 of every lane (and possibly lower ones): the
// first, in-lane sort then skips every comparator touching a register at or
// above TR, which would leave both values in place.  After the sort the
// padding of even lanes sits at the top of the sequence and that of odd lanes
// (negated) at the bottom.
template <int E, int L, int TR>
__device__ __forceinline__ void seg_sort_alternating(float (&u)[E], int ls) {
  static_assert((L & (L - 1)) == 0 && L <= 32 && E >= 2, "L a power of two");
  static_assert(TR >= 1 && TR <= E, "padding bound");
  constexpr OemNet<E> net{};
#pragma unroll
  for (int c = 0; c < net.n; ++c)
    if (net.b[c] < TR) cas(u[net.a[c]], u[net.b[c]]);
  if constexpr (L >= 2) alt_level<E, L, 2>(u, ls, (ls & 1) ? -1.f : 1.f);
}

// The same sort with the merge levels as a loop: the level's lane distances
// and each lane's role are run-time values, and the stages of all levels share
// one copy of the code (the mirror stage, the cross-lane half-cleaners at
// distance >= 2 and at distance 1, the in-lane half-cleaners).  Same
// comparisons, same results; the code is several times smaller, for kernels
// whose epilogue leaves the unrolled network short of instruction cache.
template <int E, int L, int TR>
__device__ __forceinline__ void seg_sort_alternating_looped(float (&u)[E], int ls) {
  static_assert((L & (L - 1)) == 0 && L <= 32 && E >= 2, "L a power of two");
  static_assert(TR >= 1 && TR <= E, "padding bound");
  constexpr OemNet<E> net{};
#pragma unroll
  for (int c = 0; c < net.n; ++c)
    if (net.b[c] < TR) cas(u[net.a[c]], u[net.b[c]]);
  const float s0 = (ls & 1) ? -1.f : 1.f;
#pragma unroll 1
  for (int K = 2; K <= L; K <<= 1) {
    float s = s0;
    if (K >= 4) {  // the lower run (lane bit K/2 clear) keeps the minima: it carries +v
      const float sn = (ls & (K / 2)) == 0 ? 1.f : -1.f;
      flip(u, sn * s);
      s = sn;
    }
#pragma unroll
    for (int t = 0; t < E; ++t) {  // mirror: lane ls ^ (K-1), same register
      const float o = __shfl_xor_sync(FULL_MASK, u[t], K - 1);
      u[t] = fminf(u[t], -o);
    }
#pragma unroll 1
    for (int D = K / 4; D >= 1; D >>= 1) {
      const float sn = (ls & D) == 0 ? 1.f : -1.f;
      flip(u, sn * s);
      s = sn;
      if (D >= 2) {
#pragma unroll
        for (int t = 0; t < E; ++t) {
          const float o = __shfl_xor_sync(FULL_MASK, u[t], D);
          u[t] = fminf(u[t], -o);
        }
      } else {
#pragma unroll
        for (int t = 0; t < E / 2; ++t) {
          const float a = __shfl_xor_sync(FULL_MASK, u[E - 1 - t], 1);
          const float b = __shfl_xor_sync(FULL_MASK, u[t], 1);
          u[t] = fminf(u[t], -a);
          u[E - 1 - t] = fminf(u[E - 1 - t], -b);
        }
        if constexpr (E % 2) {  // odd E: the middle register meets itself
          const float o = __shfl_xor_sync(FULL_MASK, u[E / 2], 1);
          u[E / 2] = fminf(u[E / 2], -o);
        }
      }
    }
    inlane_bitonic(u);  // (s is back at s0)
  }
}

template <int E, int L, typename T>
__device__ __forceinline__ void seg_bitonic_sort(T (&v)[E], int ls) {
  static_assert((E & (E - 1)) == 0 && (L & (L - 1)) == 0 && L <= 32 && E >= 2, "powers of two");
  // Block sizes up to E: within the lane, unrolled.
#pragma unroll
  for (int kk = 2; kk <= E; kk <<= 1) {
#pragma unroll
    for (int t = 0; t < E; ++t) {  // mirror stage: i <-> i ^ (kk - 1)
      const int p = t ^ (kk - 1);
      if (p > t) cas(v[t], v[p]);
    }
#pragma unroll
    for (int jj = kk / 4; jj >= 1; jj >>= 1) {  // half-cleaners: i <-> i ^ jj
#pragma unroll
      for (int t = 0; t < E; ++t) {
        const int p = t ^ jj;
        if (p > t) cas(v[t], v[p]);
      }
    }
  }
  // Larger blocks: the lane distances and roles are run-time values and every
  // level ends with the same in-lane half-cleaners, so the levels and their
  // cross-lane stages are loops -- one copy of the code instead of one per
  // stage, which keeps the kernel inside the instruction cache.
#pragma unroll 1
  for (int kk = 2 * E; kk <= E * L; kk <<= 1) {
    {
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
#pragma unroll 1
    for (int d = kk / (4 * E); d >= 1; d >>= 1) {  // half-cleaners at lane distance d
      const bool lower = (ls & d) == 0;
#pragma unroll
      for (int t = 0; t < E; ++t) {
        T o = __shfl_xor_sync(FULL_MASK, v[t], d);
        v[t] = keep_lo_hi(v[t], o, lower);
      }
    }
    inlane_half_cleaners<E, E / 2, T>(v);
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

// Start of the tie run holding the lane's first entry (its position in the
// segment), by the same scan as seg_runs; cont_right as there.  Enough for
// sums that take each run once, at its last entry.  ALT (float keys): the
// lanes hold their values with alternating signs (odd lanes negated), so a
// neighbour's edge value is negated before the comparison.
template <int E, int L, bool ALT = false, typename T, typename KeyEq>
__device__ __forceinline__ int seg_first_run_start(const T (&v)[E], int ls, KeyEq eq,
                                                   bool& cont_right) {
  const int pos0 = E * ls;
  T prev = __shfl_up_sync(FULL_MASK, v[E - 1], 1, L);
  T next = __shfl_down_sync(FULL_MASK, v[0], 1, L);
  if constexpr (ALT) {
    prev = -prev;
    next = -next;
  }
  const bool cont_left = (ls > 0) && eq(prev, v[0]);
  cont_right = (ls < L - 1) && eq(v[E - 1], next);
  int cnt_last = 0;
  bool all_eq = true;
#pragma unroll
  for (int t = 0; t < E; ++t) {
    cnt_last += eq(v[t], v[E - 1]) ? 1 : 0;
    all_eq = all_eq && eq(v[t], v[0]);
  }
  // start of the run holding the lane's last entry (-1: began in an earlier lane)
  int sl = (all_eq && cont_left) ? -1 : pos0 + E - cnt_last;
#pragma unroll
  for (int d = 1; d < L; d <<= 1) {
    const int o = __shfl_up_sync(FULL_MASK, sl, d, L);
    if (ls >= d && sl < 0) sl = o;
  }
  const int carry_s = __shfl_up_sync(FULL_MASK, sl, 1, L);
  return cont_left ? carry_s : pos0;
}

}  // namespace gini

namespace gini {

// ---------------------------------------------------------------------------
// Long segments (m > 1024): a warp sorts the segment in chunks of 1024 slots
// (32 registers x 32 lanes, the 64-bit network above) into shared memory, and
// each element's rank comes from binary searches in every sorted chunk.

constexpr int LONG_CHUNK = 1024;
constexpr int LONG_MAX_CHUNKS = 8;  // m <= 8192

// Shared-memory index of sorted position pos: one word of padding per 32
// keys, so the 32 lanes' stores of one register fall into 16 banks.
__device__ __forceinline__ int long_slot(int pos) { return pos + (pos >> 5); }
constexpr int LONG_CHUNK_SLOTS = LONG_CHUNK + LONG_CHUNK / 32;

// Sorts this warp's chunk of keys (kv[t] = key of chunk position t * 32 +
// lane, ~0 for padding) and stores it ascending at dst[long_slot(pos)].
__device__ __forceinline__ void long_sort_chunk(unsigned long long (&kv)[32], int lane,
                                                unsigned long long* dst) {
  seg_bitonic_sort<32, 32>(kv, lane);
#pragma unroll
  for (int t = 0; t < 32; ++t) dst[long_slot(lane * 32 + t)] = kv[t];
}

// Number of keys below k and equal to k in sorted a[0 .. len) (indices
// through long_slot).
__device__ __forceinline__ void long_count(const unsigned long long* a, int len,
                                           unsigned long long k, int& lt, int& eq) {
  int lo = 0, hi = len;  // first index with a >= k
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[long_slot(mid)] < k) lo = mid + 1;
    else hi = mid;
  }
  int lo2 = lo, hi2 = len;  // first index with a > k
  while (lo2 < hi2) {
    const int mid = (lo2 + hi2) >> 1;
    if (a[long_slot(mid)] <= k) lo2 = mid + 1;
    else hi2 = mid;
  }
  lt += lo;
  eq += lo2 - lo;
}

}  // namespace gini
