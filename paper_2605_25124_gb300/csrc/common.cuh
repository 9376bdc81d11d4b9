// Shared device helpers of libginimds (sm_103a).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "gini_mds.h"

extern "C" void gini_count_launch(unsigned n);

namespace gini {

constexpr unsigned FULL_MASK = 0xffffffffu;
constexpr int TILE = 128;  // edge B of the tiled triangle layout

// Device-side error bits, OR-ed into the first word of the workspace.
constexpr unsigned ERR_NONFINITE = 1u;
constexpr unsigned ERR_TIMEOUT = 2u;
constexpr unsigned ERR_INDEX = 4u;  // a debug build's index check failed
constexpr unsigned ERR_DEGENERATE = 8u;  // a batched fit's Delta summed to zero

// The first 256 bytes of every workspace hold the error word (and, in debug
// builds, the record of the first failed index check at byte 64).
constexpr size_t WS_HEADER = 256;

__device__ __forceinline__ void raise_error(unsigned* err, unsigned bit) {
  if (err) atomicOr(err, bit);
}

// Debug builds (-DGINI_DEBUG_CHECKS) check the offsets the hot kernels compute
// (rows of X, stored Delta entries and tiles, point arrays, partial buffers,
// shared-memory slots) against the extents the call's sizes define.  A failed
// check ORs ERR_INDEX into the error word, keeps the first failure's site
// (file id x 100000 + line), index and bound in the header's record, counts
// the failures, and the access it guards is skipped.  Release builds compile
// every check to `true`, so the kernels are the same as without them.
struct DebugRecord {
  unsigned site;
  unsigned count;
  long long index;
  long long bound;
};
constexpr size_t DEBUG_RECORD_OFF = 64;
static_assert(DEBUG_RECORD_OFF + sizeof(DebugRecord) <= WS_HEADER, "record inside the header");

#ifndef GINI_FILE_ID
#define GINI_FILE_ID 0
#endif

#ifdef GINI_DEBUG_CHECKS
static __device__ __noinline__ void index_fail(unsigned* err, unsigned site, long long idx,
                                               long long bound) {
  if (!err) return;
  atomicOr(err, ERR_INDEX);
  DebugRecord* r = reinterpret_cast<DebugRecord*>(reinterpret_cast<char*>(err) + DEBUG_RECORD_OFF);
  if (atomicCAS(&r->site, 0u, site) == 0u) {
    r->index = idx;
    r->bound = bound;
  }
  atomicAdd(&r->count, 1u);
}
__device__ __forceinline__ bool idx_ok(unsigned* err, unsigned site, long long idx,
                                       long long bound) {
  if (idx >= 0 && idx < bound) return true;
  index_fail(err, site, idx, bound);
  return false;
}
// true when 0 <= idx < bound; otherwise records the failure and is false
#define GINI_IDX_OK(err, idx, bound)                                                    \
  ::gini::idx_ok((err), (unsigned)(GINI_FILE_ID * 100000 + __LINE__), (long long)(idx), \
                 (long long)(bound))
#else
#define GINI_IDX_OK(err, idx, bound) true
#endif

// Number of tiles along one edge for n points.
__host__ __device__ __forceinline__ int64_t tiles_1d(int64_t n) { return (n + TILE - 1) / TILE; }

// Linear index of tile (I, J), I <= J, in the row-major upper-triangular order.
__host__ __device__ __forceinline__ int64_t tile_offset(int64_t I, int64_t J, int64_t T) {
  return I * T - I * (I - 1) / 2 + (J - I);
}

// Inverse of tile_offset: the tile (I, J) with linear index t.  I is the last
// tile row whose first tile is at or before t, found by binary search in
// integers (GB300's FP64 rate is low, and every thread of a CTA decodes its
// first tile at once: a double sqrt here kept the FP64 pipe 10-14 % busy).
__device__ __forceinline__ void tile_decode(int64_t t, int64_t T, int& I, int& J) {
  int64_t lo = 0, hi = T - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (tile_offset(mid, mid, T) <= t) lo = mid;
    else hi = mid - 1;
  }
  I = (int)lo;
  J = (int)(t - tile_offset(lo, lo, T) + lo);
}

// Next tile in row-major upper-triangular order (integer only; GB300's FP64
// rate is far too low for a sqrt per tile).
__host__ __device__ __forceinline__ void tile_next(int& I, int& J, int64_t T) {
  if (++J == T) {
    ++I;
    J = I;
  }
}

// Offset (in elements) of delta(i, j), i < j, in one plane of the tiled layout.
__device__ __forceinline__ int64_t tiled_index(int64_t i, int64_t j, int64_t T) {
  int64_t I = i / TILE, J = j / TILE;
  return tile_offset(I, J, T) * (int64_t)(TILE * TILE) + (i % TILE) * TILE + (j % TILE);
}

// Exact difference a - b = hi + lo for floats (TwoSum, Knuth).  Exact as long
// as nothing underflows.
__device__ __forceinline__ float2 two_diff(float a, float b) {
  float s = __fsub_rn(a, b);
  float bb = __fsub_rn(s, a);
  float lo = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(-b, bb));
  return make_float2(s, lo);
}

// The point pairs of the iteration kernels: u = a - b as (hi, lo * 2^24), with
// hi + lo = a - b exactly (two_diff).  |lo| <= ulp(hi)/2 <= 2^-24 |hi|, so the
// scaled part cannot overflow, and scaling by a power of two is exact and
// keeps the order of the lo parts.  Two pairs' difference is then
// dh = hi_i - hi_j and dl' = lo'_i - lo'_j = 2^24 fl(lo_i - lo_j):
//   the exact sign: a = fma(dh, 2^88, dl') = 2^24 fl(dh 2^64 + dl) (dh decides
//   when it is not zero, dl when it is), and every nonzero a has magnitude at
//   least 2^-125, so sat(fma(a, 2^126, 1/2)) is exactly 0, 1/2 or 1 -- one
//   FMA fewer than scaling a by 2^150 in two steps;
//   the value:     s = fma(dl', 2^-24, dh) = fl(dh + dl), as without the
//   scaling.  Its sign is 0 or the exact sign (rounding is monotone and -dh
//   is a float, so it cannot cross it), so |s| = s sigma exactly.
constexpr float LO_SCALE = 0x1p24f;
constexpr float LO_UNSCALE = 0x1p-24f;
constexpr float SIGN_HI = 0x1p88f;    // weight of dh in a
constexpr float SIGN_SAT = 0x1p126f;  // takes every nonzero a to magnitude >= 2

// |x| of both halves by clearing the sign bits (ALU pipe, not the FMA pipe).
__device__ __forceinline__ float2 abs2_alu(float2 x) {
  return make_float2(__uint_as_float(__float_as_uint(x.x) & 0x7fffffffu),
                     __uint_as_float(__float_as_uint(x.y) & 0x7fffffffu));
}

__device__ __forceinline__ float2 point_pair(float a, float b) {
  const float2 t = two_diff(a, b);
  return make_float2(t.x, t.y * LO_SCALE);
}

// Sign of (p.hi + p.lo) - (q.hi + q.lo) for two exact pairs produced by
// two_diff (|lo| <= ulp(hi)/2), or by point_pair (lo scaled).  Rounding is
// monotone, so different hi parts already order the exact values; equal hi
// parts are ordered by lo.
__device__ __forceinline__ int exact_cmp(float2 p, float2 q) {
  if (p.x != q.x) return p.x < q.x ? -1 : 1;
  if (p.y != q.y) return p.y < q.y ? -1 : 1;
  return 0;
}

__device__ __forceinline__ float bf16_bits_to_float(uint32_t h16) {
  return __uint_as_float(h16 << 16);
}

// Workspaces are 256-byte aligned (cudaMalloc's guarantee): the carved
// regions are 256-byte multiples from the start, so every region keeps the
// alignment bulk copies and vector loads need.
inline bool ws_misaligned(const void* ws) { return (reinterpret_cast<uintptr_t>(ws) & 255) != 0; }

// NVTX range around an entry point's host work (the enqueueing of its
// kernels), named after the entry point, so profilers can group the kernels
// by call (ncu --nvtx --nvtx-include "gini_dist/").  Header-only NVTX 3: a
// no-op unless a profiling tool is attached.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace gini
