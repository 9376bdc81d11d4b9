// Batched Gini-MDS fits: many problems x a nu grid x random restarts, k = 2
// (the loops of Algorithm 1 over nu and over starts, run together).
//
// Every (problem, nu) pair is a "segment" with its own tiled FP32 Delta (built
// by gini_dist, one sort per pair serving the whole nu grid).  One iteration
// of every fit is one launch of a persistent kernel over the flattened list of
// all segments' tiles; a tile's 128 x 128 dissimilarities are loaded into
// registers once and every restart of the segment is evaluated against them,
// so one read of Delta serves R embeddings.  The T iterations (and the final
// stress pass) are captured once into a CUDA graph and relaunched.
//
// The kernel's row-block shape (rows of a tile per warp, and so warps per CTA)
// and the number of CTAs per SM are picked by a small autotuner that times the
// candidates on the caller's batch at its first call and caches the choice.
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#define GINI_FILE_ID 3  // site numbers of the debug index checks
#include "common.cuh"

namespace gini {

constexpr int BATCH_RMAX = 16;  // restarts per segment

struct BatchSeg {
  int64_t n;           // points of the problem
  int64_t tiles;       // tiles along one edge
  int64_t tile_begin;  // first work item (global tile index) of this segment
  int64_t delta_off;   // element offset of its tiled Delta in the pool
  int64_t pt_off;      // point-pair offset of restart 0 (restart r at + r * npad)
  int64_t npad;        // points rounded up to whole tiles
  int64_t h_off;       // accumulator offset of restart 0 (restart r at + r * n)
  int64_t y_off;       // float offset of restart 0 of Y (restart r at + r * 2n)
  int64_t y0_off;      // float offset of restart 0 of Y0 (shared by the nu of a problem)
  float c2;            // 2^{1-nu}
  float scale;         // step: y -= scale * c2 * h  (scale = 2 eta / sum_delta2)
  int fit0;            // index of restart 0 of this segment among all fits
  int sd2_index;       // index of its sum_delta2
};

struct BatchParams {
  const BatchSeg* segs;
  int nseg;
  int restarts;
  int64_t total_tiles;
  const void* delta;   // tiled pool of every segment's Delta (FP32 or BF16)
  float2* P;           // point pairs (hi, lo of y0 - y1)
  float* h;            // gradient accumulators
  double* acc;         // stress accumulators of the current pass: one per fit
  unsigned* err;
  // Deterministic mode (else null): per (tile, restart) partials instead of
  // atomics.  Work item g, restart r: row sums at part[((g R + r) 2) 128 ..],
  // column sums at part[((g R + r) 2 + 1) 128 ..], stress at spart[g R + r];
  // k_batch_det_reduce adds them up per point and per fit in a fixed order.
  float* part;
  float* spart;
  int64_t delta_elems;  // extents of the pool and the point pairs (debug index checks)
  int64_t pts;
};

__device__ __forceinline__ int find_seg(const BatchSeg* segs, int nseg, int64_t g) {
  int lo = 0, hi = nseg - 1;
  while (lo < hi) {  // last segment with tile_begin <= g
    const int mid = (lo + hi + 1) >> 1;
    if (segs[mid].tile_begin <= g) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Sums a[0..ROWS) over the 32 lanes; lane l returns the total of entry
// bit-reverse(l mod ROWS) (ROWS = 8 or 16).
template <int ROWS>
__device__ __forceinline__ float reduce_rows(float (&a)[ROWS], int lane) {
  constexpr int STEPS = ROWS == 16 ? 4 : 3;
#pragma unroll
  for (int s = 0; s < STEPS; ++s) {
    const int h = (ROWS / 2) >> s, x = 1 << s;
    const bool upper = (lane & x) != 0;
#pragma unroll
    for (int i = 0; i < ROWS / 2; ++i) {
      if (i < h) {
        const float send = upper ? a[i] : a[i + h];
        const float keep = upper ? a[i + h] : a[i];
        a[i] = keep + __shfl_xor_sync(FULL_MASK, send, x);
      }
    }
  }
  float v = a[0];
#pragma unroll
  for (int x = ROWS; x < 32; x <<= 1) v += __shfl_xor_sync(FULL_MASK, v, x);
  return v;
}

template <int ROWS>
__device__ __forceinline__ int row_of_lane(int lane) {
  int r = 0;
  constexpr int BITS = ROWS == 16 ? 4 : 3;
#pragma unroll
  for (int b = 0; b < BITS; ++b) r |= ((lane >> b) & 1) << (BITS - 1 - b);
  return r;
}

// Persistent batched iteration.  ROWS rows of a tile per warp, TILE / ROWS
// warps per CTA; lane l takes columns 4l .. 4l+3.  GRAD = false is the final
// stress-only pass.
template <int ROWS, bool GRAD, int DT>
__global__ void __launch_bounds__(TILE / ROWS * 32, ROWS == 16 ? 2 : 0)
k_batch_iter(const BatchParams B) {  // held to 128 registers: two 16-row CTAs per SM
  constexpr int WARPS = TILE / ROWS;
  constexpr int NT = WARPS * 32;
  __shared__ float2 s_u[2][BATCH_RMAX][TILE];  // [rows | cols][restart][point]
  // column and stress partials, double-buffered by restart parity where the
  // static shared memory allows (8 warps): restart r + 1 fills the other
  // buffer while restart r's is still being summed, so one barrier per restart
  // suffices (restart r + 2 reuses a buffer only after every thread has passed
  // restart r + 1's barrier, i.e. finished reading it).  16 warps: one buffer,
  // a second barrier per restart.
  constexpr int NBUF = WARPS <= 8 ? 2 : 1;
  __shared__ float s_col[NBUF][WARPS][TILE];
  __shared__ float s_S[NBUF][WARPS];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int R = B.restarts;
  const int64_t g_begin = B.total_tiles * blockIdx.x / gridDim.x;
  const int64_t g_end = B.total_tiles * (blockIdx.x + 1) / gridDim.x;
  if (g_begin >= g_end) return;
  int s = find_seg(B.segs, B.nseg, g_begin);
  int I, J;
  tile_decode(g_begin - B.segs[s].tile_begin, B.segs[s].tiles, I, J);
  for (int64_t g = g_begin; g < g_end; ++g) {
    if (g > g_begin) {
      tile_next(I, J, B.segs[s].tiles);
      if (I == B.segs[s].tiles) {  // past this segment's last tile
        ++s;
        I = 0;
        J = 0;
      }
    }
    if (!(GINI_IDX_OK(B.err, s, B.nseg))) break;  // (debug builds) uniform over the CTA
    const BatchSeg& sg = B.segs[s];
    const int64_t n = sg.n;
    const int64_t i0 = (int64_t)I * TILE, j0 = (int64_t)J * TILE;
    const int64_t t_local = g - sg.tile_begin;
    const int64_t tile_off = sg.delta_off + t_local * (int64_t)(TILE * TILE);
    // (debug builds) the segment and its tile inside the pool; uniform over
    // the CTA, so skipping the tile skips its barriers in every thread
    if (!(GINI_IDX_OK(B.err, t_local, sg.tiles * (sg.tiles + 1) / 2) &&
          GINI_IDX_OK(B.err, tile_off + TILE * TILE - 1, B.delta_elems)))
      continue;
    // this thread's ROWS x 4 dissimilarities, kept in registers (as floats)
    // for all restarts
    float4 d[ROWS];
#pragma unroll
    for (int q = 0; q < ROWS; ++q) {
      const int64_t off = tile_off + (warp * ROWS + q) * TILE + 4 * lane;
      if (DT == GINI_F32) {
        d[q] = __ldcs(reinterpret_cast<const float4*>(reinterpret_cast<const float*>(B.delta) + off));
      } else {  // GINI_BF16: four bf16 values in 8 bytes
        const uint2 h = __ldcs(reinterpret_cast<const uint2*>(
            reinterpret_cast<const uint16_t*>(B.delta) + off));
        d[q] = make_float4(bf16_bits_to_float(h.x & 0xffffu), __uint_as_float(h.x & 0xffff0000u),
                           bf16_bits_to_float(h.y & 0xffffu), __uint_as_float(h.y & 0xffff0000u));
      }
    }
    __syncthreads();  // previous tile's shared data fully consumed
    for (int e = threadIdx.x; e < 2 * R * TILE; e += NT) {
      const int side = e / (R * TILE), rr = (e / TILE) % R, l = e % TILE;
      const int64_t pt = (side ? j0 : i0) + l;  // < npad: padding pairs are zero
      const int64_t pi = sg.pt_off + rr * sg.npad + pt;
      s_u[side][rr][l] = GINI_IDX_OK(B.err, pi, B.pts) ? B.P[pi] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const bool masked = (I == J) || (i0 + TILE > n) || (j0 + TILE > n);
    const float2 khi = make_float2(SIGN_HI, SIGN_HI);
    const float2 kun = make_float2(LO_UNSCALE, LO_UNSCALE);
    const float2 m1 = make_float2(-1.f, -1.f);
    const float2 k2 = make_float2(2.f, 2.f);
    const float2 nc2 = make_float2(-sg.c2, -sg.c2);
    for (int r = 0; r < R; ++r) {
      float rowv[ROWS];
      float2 col2[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
      float2 S2 = make_float2(0.f, 0.f);
      // columns 4l+2p, 4l+2p+1 as packed pairs, negated: s = u_i - u_j = u_i + (-u_j)
      float2 nuh[2], nul[2];
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        const float2 a = s_u[1][r][4 * lane + 2 * p], b = s_u[1][r][4 * lane + 2 * p + 1];
        nuh[p] = make_float2(-a.x, -b.x);
        nul[p] = make_float2(-a.y, -b.y);
      }
#pragma unroll
      for (int q = 0; q < ROWS; ++q) {
        const int rl = warp * ROWS + q;
        const float2 ur = s_u[0][r][rl];
        const float2 uh2 = make_float2(ur.x, ur.x), ul2 = make_float2(ur.y, ur.y);
        const float2 dv[2] = {make_float2(d[q].x, d[q].y), make_float2(d[q].z, d[q].w)};
        float2 row2 = make_float2(0.f, 0.f);
#pragma unroll
        for (int p = 0; p < 2; ++p) {
          const float2 dh = __fadd2_rn(uh2, nuh[p]);
          const float2 dlo = __fadd2_rn(ul2, nul[p]);  // lo parts scaled by 2^24
          const float2 s2 = __ffma2_rn(dlo, kun, dh);
          // exact sign of u_i - u_j on the FMA pipe: dh dominates dlo unless it is
          // zero; 2^126 takes any nonzero a (>= 2^-125 with the scaled lo parts)
          // to magnitude >= 2, so the saturating FMA gives 1, 1/2 or 0
          const float2 a2 = __ffma2_rn(dh, khi, dlo);
          // sp = (sigma + 1) / 2 in {0, 1/2, 1}: one saturating FMA per column
          const float2 sp = make_float2(__saturatef(fmaf(a2.x, SIGN_SAT, 0.5f)),
                                        __saturatef(fmaf(a2.y, SIGN_SAT, 0.5f)));
          const float2 sig = __ffma2_rn(sp, k2, m1);  // 2 sp - 1
          // r' = delta - c2 |s|; s has the sign 0 or sigma, so |s| = s sigma (an AND)
          float2 rp = __ffma2_rn(nc2, abs2_alu(s2), dv[p]);
          if (masked) {
            const int cl = 4 * lane + 2 * p;
            const bool rok = i0 + rl < n;
            const bool ok0 = rok && (j0 + cl < n) && (I != J || rl < cl);
            const bool ok1 = rok && (j0 + cl + 1 < n) && (I != J || rl < cl + 1);
            rp.x = ok0 ? rp.x : 0.f;
            rp.y = ok1 ? rp.y : 0.f;
          }
          S2 = __ffma2_rn(rp, rp, S2);
          if (GRAD) {  // r' sigma = -(r sign(s))
            row2 = __ffma2_rn(rp, sig, row2);
            col2[p] = __ffma2_rn(rp, sig, col2[p]);
          }
        }
        rowv[q] = -(row2.x + row2.y);
      }
      float S = S2.x + S2.y;
      // column j receives -r sign(s), which is what the packed sums hold
      const float col[4] = {col2[0].x, col2[0].y, col2[1].x, col2[1].y};
      // stress of this (fit, tile)
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) S += __shfl_xor_sync(FULL_MASK, S, o);
      const int buf = NBUF == 2 ? (r & 1) : 0;
      if (lane == 0) s_S[buf][warp] = S;
      if (GRAD) {
        const float rs = reduce_rows<ROWS>(rowv, lane);
        if (lane < ROWS) {
          const int rl = warp * ROWS + row_of_lane<ROWS>(lane);
          const int64_t gi = i0 + rl;
          if (B.part) {
            if (GINI_IDX_OK(B.err, ((g * R + r) * 2) * TILE + rl, B.total_tiles * R * 2 * TILE))
              B.part[((g * R + r) * 2) * TILE + rl] = rs;
          } else if (gi < n) {
            atomicAdd(B.h + sg.h_off + r * n + gi, rs);
          }
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) s_col[buf][warp][4 * lane + c] = col[c];
      }
      __syncthreads();
      if (GRAD && threadIdx.x < TILE) {
        float v = 0.f;
#pragma unroll
        for (int w = 0; w < WARPS; ++w) v += s_col[buf][w][threadIdx.x];
        const int64_t gj = j0 + threadIdx.x;
        if (B.part) {
          if (GINI_IDX_OK(B.err, ((g * R + r) * 2 + 1) * TILE + threadIdx.x,
                          B.total_tiles * R * 2 * TILE))
            B.part[((g * R + r) * 2 + 1) * TILE + threadIdx.x] = v;
        } else if (gj < n) {
          atomicAdd(B.h + sg.h_off + r * n + gj, v);
        }
      }
      if (threadIdx.x == 0) {
        float v = 0.f;
        for (int w = 0; w < WARPS; ++w) v += s_S[buf][w];
        if (B.spart) {
          if (GINI_IDX_OK(B.err, g * R + r, B.total_tiles * R)) B.spart[g * R + r] = v;
        } else {
          atomicAdd(B.acc + sg.fit0 + r, (double)v);
        }
      }
      if constexpr (NBUF == 1) __syncthreads();
    }
  }
}

// Deterministic mode: h of every (segment, restart, point) from the per-tile
// partials, row tiles (I, J >= I) then column tiles (J' <= I, I) in order, and
// (point 0's thread) the fit's stress from its tiles' partials in order.
// One thread per (segment, restart, point), as k_batch_update.
__global__ void k_batch_det_reduce(const BatchSeg* segs, int nseg, int R, const int64_t* pt_prefix,
                                   int64_t total, const float* part, const float* spart,
                                   float* h, double* acc) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= total) return;
  int lo = 0, hi = nseg - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pt_prefix[mid] <= e) lo = mid;
    else hi = mid - 1;
  }
  const BatchSeg& sg = segs[lo];
  const int64_t local = e - pt_prefix[lo];
  const int r = (int)(local / sg.n);
  const int64_t i = local % sg.n;
  const int64_t I = i / TILE, T = sg.tiles;
  const int rl = (int)(i % TILE);
  float v = 0.f;
  for (int64_t J = I; J < T; ++J) {
    const int64_t g = sg.tile_begin + tile_offset(I, J, T);
    v += part[((g * R + r) * 2) * TILE + rl];
  }
  for (int64_t J = 0; J <= I; ++J) {
    const int64_t g = sg.tile_begin + tile_offset(J, I, T);
    v += part[((g * R + r) * 2 + 1) * TILE + rl];
  }
  h[sg.h_off + (int64_t)r * sg.n + i] = v;
  if (i == 0) {
    double S = 0.0;
    const int64_t nt = T * (T + 1) / 2;
    for (int64_t t = 0; t < nt; ++t) S += (double)spart[(sg.tile_begin + t) * R + r];
    acc[sg.fit0 + r] = S;
  }
}

// Y <- Y - scale c2 h (k = 2: the gradient of point i is c2 h_i (1, -1)), then
// refresh the point pairs and clear h.  One thread per (segment, restart, point).
__global__ void k_batch_update(const BatchSeg* segs, int nseg, int R, const int64_t* pt_prefix,
                               int64_t total, float* Y, float2* P, float* h, unsigned* err) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool bad = false;
  if (e < total) {
    int lo = 0, hi = nseg - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (pt_prefix[mid] <= e) lo = mid;
      else hi = mid - 1;
    }
    const BatchSeg& sg = segs[lo];
    const int64_t local = e - pt_prefix[lo];
    const int r = (int)(local / sg.n);
    const int64_t i = local % sg.n;
    float* y = Y + sg.y_off + (int64_t)r * 2 * sg.n + 2 * i;
    float* hp = h + sg.h_off + (int64_t)r * sg.n + i;
    const float gstep = sg.scale * sg.c2 * (*hp);
    const float y0 = y[0] - gstep, y1 = y[1] + gstep;
    y[0] = y0;
    y[1] = y1;
    *hp = 0.f;
    P[sg.pt_off + (int64_t)r * sg.npad + i] = point_pair(y0, y1);
    bad = !isfinite(y0) || !isfinite(y1);
  }
  if (__any_sync(FULL_MASK, bad) && (threadIdx.x & 31) == 0) raise_error(err, ERR_NONFINITE);
}

// Copies Y0 of (problem, restart) into every nu's Y, zero-fills the point
// padding, writes the point pairs and clears h.
__global__ void k_batch_init(const BatchSeg* segs, int nseg, int R, const int64_t* pad_prefix,
                             int64_t total, const float* Y0, float* Y, float2* P, float* h) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= total) return;
  int lo = 0, hi = nseg - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pad_prefix[mid] <= e) lo = mid;
    else hi = mid - 1;
  }
  const BatchSeg& sg = segs[lo];
  const int64_t local = e - pad_prefix[lo];
  const int r = (int)(local / sg.npad);
  const int64_t i = local % sg.npad;
  float2 pr = make_float2(0.f, 0.f);
  if (i < sg.n) {
    const float* y0 = Y0 + sg.y0_off + (int64_t)r * 2 * sg.n + 2 * i;
    float* y = Y + sg.y_off + (int64_t)r * 2 * sg.n + 2 * i;
    y[0] = y0[0];
    y[1] = y0[1];
    pr = point_pair(y0[0], y0[1]);
    h[sg.h_off + (int64_t)r * sg.n + i] = 0.f;
  }
  P[sg.pt_off + (int64_t)r * sg.npad + i] = pr;
}

// A Delta whose squares sum to zero (every pseudo-distance zero) leaves the
// normalised stress undefined: its fits are recorded as degenerate and their S
// is left as the quotient by zero.
__global__ void k_batch_finalize(const BatchSeg* segs, int nseg, int R, const double* sd2,
                                 const double* acc, int iters, int nfits, double* hist,
                                 double* final_out, unsigned* err) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)(iters + 1) * nfits) return;
  const int it = (int)(e / nfits), f = (int)(e % nfits);
  const int s = f / R;
  const double d2 = sd2[segs[s].sd2_index];
  if (it == 0 && !(d2 > 0.0)) raise_error(err, ERR_DEGENERATE);
  const double v = acc[e] / d2;
  if (hist) hist[e] = v;
  if (it == iters && final_out) final_out[f] = v;
}

// ------------------------------------------------------------------- host --

struct BatchPlan {
  std::vector<BatchSeg> segs;
  std::vector<int64_t> pt_prefix, pad_prefix;  // per segment: restarts x points / x padded
  int64_t total_tiles = 0, delta_elems = 0, pts = 0, hs = 0, ys = 0, total_upd = 0,
          total_pad = 0;
  int nfits = 0, max_p = 1;
};

static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

struct BatchWs {
  unsigned* err;
  void* delta;
  double* sd2;
  BatchSeg* segs;
  int64_t* pt_prefix;
  int64_t* pad_prefix;
  float2* P;
  float* h;
  double* acc;
  float* wtab;
  float* part;   // deterministic mode only
  float* spart;
  size_t total;
};

static BatchWs batch_layout(const BatchPlan& pl, int nprob, int n_nu, int iters, bool det,
                            int dtype, char* base) {
  BatchWs w{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = base ? base + off : nullptr;
    off += al256(bytes);
    return p;
  };
  // gini_dist's workspace (error word + weight tables for the largest p) comes
  // first, so its error word is the batch's error word too.
  w.wtab = (float*)take(gini_workspace_size(GINI_OP_DIST, 2, pl.max_p, 0, 0));
  w.err = (unsigned*)w.wtab;
  w.delta = take((dtype == GINI_BF16 ? 2 : 4) * (size_t)pl.delta_elems);
  w.sd2 = (double*)take(sizeof(double) * (size_t)nprob * n_nu);
  w.segs = (BatchSeg*)take(sizeof(BatchSeg) * pl.segs.size());
  w.pt_prefix = (int64_t*)take(sizeof(int64_t) * pl.segs.size());
  w.pad_prefix = (int64_t*)take(sizeof(int64_t) * pl.segs.size());
  w.P = (float2*)take(sizeof(float2) * (size_t)pl.pts);
  w.h = (float*)take(sizeof(float) * (size_t)pl.hs);
  w.acc = (double*)take(sizeof(double) * (size_t)(iters + 1) * pl.nfits);
  const size_t items = (size_t)pl.total_tiles * (pl.nfits / std::max<size_t>(1, pl.segs.size()));
  w.part = det ? (float*)take(sizeof(float) * items * 2 * TILE) : nullptr;
  w.spart = det ? (float*)take(sizeof(float) * items) : nullptr;
  w.total = off;
  return w;
}

static BatchPlan make_plan(const gini_problem* probs, int nprob, const double* nu, int n_nu,
                           int R, double eta0) {
  BatchPlan pl;
  int64_t y0 = 0;
  std::vector<int64_t> y0_off(nprob);
  for (int q = 0; q < nprob; ++q) {
    y0_off[q] = y0;
    y0 += (int64_t)R * 2 * probs[q].n;
    pl.max_p = std::max<int>(pl.max_p, (int)probs[q].p);
  }
  for (int q = 0; q < nprob; ++q) {
    const int64_t n = probs[q].n, T = tiles_1d(n), plane = gini_tiled_elems(n);
    for (int v = 0; v < n_nu; ++v) {
      BatchSeg s{};
      s.n = n;
      s.tiles = T;
      s.tile_begin = pl.total_tiles;
      s.delta_off = pl.delta_elems + (int64_t)v * plane;
      s.npad = T * TILE;
      s.pt_off = pl.pts;
      s.h_off = pl.hs;
      s.y_off = pl.ys;
      s.y0_off = y0_off[q];
      const double c2 = pow(2.0, 1.0 - nu[v]);
      s.c2 = (float)c2;
      // 2 eta / sum_delta2 with eta = gini_default_step(n, 2, nu, sum_delta2, eta0)
      s.scale = (float)(eta0 / ((double)(n - 1) * 2.0 * c2 * c2));
      s.fit0 = pl.nfits;
      s.sd2_index = q * n_nu + v;
      pl.pt_prefix.push_back(pl.total_upd);
      pl.pad_prefix.push_back(pl.total_pad);
      pl.total_tiles += T * (T + 1) / 2;
      pl.pts += (int64_t)R * s.npad;
      pl.hs += (int64_t)R * n;
      pl.ys += (int64_t)R * 2 * n;
      pl.total_upd += (int64_t)R * n;
      pl.total_pad += (int64_t)R * s.npad;
      pl.nfits += R;
      pl.segs.push_back(s);
    }
    pl.delta_elems += (int64_t)n_nu * plane;
  }
  return pl;
}

// --- autotuner ---------------------------------------------------------------

struct TuneChoice {
  int rows = 16;     // rows of a tile per warp (16 -> 8 warps, 8 -> 16 warps per CTA)
  int per_sm = 2;    // CTAs per SM
  int dtype = GINI_F32;  // storage of the Delta pool
};

template <int DT>
static void launch_iter_dt(const TuneChoice& tc, bool grad, unsigned grid, const BatchParams& P,
                           cudaStream_t s) {
  if (tc.rows == 16) {
    if (grad) k_batch_iter<16, true, DT><<<grid, 8 * 32, 0, s>>>(P);
    else k_batch_iter<16, false, DT><<<grid, 8 * 32, 0, s>>>(P);
  } else {
    if (grad) k_batch_iter<8, true, DT><<<grid, 16 * 32, 0, s>>>(P);
    else k_batch_iter<8, false, DT><<<grid, 16 * 32, 0, s>>>(P);
  }
}

static std::mutex g_tune_mu;
static std::map<std::string, TuneChoice> g_tune_cache;

static int sms_of_current_device() {
  int dev = 0, v = 148;
  if (cudaGetDevice(&dev) == cudaSuccess)
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
  return v;
}

static void launch_iter(const TuneChoice& tc, bool grad, const BatchParams& P, cudaStream_t s) {
  const int64_t cap = (int64_t)sms_of_current_device() * tc.per_sm;
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(P.total_tiles, cap));
  gini_count_launch(1);
  if (tc.dtype == GINI_BF16) launch_iter_dt<GINI_BF16>(tc, grad, grid, P, s);
  else launch_iter_dt<GINI_F32>(tc, grad, grid, P, s);
}

static std::string tune_key(const BatchPlan& pl, int R, int dtype) {
  // same tile counts, restarts and storage -> same choice
  return std::to_string(pl.total_tiles) + "/" + std::to_string(pl.segs.size()) + "/" +
         std::to_string(R) + "/" + std::to_string(dtype);
}

// Times every candidate on one gradient pass of the real batch (the
// accumulators it disturbs are reset by the graph before the fit proper).
static TuneChoice autotune(const BatchPlan& pl, int R, int dtype, const BatchParams& P,
                           cudaStream_t s) {
  const std::string key = tune_key(pl, R, dtype);
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) return it->second;
  }
  // Each candidate's best of three rounds, the rounds interleaved so that a
  // slow moment of the GPU does not fall on one candidate only; the default
  // shape (cands[1]) is kept unless another is more than 2 % faster.
  constexpr int NC = 5, ROUNDS = 3;
  const TuneChoice cands[NC] = {{16, 1, dtype}, {16, 2, dtype}, {16, 3, dtype}, {8, 1, dtype},
                                {8, 2, dtype}};
  float best_of[NC];
  for (int c = 0; c < NC; ++c) best_of[c] = 1e30f;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  bool ok = true;
  for (int round = 0; round < ROUNDS && ok; ++round) {
    for (int c = 0; c < NC && ok; ++c) {
      launch_iter(cands[c], true, P, s);  // warm
      cudaEventRecord(e0, s);
      launch_iter(cands[c], true, P, s);
      launch_iter(cands[c], true, P, s);
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        ok = false;
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      best_of[c] = std::min(best_of[c], ms);
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  TuneChoice best = cands[1];
  float best_ms = best_of[1] * 0.98f;
  for (int c = 0; c < NC; ++c) {
    if (best_of[c] < best_ms) {
      best_ms = best_of[c];
      best = cands[c];
    }
  }
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune_cache[key] = best;
  return best;
}

// --- graph cache ---------------------------------------------------------------

struct GraphEntry {
  std::string key;
  cudaGraphExec_t exec = nullptr;
};
static std::mutex g_graph_mu;
static GraphEntry g_graph;

}  // namespace gini

using namespace gini;

extern "C" void gini_set_cuda_error(cudaError_t e);
extern "C" int gini_get_deterministic(void);

static bool batch_det(const gini_batch_opts* o) {
  return (o && o->deterministic) || gini_get_deterministic();
}

static int batch_dtype(const gini_batch_opts* o) { return o ? o->delta_dtype : GINI_F32; }

extern "C" size_t gini_batch_workspace_size(const gini_problem* probs, int nprob, int n_nu,
                                            int restarts, int iters,
                                            const gini_batch_opts* opts) {
  if (!probs || nprob < 1 || n_nu < 1 || restarts < 1 || iters < 0) return 0;
  std::vector<double> nu(n_nu, 2.0);
  BatchPlan pl = make_plan(probs, nprob, nu.data(), n_nu, restarts, 1.0);
  return batch_layout(pl, nprob, n_nu, iters, batch_det(opts), batch_dtype(opts), nullptr).total;
}

extern "C" int gini_fit_batched(const gini_problem* probs, int nprob, const double* nu_host,
                                int n_nu, int restarts, int iters, double eta0,
                                const float* Y0_dev, float* Y_dev, double* history_dev,
                                double* final_stress_dev, int* tuned_rows,
                                const gini_batch_opts* opts, void* ws, size_t ws_bytes,
                                void* stream) {
  NvtxRange nvtx_range("gini_fit_batched");
  if (!probs || !nu_host || !Y0_dev || !Y_dev || !ws) return GINI_EINVAL;
  if (ws_misaligned(ws)) return GINI_EINVAL;
  if (nprob < 1 || n_nu < 1 || n_nu > 8 || restarts < 1 || restarts > BATCH_RMAX || iters < 0)
    return GINI_EINVAL;
  if (!(eta0 > 0.0) || !isfinite(eta0)) return GINI_EINVAL;
  const int dtype = batch_dtype(opts);
  if (dtype != GINI_F32 && dtype != GINI_BF16) return GINI_EINVAL;
  if (opts && opts->tile_rows &&
      ((opts->tile_rows != 8 && opts->tile_rows != 16) || opts->ctas_per_sm < 1 ||
       opts->ctas_per_sm > 3))
    return GINI_EINVAL;
  for (int v = 0; v < n_nu; ++v)
    if (!(nu_host[v] > 1.0) || !isfinite(nu_host[v])) return GINI_EINVAL;
  for (int q = 0; q < nprob; ++q) {
    const gini_problem& pq = probs[q];
    if (!pq.X_dev || pq.n < 2 || pq.n > 65535 * 8 || pq.p < 1 || pq.p > 8192 || pq.ldx < pq.p)
      return GINI_EINVAL;
  }
  BatchPlan pl = make_plan(probs, nprob, nu_host, n_nu, restarts, eta0);
  if (pl.nfits > (1 << 30)) return GINI_EINVAL;
  const bool det = batch_det(opts);
  BatchWs w = batch_layout(pl, nprob, n_nu, iters, det, dtype, reinterpret_cast<char*>(ws));
  if (ws_bytes < w.total) return GINI_ENOMEM;
  cudaStream_t s = (cudaStream_t)stream;

  // 1. Delta for every (problem, nu): one gini_dist per problem, all nu at once.
  cudaError_t e;
  for (int q = 0; q < nprob; ++q) {
    const BatchSeg& s0 = pl.segs[(size_t)q * n_nu];
    const int64_t plane = gini_tiled_elems(probs[q].n);
    const int st = gini_dist(probs[q].X_dev, probs[q].n, probs[q].p, probs[q].ldx, nu_host, n_nu,
                             GINI_LAYOUT_TILED, dtype,
                             reinterpret_cast<char*>(w.delta) +
                                 (size_t)s0.delta_off * (dtype == GINI_BF16 ? 2 : 4),
                             0, plane, nullptr, w.sd2 + (size_t)q * n_nu, w.wtab,
                             gini_workspace_size(GINI_OP_DIST, 2, pl.max_p, 0, 0), stream);
    if (st != GINI_OK) return st;
  }

  // 2. Tables (pageable copies are staged before return).
  e = cudaMemcpyAsync(w.segs, pl.segs.data(), sizeof(BatchSeg) * pl.segs.size(),
                      cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(w.pt_prefix, pl.pt_prefix.data(), sizeof(int64_t) * pl.segs.size(),
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(w.pad_prefix, pl.pad_prefix.data(), sizeof(int64_t) * pl.segs.size(),
                        cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) { gini_set_cuda_error(e); return GINI_ECUDA; }

  BatchParams P{};
  P.segs = w.segs;
  P.nseg = (int)pl.segs.size();
  P.restarts = restarts;
  P.total_tiles = pl.total_tiles;
  P.delta = w.delta;
  P.P = w.P;
  P.h = w.h;
  P.err = w.err;
  P.part = w.part;
  P.spart = w.spart;
  P.delta_elems = pl.delta_elems;
  P.pts = pl.pts;
  const int nseg = (int)pl.segs.size();
  // deterministic mode: h and each fit's stress from the partials of a pass
  auto det_reduce = [&](double* acc) {
    gini_count_launch(1);
    k_batch_det_reduce<<<(unsigned)((pl.total_upd + 255) / 256), 256, 0, s>>>(
        w.segs, nseg, restarts, w.pt_prefix, pl.total_upd, w.part, w.spart, w.h, acc);
  };
  auto init = [&]() {
    gini_count_launch(1);
    k_batch_init<<<(unsigned)((pl.total_pad + 255) / 256), 256, 0, s>>>(
        w.segs, nseg, restarts, w.pad_prefix, pl.total_pad, Y0_dev, Y_dev, w.P, w.h);
  };

  // 3. Autotune on the real batch (first call for this shape only).
  init();
  P.acc = w.acc;
  TuneChoice tc;
  if (opts && opts->tile_rows) tc = TuneChoice{opts->tile_rows, opts->ctas_per_sm, dtype};
  else tc = autotune(pl, restarts, dtype, P, s);
  if (tuned_rows) *tuned_rows = tc.rows * 100 + tc.per_sm;

  // 4. The fit as one graph: reset, T x (iteration + update), final pass, finalize.
  char keybuf[512];
  snprintf(keybuf, sizeof(keybuf), "%p/%p/%p/%p/%p/%d/%d/%d/%lld/%d/%d/%d/%d", ws,
           (const void*)Y0_dev, (void*)Y_dev, (void*)history_dev, (void*)final_stress_dev, iters,
           restarts, nprob, (long long)pl.total_tiles, tc.rows, tc.per_sm, det ? 1 : 0, dtype);
  std::string key(keybuf);
  for (int q = 0; q < nprob; ++q) key += "/" + std::to_string((long long)probs[q].n);
  for (int v = 0; v < n_nu; ++v) key += "/" + std::to_string(nu_host[v]);
  key += "/" + std::to_string(eta0);
  std::lock_guard<std::mutex> lock(g_graph_mu);
  if (g_graph.key != key) {
    if (g_graph.exec) {
      cudaStreamSynchronize(s);
      cudaGraphExecDestroy(g_graph.exec);
      g_graph.exec = nullptr;
    }
    cudaStream_t cap;
    e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) { gini_set_cuda_error(e); return GINI_ECUDA; }
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) { cudaStreamDestroy(cap); gini_set_cuda_error(e); return GINI_ECUDA; }
    {
      cudaStream_t keep = s;
      s = cap;
      cudaMemsetAsync(w.acc, 0, sizeof(double) * (size_t)(iters + 1) * pl.nfits, s);
      init();
      for (int t = 0; t < iters; ++t) {
        P.acc = w.acc + (size_t)t * pl.nfits;
        launch_iter(tc, true, P, s);
        if (det) det_reduce(P.acc);
        gini_count_launch(1);
        k_batch_update<<<(unsigned)((pl.total_upd + 255) / 256), 256, 0, s>>>(
            w.segs, nseg, restarts, w.pt_prefix, pl.total_upd, Y_dev, w.P, w.h, w.err);
      }
      P.acc = w.acc + (size_t)iters * pl.nfits;
      launch_iter(tc, false, P, s);
      if (det) det_reduce(P.acc);
      const int64_t nfin = (int64_t)(iters + 1) * pl.nfits;
      gini_count_launch(1);
      k_batch_finalize<<<(unsigned)((nfin + 255) / 256), 256, 0, s>>>(
          w.segs, nseg, restarts, w.sd2, w.acc, iters, pl.nfits, history_dev, final_stress_dev,
          w.err);
      s = keep;
    }
    cudaGraph_t graph;
    e = cudaStreamEndCapture(cap, &graph);
    cudaStreamDestroy(cap);
    if (e != cudaSuccess) { gini_set_cuda_error(e); return GINI_ECUDA; }
    e = cudaGraphInstantiate(&g_graph.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) { g_graph.exec = nullptr; gini_set_cuda_error(e); return GINI_ECUDA; }
    g_graph.key = key;
  }
  e = cudaGraphLaunch(g_graph.exec, s);
  if (e != cudaSuccess) { gini_set_cuda_error(e); return GINI_ECUDA; }
  return GINI_OK;
}
