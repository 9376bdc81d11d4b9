// Segmented midranks (Definition 1 with midpoint ranks for ties, Eq. (rank-ties)).
//
// A segment of m <= 1024 values is sorted as 64-bit keys (order-preserving
// bits of the float in the high word, the element's index in the low word) by
// the register bitonic network; tie runs are detected on the high word, and
// 2R = first + last position of the run + 2 is scattered back to the index.
// Longer segments (up to 8192) are sorted in chunks and ranked by search
// (k_rank_long).
#define GINI_FILE_ID 4  // site numbers of the debug index checks
#include "common.cuh"
#include "sortnet.cuh"

namespace gini {

constexpr int RANK_WARPS = 8;

// Monotone map float -> uint32 (total order of non-NaN floats; -0 == +0).
__device__ __forceinline__ uint32_t ordered_bits(float x) {
  uint32_t b = __float_as_uint(x == 0.f ? 0.f : x);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

template <int E, int L>
__global__ void __launch_bounds__(RANK_WARPS * 32)
k_rank(const float* __restrict__ v, int64_t nseg, int m, int64_t ld, int32_t* __restrict__ out,
       unsigned* err) {
  constexpr int G = 32 / L;
  const int lane = threadIdx.x & 31, seg = lane / L, ls = lane % L;
  const int64_t warp_id = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t sidx = warp_id * G + seg;
  const bool active = sidx < nseg;

  unsigned long long key[E];
  bool bad = false;
#pragma unroll
  for (int t = 0; t < E; ++t) {
    const int e = t * L + ls;
    if (active && e < m) {
      const float x = v[sidx * ld + e];
      bad |= !isfinite(x);
      key[t] = ((unsigned long long)ordered_bits(x) << 32) | (unsigned)e;
    } else {
      key[t] = ~0ull;  // padding sorts last; its high word never matches a finite value
    }
  }
  if (__any_sync(FULL_MASK, bad) && lane == 0) raise_error(err, ERR_NONFINITE);

  seg_bitonic_sort<E, L>(key, ls);

  auto eq = [](unsigned long long a, unsigned long long b) { return (a >> 32) == (b >> 32); };
  int run_lo[E];
  int carry_e;
  bool cont_right;
  seg_runs<E, L>(key, ls, eq, run_lo, carry_e, cont_right);
  const int pos0 = E * ls;
  int e = cont_right ? carry_e : pos0 + E - 1;
#pragma unroll
  for (int t = E - 1; t >= 0; --t) {
    if (t < E - 1) e = eq(key[t], key[t + 1]) ? e : pos0 + t;
    // (debug builds) a real position holds a real element's index
    if (active && pos0 + t < m && GINI_IDX_OK(err, (int64_t)(key[t] & 0xffffffffu), m))
      out[sidx * m + (int)(key[t] & 0xffffffffu)] = run_lo[t] + e + 2;
  }
}

// Segments longer than 1024: one warp per segment sorts the value keys
// (ordered bits in the high word) chunk by chunk into shared memory, and each
// element's 2R = 2 #{below} + #{equal, itself included} + 1 comes from
// binary searches in every chunk.
constexpr int RANK_LONG_WARPS = 2;

__global__ void __launch_bounds__(RANK_LONG_WARPS * 32)
k_rank_long(const float* __restrict__ v, int64_t nseg, int m, int64_t ld, int nchunk,
            int32_t* __restrict__ out, unsigned* err) {
  extern __shared__ unsigned long long s_rk[];  // [RANK_LONG_WARPS][nchunk][LONG_CHUNK_SLOTS]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t sidx = (int64_t)blockIdx.x * RANK_LONG_WARPS + warp;
  if (sidx >= nseg) return;  // warp-uniform; no CTA barrier below
  if (!(GINI_IDX_OK(err, m - 1, (int64_t)nchunk * LONG_CHUNK))) return;  // (debug builds)
  unsigned long long* K = s_rk + (size_t)warp * nchunk * LONG_CHUNK_SLOTS;
  const float* row = v + sidx * ld;
  bool bad = false;
  for (int c = 0; c < nchunk; ++c) {
    unsigned long long kv[32];
#pragma unroll
    for (int t = 0; t < 32; ++t) {
      const int e = c * LONG_CHUNK + t * 32 + lane;
      if (e < m) {
        const float x = row[e];
        bad |= !isfinite(x);
        kv[t] = (unsigned long long)ordered_bits(x) << 32;
      } else {
        kv[t] = ~0ull;
      }
    }
    long_sort_chunk(kv, lane, K + (size_t)c * LONG_CHUNK_SLOTS);
  }
  if (__any_sync(FULL_MASK, bad) && lane == 0) raise_error(err, ERR_NONFINITE);
  __syncwarp();
  for (int e = lane; e < m; e += 32) {
    const unsigned long long k = (unsigned long long)ordered_bits(row[e]) << 32;
    int lt = 0, eq = 0;
    for (int c = 0; c < nchunk; ++c)
      long_count(K + (size_t)c * LONG_CHUNK_SLOTS, min(LONG_CHUNK, m - c * LONG_CHUNK), k, lt, eq);
    out[sidx * m + e] = 2 * lt + eq + 1;
  }
}

template <int E, int L>
static cudaError_t launch_rank(const float* v, int64_t nseg, int m, int64_t ld, int32_t* out,
                               unsigned* err, cudaStream_t s) {
  constexpr int G = 32 / L;
  const int64_t warps = (nseg + G - 1) / G;
  const int64_t blocks = (warps + RANK_WARPS - 1) / RANK_WARPS;
  gini_count_launch(1);
  k_rank<E, L><<<(unsigned)blocks, RANK_WARPS * 32, 0, s>>>(v, nseg, m, ld, out, err);
  return cudaGetLastError();
}

}  // namespace gini

using namespace gini;

extern "C" void gini_set_cuda_error(cudaError_t e);

extern "C" int gini_rank(const float* v_dev, int64_t nseg, int64_t m, int64_t ld,
                         int32_t* rank2_dev, void* ws, size_t ws_bytes, void* stream) {
  NvtxRange nvtx_range("gini_rank");
  if (nseg < 0 || m < 1 || m > (int64_t)LONG_CHUNK * LONG_MAX_CHUNKS || ld < m) return GINI_EINVAL;
  if (nseg == 0) return GINI_OK;  // nothing to rank; pointers may be null
  if (!v_dev || !rank2_dev || !ws) return GINI_EINVAL;
  if (ws_misaligned(ws)) return GINI_EINVAL;
  if (ws_bytes < gini_workspace_size(GINI_OP_RANK, nseg, m, 0, 0)) return GINI_ENOMEM;
  if (nseg > ((int64_t)1 << 34)) return GINI_EINVAL;  // grid size limit
  if (m > LONG_CHUNK && nseg > ((int64_t)1 << 31)) return GINI_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned* err = reinterpret_cast<unsigned*>(ws);
  const int mi = (int)m;
  cudaError_t e;
  if (m <= 4) e = launch_rank<4, 1>(v_dev, nseg, mi, ld, rank2_dev, err, s);
  else if (m <= 8) e = launch_rank<8, 1>(v_dev, nseg, mi, ld, rank2_dev, err, s);
  else if (m <= 16) e = launch_rank<16, 1>(v_dev, nseg, mi, ld, rank2_dev, err, s);
  else if (m <= 32) e = launch_rank<16, 2>(v_dev, nseg, mi, ld, rank2_dev, err, s);
  else if (m <= 64) e = launch_rank<16, 4>(v_dev, nseg, mi, ld, rank2_dev, err, s);
  else if (m <= 128) e = launch_rank<16, 8>(v_dev, nseg, mi, ld, rank2_dev, err, s);
  else if (m <= 256) e = launch_rank<16, 16>(v_dev, nseg, mi, ld, rank2_dev, err, s);
  else if (m <= 512) e = launch_rank<16, 32>(v_dev, nseg, mi, ld, rank2_dev, err, s);
  else if (m <= LONG_CHUNK) e = launch_rank<32, 32>(v_dev, nseg, mi, ld, rank2_dev, err, s);
  else {
    const int nchunk = (mi + LONG_CHUNK - 1) / LONG_CHUNK;
    const size_t smem = sizeof(unsigned long long) * RANK_LONG_WARPS * nchunk * LONG_CHUNK_SLOTS;
    e = cudaFuncSetAttribute(k_rank_long, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) {
      gini_count_launch(1);
      k_rank_long<<<(unsigned)((nseg + RANK_LONG_WARPS - 1) / RANK_LONG_WARPS),
                    RANK_LONG_WARPS * 32, smem, s>>>(v_dev, nseg, mi, ld, nchunk, rank2_dev, err);
      e = cudaGetLastError();
    }
  }
  if (e != cudaSuccess) { gini_set_cuda_error(e); return GINI_ECUDA; }
  return GINI_OK;
}
