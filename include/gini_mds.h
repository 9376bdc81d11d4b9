/*
 * gini_mds.h -- C ABI of libginimds.so, the sm_103a (GB300) Gini-MDS library.
 *
 * What it computes (Mussard & Mussard, "Optimizing Multidimensional Scaling in
 * Gini Metric Spaces"):
 *   - midranks of the components of a vector (Definition 1, Eq. (rank-ties));
 *   - the symmetrized generalized Gini pseudo-distance of Section III-B,
 *       Dbar_{G,nu}(x,y) = 1/2 D_{G,nu}(x,y) + 1/2 D_{G,nu}(y,x),
 *       D_{G,nu}(x,y)    = -d sum_j z_j (Fbar^{nu-1}(z_j) - Fbar^{nu-1}(0)),
 *     z = x - y, ranks taken across the d components of z, midranks for ties,
 *     Fbar(t) = 1 - R(t)/d.  The two terms combine into
 *       Dbar = (d/2) sum_j z_j W(R_j),  W(R) = ((R-1)/d)^{nu-1} - ((d-R)/d)^{nu-1},
 *     which is what the kernels evaluate;
 *   - the dissimilarity matrix Delta = [Dbar(x_i, x_j)] (Algorithm 1);
 *   - Kruskal's stress (Section IV-B) between Delta and the pseudo-distances of
 *     an embedding Y (n x k), normalized as S = sum_{i<j} (d_ij - delta_ij)^2 /
 *     sum_{i<j} delta_ij^2 (KS = sqrt(S)), and its gradient with the ranks held
 *     fixed;
 *   - fixed-step gradient descent on S ("Run MDS" of Algorithm 1).
 *
 * Conventions for every entry point:
 *   - Pointers named *_dev are device memory owned by the caller; pointers
 *     named *_host are host memory owned by the caller.  The library never
 *     allocates device memory: scratch space comes from the caller's
 *     workspace `ws` of `ws_bytes` bytes (see gini_workspace_size), 256-byte
 *     aligned (as cudaMalloc returns; GINI_EINVAL otherwise).  A fresh
 *     workspace must be zero-filled once before first use.
 *   - Work is enqueued on `stream` (a cudaStream_t passed as void*; NULL is
 *     the legacy default stream) and runs asynchronously.  Argument errors are
 *     detected on the host and returned immediately, before anything is
 *     enqueued.  Errors found by the kernels (non-finite data, an expired
 *     bounded wait) are recorded in the workspace and returned by gini_check.
 *   - Return values are gini_status codes.
 *   - Row-major storage; leading dimensions are in elements.
 */
#ifndef GINI_MDS_H
#define GINI_MDS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GINI_OK = 0,
  GINI_EINVAL = 1,      /* invalid argument: size, null pointer, alignment, nu <= 1 */
  GINI_ENONFINITE = 2,  /* NaN or Inf in the input (reported by gini_check) */
  GINI_EDEGENERATE = 3, /* sum of squared dissimilarities is zero: stress undefined
                           (gini_fit_batched, gini_nu_search: reported by gini_check) */
  GINI_ENOMEM = 4,      /* workspace smaller than gini_workspace_size */
  GINI_ECUDA = 5,       /* a CUDA runtime call failed (see gini_last_cuda_error) */
  GINI_ETIMEOUT = 6,    /* a bounded device-side wait expired (reported by gini_check) */
  GINI_EINDEX = 7       /* a device-side index check failed: debug builds only (gini_check) */
} gini_status;

/* Storage type of a dissimilarity matrix. */
typedef enum {
  GINI_F32 = 0,     /* float */
  GINI_BF16 = 1,    /* bfloat16, round to nearest */
  GINI_BF16X2 = 2,  /* two bfloat16 planes, hi = bf16(delta), lo = bf16(delta - hi) */
  GINI_FP8E4M3 = 3  /* e4m3 with a float scale per column: delta ~ q * col_scale[j] */
} gini_dtype;

/* Layout of a dissimilarity matrix. */
typedef enum {
  /* n x n, leading dimension ldd, symmetric, zero diagonal.  F32 only. */
  GINI_LAYOUT_FULL = 0,
  /* Upper triangle in B x B tiles (B = gini_tile_size()).  Tiles (I, J) with
   * I <= J are stored one after another in row-major order of (I, J); inside
   * a tile, element (r, c) is at r*B + c and holds delta(I*B + r, J*B + c).
   * Only entries with row < column and both < n are meaningful; the rest are
   * never read.  One plane holds gini_tiled_elems(n) elements; GINI_BF16X2
   * stores the lo plane right after the hi plane. */
  GINI_LAYOUT_TILED = 1
} gini_layout;

/* Distance measured between embedded points. */
typedef enum {
  GINI_METRIC_GINI = 0,   /* Dbar_{G,nu} in k dimensions (the default) */
  GINI_METRIC_EUCLID = 1  /* ||y_i - y_j||_2, as in Algorithm 1's Kruskal stress line */
} gini_metric;

/* Loss between embedding distances d_ij and dissimilarities delta_ij. */
typedef enum {
  /* S = sum_{i<j} (d - delta)^2 / norm, norm = sum_{i<j} delta^2 (Kruskal) */
  GINI_LOSS_KRUSKAL = 0,
  /* S = sum_{i<j, delta > 0} (d - delta)^2 / delta / norm, norm = sum_{i<j} delta
   * (Sammon, Section IV-B; the objective of Algorithm 2) */
  GINI_LOSS_SAMMON = 1
} gini_loss;

/* Workspace queries (see gini_workspace_size). */
typedef enum {
  GINI_OP_RANK = 0,
  GINI_OP_DIST = 1,
  GINI_OP_STRESS = 2,
  GINI_OP_FIT = 3,
  GINI_OP_STRESS_DET = 4,  /* GINI_OP_STRESS in deterministic mode (larger) */
  GINI_OP_FIT_DET = 5,     /* GINI_OP_FIT in deterministic mode (larger) */
  GINI_OP_DIST_FP8 = 6     /* GINI_OP_DIST with FP8 output (strip scratch) */
} gini_op;

/* Human-readable name of a status code (static string). */
const char* gini_status_str(int status);

/* Last CUDA error string recorded by a failing call on this thread. */
const char* gini_last_cuda_error(void);

/* ABI version of this header (incremented on incompatible change). */
int gini_version(void);

/* Number of kernels the library has launched in this process (all threads,
 * all devices), for launch accounting by callers. */
uint64_t gini_launch_count(void);

/* Tile edge B of GINI_LAYOUT_TILED. */
int gini_tile_size(void);

/* Elements in one plane of the tiled upper triangle for n points:
 * T(T+1)/2 * B*B with T = ceil(n / B). */
int64_t gini_tiled_elems(int64_t n);

/* Bytes of workspace that `op` needs.  n: points (or segments for RANK);
 * m: vector length (features p for DIST, segment length for RANK); k:
 * embedding dimension; iters: iterations (FIT).  Unused arguments are ignored.
 * Returns 0 for an unknown op. */
size_t gini_workspace_size(int op, int64_t n, int64_t m, int k, int iters);

/* Deterministic mode for the calling host thread (0 at start; no
 * counterpart in the paper).  Two things are reduced in a fixed order in
 * every mode, whatever order the CTAs finish in:
 *   - each pass's stress (every CTA stores a partial in its own slot, and the
 *     slots are summed in index order);
 *   - Sum delta^2 of gini_dist (an exact 128-bit integer accumulator).
 * With the mode on, the tiled fused kernels also stop adding row and column
 * gradient terms with float atomics.  They write per-tile partials, which one
 * more kernel per pass sums point by point in a fixed order.  The results of
 * gini_stress_grad(_ex), gini_mds_fit, gini_fit_batched and gini_nu_search
 * are then bit-identical from run to run for equal inputs on one device and
 * library build, and a fit resumed from its own Y_t continues bit for bit.
 * Cost: a few percent per iteration, and the larger workspaces of
 * GINI_OP_STRESS_DET / GINI_OP_FIT_DET (2 B k floats per stored tile, about n^2 k / 32
 * bytes, B = gini_tile_size()).  The plain (FULL) form is deterministic in both
 * modes. */
void gini_set_deterministic(int on);

/* The calling thread's deterministic mode (0 or 1). */
int gini_get_deterministic(void);

/* Synchronizes `stream`, then returns and clears the status the kernels
 * recorded in `ws` since the last gini_check (GINI_OK, GINI_ENONFINITE,
 * GINI_EDEGENERATE, GINI_ETIMEOUT, or in debug builds GINI_EINDEX; precedence
 * EINDEX, ETIMEOUT, EDEGENERATE, ENONFINITE), or
 * GINI_ECUDA if the stream reports an error. */
int gini_check(void* ws, void* stream);

/* Segmented midranks (Definition 1 with midpoint ranks for ties,
 * Eq. (rank-ties)).
 *   v_dev     [nseg][ld] float, segment s = v_dev[s*ld .. s*ld + m)
 *   rank2_dev [nseg][m] int32 out: rank2[s*m + a] = 2 R(v_a)
 *             = 2 #{b: v_b < v_a} + #{b: v_b == v_a} + 1  (exact integers;
 *             -0.0 and +0.0 are equal)
 * 1 <= m <= 8192 (above 1024 the segment is sorted in chunks and ranked by
 * search), ld >= m.  NaN/Inf inputs are reported as GINI_ENONFINITE
 * by gini_check (their ranks are then unspecified). */
int gini_rank(const float* v_dev, int64_t nseg, int64_t m, int64_t ld, int32_t* rank2_dev,
              void* ws, size_t ws_bytes, void* stream);

/* Dissimilarity matrices Delta_q = [Dbar_{G,nu_q}(x_i, x_j)] for every nu_q
 * (Section III-B; Algorithm 1, "Compute Gini pseudo-distances"), one sort of
 * each pair's difference vector serving all nu values.
 *   X_dev      [n][ldx] float data, 2 <= n, 1 <= p <= 8192, ldx >= p (above
 *              1024 one warp sorts each pair's vector in 1024-element chunks
 *              and ranks by search, with n <= 65536)
 *   nu_host    n_nu values, each > 1 and finite, 1 <= n_nu <= 8
 *   layout, dtype: GINI_LAYOUT_FULL with GINI_F32, or GINI_LAYOUT_TILED with
 *              GINI_F32, GINI_BF16, GINI_BF16X2 or GINI_FP8E4M3
 *   delta_dev  output; matrix q starts at element q * nu_stride (in elements
 *              of the storage type; for BF16X2 the stride covers both planes)
 *   ldd        leading dimension of a FULL matrix (>= n); ignored for TILED
 *   col_scale_dev  GINI_FP8E4M3 only (else NULL): n_nu x n floats out; matrix
 *              q's column j holds col_scale[q n + j] = max_{i<j} |delta_ij| / 448
 *              (1 for an all-zero column) and its tiles e4m3(delta_ij /
 *              col_scale[q n + j]) (saturating), as gini_pack stores them.  The
 *              matrix is built one strip of columns at a time into FP32 scratch
 *              in the workspace (at least 4 n B n_nu bytes beyond
 *              gini_workspace_size(GINI_OP_DIST, ...), B = gini_tile_size();
 *              gini_workspace_size(GINI_OP_DIST_FP8, n, p, 0, 0) gives room for
 *              all columns up to 128 MiB; a larger workspace gives wider
 *              strips), so no n x n FP32 intermediate exists.
 *   sum_delta2_dev  n_nu doubles out: sum_{i<j} delta_ij^2 (FP32 values,
 *              exact FP64 sum, the same bits on every run), or NULL
 * The differences x_i - x_j are ranked in their exact order (a single nu = 2
 * or nu = 3 needs no order among equal FP32 values: (d/2) W_{d,3} =
 * ((d-1)/d) (d/2) W_{d,2} is affine in the rank).  Every other nu sorts 32-bit
 * cell keys: twice the FP32 grid index of x_i - x_j when it is an FP32 value,
 * the odd number between two grid indices otherwise; ties between two inexact
 * differences in one FP32 cell are broken by their exact TwoSum pairs.  Sums
 * use the cell end nearer zero (within one FP32 ulp of the difference).
 * Non-finite X is reported as GINI_ENONFINITE by gini_check. */
int gini_dist(const float* X_dev, int64_t n, int64_t p, int64_t ldx, const double* nu_host,
              int n_nu, int layout, int dtype, void* delta_dev, int64_t ldd, int64_t nu_stride,
              float* col_scale_dev, double* sum_delta2_dev, void* ws, size_t ws_bytes,
              void* stream);

/* Converts a FULL F32 dissimilarity matrix (n x n, leading dimension ldd) to
 * the TILED layout of `dtype`.  For GINI_FP8E4M3, col_scale_dev (n floats,
 * out) receives max_{i<j} |delta_ij| / 448 for column j (1 if the column is
 * all zero) and the tile holds e4m3(delta_ij / col_scale[j]) (saturating);
 * col_scale_dev is ignored otherwise.  packed_dev needs gini_tiled_elems(n)
 * elements (two planes for BF16X2). */
int gini_pack(const float* delta_full_dev, int64_t n, int64_t ldd, int dtype, void* packed_dev,
              float* col_scale_dev, void* stream);

/* Normalized Kruskal stress and its gradient for an embedding
 * (Section IV-B; the embedding distance is Dbar_{G,nu} in k dimensions):
 *   S = sum_{i<j} (d_ij - delta_ij)^2 / sum_delta2,  d_ij = Dbar_{G,nu}(y_i, y_j)
 *   dS/dy_i = sum_{j != i} 2 (d_ij - delta_ij) / sum_delta2 * dd_ij/dy_i
 * with the ranks of y_i - y_j held fixed (subgradient W(midrank) at ties).
 *   Y_dev       [n][k] float, 2 <= n, 2 <= k <= 8 (k = 1 makes every
 *               pseudo-distance zero and is rejected)
 *   delta_dev   dissimilarities in (layout, dtype); FULL requires F32.
 *               BF16X2 reads both planes.  col_scale_dev for FP8, else NULL.
 *   ldd         leading dimension for FULL, ignored for TILED
 *   sum_delta2  > 0 (GINI_EDEGENERATE otherwise)
 *   stress_dev  1 double out: S (FP64 reduction)
 *   grad_dev    [n][k] float out, or NULL for the stress only
 * FULL runs the plain form: a forward kernel over i<j, then an adjoint kernel
 * that recomputes every pair.  TILED runs the fused kernel: one pass over the
 * stored triangle produces the stress and both row and column gradient terms. */
int gini_stress_grad(const float* Y_dev, int64_t n, int k, double nu, const void* delta_dev,
                     int layout, int dtype, int64_t ldd, const float* col_scale_dev,
                     double sum_delta2, double* stress_dev, float* grad_dev, void* ws,
                     size_t ws_bytes, void* stream);

/* gini_stress_grad for callers that cannot allocate device memory.  The paper
 * has no counterpart; this is a library service.  Some callers may not call
 * cudaMalloc at all: plugins whose host application owns every byte of device
 * memory through its own pool, and real-time or latency-bound loops that
 * cannot afford the device-wide synchronisation that cudaMalloc and cudaFree
 * imply.  They pass inputs and outputs exactly as for gini_stress_grad, but no
 * workspace: the scratch space is a fixed 8 MiB array inside the library, which
 * every GPU that loads the library holds until the process exits.
 *   - Sizes whose gini_workspace_size(GINI_OP_STRESS, n, 0, k, 0) exceeds 8 MiB
 *     (about 520,000 points at k = 2, 160,000 at k = 3) return GINI_ENOMEM
 *     before anything is enqueued.
 *   - The first call on a device looks up the array's device address with that
 *     device current and keeps it for later calls.
 *   - Nothing is allocated: no cudaMalloc, no cudaFree, no allocating library
 *     routine.  The array keeps the previous call's contents; the call clears
 *     what must start at zero.
 *   - All calls share the one array, so calls whose work overlaps on the GPU
 *     (different streams, or host threads without ordering) race and corrupt
 *     each other's results.  Order them on one stream.
 *   - There is no workspace for gini_check: a device-side error (non-finite Y,
 *     an expired bounded wait) is reported by writing NaN to *stress_dev. */
int gini_stress_grad_noalloc(const float* Y_dev, int64_t n, int k, double nu,
                             const void* delta_dev, int layout, int dtype, int64_t ldd,
                             const float* col_scale_dev, double sum_delta2, double* stress_dev,
                             float* grad_dev, void* stream);

/* gini_stress_grad for any metric and loss.  `norm` is the loss's
 * normaliser (sum_{i<j} delta^2 for Kruskal, sum_{i<j} delta for Sammon; see
 * gini_delta_sums), > 0.  dd/dy is (k/2) W(midrank) for the Gini metric and
 * (y_i - y_j)/d (0 at d = 0) for the Euclidean one.  Same layouts, storage
 * types, workspace and errors as gini_stress_grad (which is the Gini/Kruskal
 * case of this function). */
int gini_stress_grad_ex(const float* Y_dev, int64_t n, int k, double nu, const void* delta_dev,
                        int layout, int dtype, int64_t ldd, const float* col_scale_dev,
                        int metric, int loss, double norm, double* stress_dev, float* grad_dev,
                        void* ws, size_t ws_bytes, void* stream);

/* sums_dev[0] = sum_{i<j} delta_ij and sums_dev[1] = sum_{i<j} delta_ij^2 (FP64)
 * of a stored dissimilarity matrix (any layout and storage type). */
int gini_delta_sums(const void* delta_dev, int64_t n, int layout, int dtype, int64_t ldd,
                    const float* col_scale_dev, double* sums_dev, void* stream);

/* Arguments of gini_mds_fit. */
typedef struct {
  int64_t n;                  /* points, >= 2 */
  int k;                      /* embedding dimension, 2..8 */
  double nu;                  /* > 1 */
  const void* delta_dev;      /* dissimilarities (layout, dtype) as in gini_stress_grad */
  int layout;
  int dtype;
  int64_t ldd;
  const float* col_scale_dev; /* FP8 only */
  double sum_delta2;          /* > 0 */
  double eta;                 /* fixed step on S, > 0 (see gini_default_step) */
  int iters;                  /* T >= 0 */
  int polish_iters;           /* BF16X2 only: the last polish_iters iterations read
                                 hi + lo, earlier ones the hi plane only; the final
                                 stress always reads hi + lo.  Ignored otherwise. */
  float* Y_dev;               /* [n][k] in: Y_0, out: Y_T */
  double* history_dev;        /* iters + 1 doubles out, S(Y_t) for t = 0..T, or NULL */
  double* final_stress_dev;   /* 1 double out, S(Y_T), or NULL */
  int metric;                 /* gini_metric (0: Gini) */
  int loss;                   /* gini_loss (0: Kruskal); sum_delta2 then holds the loss's
                                 normaliser (sum delta^2, or sum delta for Sammon) */
  int deterministic;          /* 1: fixed-order gradient reductions (see
                                 gini_set_deterministic); 0: the thread's setting */
} gini_fit_args;

/* T iterations of Y_{t+1} = Y_t - eta * dS/dY(Y_t) (the "Run MDS" step of
 * Algorithm 1 read as fixed-step gradient descent on Kruskal stress), then
 * S(Y_T).  Each iteration is one pass over Delta: the TILED layout uses the
 * fused stress+adjoint kernel, FULL the plain forward + adjoint kernels. */
int gini_mds_fit(const gini_fit_args* args, void* ws, size_t ws_bytes, void* stream);

/* One data set of a batched fit. */
typedef struct {
  const float* X_dev;  /* [n][ldx] float data */
  int64_t n;           /* points, 2 .. 524,280 */
  int64_t p;           /* features, 1 .. 8192 */
  int64_t ldx;         /* >= p */
} gini_problem;

/* Options of gini_fit_batched (NULL: all zero). */
typedef struct {
  int deterministic;  /* 1: per (tile, restart) partials summed in a fixed order instead of
                         atomics, so results repeat bit for bit (also on when the thread's mode
                         is, gini_set_deterministic); needs the larger workspace below */
  int delta_dtype;    /* storage of the Delta pool: GINI_F32 (0) or GINI_BF16 (half the
                         memory; the iterations read bf16 values) */
  int tile_rows;      /* 0: the autotuner chooses; else 8 or 16 rows of a tile per warp ... */
  int ctas_per_sm;    /* ... and 1..3 CTAs per SM */
} gini_batch_opts;

/* Bytes of workspace gini_fit_batched needs for these problems and options. */
size_t gini_batch_workspace_size(const gini_problem* probs, int nprob, int n_nu, int restarts,
                                 int iters, const gini_batch_opts* opts);

/* Many k = 2 fits at once: every problem x every nu of the grid x `restarts`
 * starting points (the loops of Algorithm 1 over nu and starts).  For each
 * problem one gini_dist call builds Delta for the whole grid (one sort per
 * pair); then each iteration of all fits is one launch of a persistent kernel
 * over every (problem, nu) tile, evaluating all restarts of a tile against one
 * read of its dissimilarities; the T iterations, the final stress pass and the
 * finalisation are captured once into a CUDA graph (kept for later calls with
 * the same arguments) and launched on `stream`.  The kernel's row-block shape
 * and CTAs per SM are chosen by timing the candidates on this batch at its
 * first call (cached per batch shape).  Each fit runs gini_mds_fit's iteration
 * with eta = gini_default_step(n, 2, nu, sum_delta2, eta0).
 *   nu_host      n_nu values (1..8), each > 1
 *   restarts     1..16
 *   Y0_dev       starting points, problem-major: problem q holds restarts x n_q x 2
 *                floats (the same starts serve every nu)
 *   Y_dev        out, (problem, nu, restart)-major: restarts x n_q x 2 floats per
 *                (q, nu)
 *   history_dev  (iters + 1) x nfits doubles out (S after t iterations), or NULL;
 *                fits are ordered (problem, nu, restart)
 *   final_stress_dev  nfits doubles out, S(Y_T)
 *   tuned_config out (host), or NULL: 100 x rows-per-warp + CTAs per SM used
 *   opts         gini_batch_opts, or NULL for the defaults (atomics, FP32 pool,
 *                autotuned shape); the workspace must be sized with the same
 *                options
 * Non-finite data are reported by gini_check(ws, stream), and so is a problem
 * whose Delta for some nu is all zero (GINI_EDEGENERATE: its S values are then
 * the quotient by zero). */
int gini_fit_batched(const gini_problem* probs, int nprob, const double* nu_host, int n_nu,
                     int restarts, int iters, double eta0, const float* Y0_dev, float* Y_dev,
                     double* history_dev, double* final_stress_dev, int* tuned_config,
                     const gini_batch_opts* opts, void* ws, size_t ws_bytes, void* stream);

/* Bytes of workspace gini_nu_search needs (0 on invalid folds or sizes). */
size_t gini_nu_search_workspace_size(int64_t n, int64_t p, const int32_t* fold_host, int K,
                                     int n_nu, int restarts, int iters);

/* The nu search of Algorithm 1: for every nu of the grid and every fold, the
 * fold's dissimilarities (pairs of points of that fold only), `restarts` k = 2
 * fits of `iters` steps as in gini_fit_batched, and KS = sqrt(S(Y_T)) of the
 * best restart; nu* minimises the mean KS over the folds.  The folds are the
 * problems of one gini_fit_batched call per 8 grid values.
 *   X_dev        n x p floats, row stride ldx
 *   fold_host    n fold labels in [0, K) (host); every fold needs >= 2 points
 *   K            1..64 folds; n_nu 1..64 grid values, each > 1
 *   Y0_dev       restarts x n x 2 floats: starting points in point order (a
 *                point's start is the same for every nu)
 *   ks_dev       n_nu x K doubles out (nu-major)
 *   mean_ks_dev  n_nu doubles out
 *   best_dev     one int out: the index of nu* in nu_host (the first minimiser)
 *   Y_dev        n x 2 floats out: each point's embedding in its fold's best
 *                restart at nu*
 * Asynchronous on `stream` except where gini_fit_batched synchronises (its
 * first call for a batch shape times the kernel candidates).  A fold whose
 * Delta is all zero is reported as GINI_EDEGENERATE by gini_check. */
int gini_nu_search(const float* X_dev, int64_t n, int64_t p, int64_t ldx, const int32_t* fold_host,
                   int K, const double* nu_host, int n_nu, int restarts, int iters, double eta0,
                   const float* Y0_dev, double* ks_dev, double* mean_ks_dev, int* best_dev,
                   float* Y_dev, void* ws, size_t ws_bytes, void* stream);

/* Bytes of workspace gini_alternating_nu needs. */
size_t gini_alternating_nu_workspace_size(int64_t n, int64_t p, int k, int n_nu, int iters);

/* The alternating nu update of the heavy-tail experiment (Algorithm 2): from
 * nu_0 = nu_start, for t = 0 .. rounds-1: fit Y (gini_mds_fit, `iters` steps
 * of the given metric and loss, warm-started from the previous round) on
 * Delta_{nu_t}; then KS(nu) = sqrt(Kruskal stress) of that fixed Y against
 * Delta_nu for every nu of the grid (the same metric), and nu_{t+1} = the first
 * minimiser.  Delta is built once for the grid and nu_start (tiled F32, kept in
 * the workspace).  The step is eta0 over a Gershgorin bound on the
 * Gauss-Newton curvature of the loss: with c = k ((k/2) w_max)^2 (Gini
 * metric) or 1 (Euclidean),
 *   Kruskal: eta = eta0 sum delta^2 / (2 (n-1) c)
 *   Sammon:  eta = eta0 sum delta / (2 c max_i sum_{j: delta_ij > 0} 1/delta_ij).
 *   X_dev         n x p floats (p <= 8192), row stride ldx
 *   nu_host       n_nu (1..64) grid values, each > 1; nu_start > 1
 *   k             2..8; metric gini_metric; loss gini_loss (Algorithm 2: Sammon)
 *   Y_dev         n x k floats, in: Y_0, out: the last round's fit
 *   nu_path_host  rounds + 1 doubles out: nu_0 .. nu_rounds
 *   ks_host       rounds x n_nu doubles out: KS(nu) after each round's fit
 * Synchronises `stream` (the host chooses each round's nu); device-side errors
 * are returned directly.  GINI_EDEGENERATE if some Delta is all zero. */
int gini_alternating_nu(const float* X_dev, int64_t n, int64_t p, int64_t ldx, int k,
                        const double* nu_host, int n_nu, double nu_start, int rounds, int iters,
                        double eta0, int metric, int loss, float* Y_dev, double* nu_path_host,
                        double* ks_host, void* ws, size_t ws_bytes, void* stream);

/* Bytes of workspace gini_classical_mds needs. */
size_t gini_cmds_workspace_size(int64_t n, int k);

/* Classical MDS of a dissimilarity matrix (Section IV-A): the top k
 * eigenpairs of B = -1/2 H D2 H (D2 = elementwise squares of Delta,
 * H = I - 11'/n) and the embedding Y = V_k Lambda_k^{1/2} (a negative
 * eigenvalue gives a zero column).  B is not formed: block subspace iteration
 * (16 columns, or n if fewer) streams Delta once per product -- `iters`
 * products plus one for the final Rayleigh-Ritz step; after the first 5 the
 * block iterates on B + s I, s the most negative Ritz value's magnitude, so
 * the largest algebraic eigenvalues are found even where B has large negative
 * ones.  A starting point for gini_mds_fit.
 *   delta_dev    any layout / storage type (as gini_stress_grad)
 *   k            1..8, <= n
 *   iters        >= 1 (20 is ample for well separated eigenvalues)
 *   seed         seeds the start block (SplitMix64 of seed + element index)
 *   Y_dev        [n][k] float out
 *   eigvals_dev  k doubles out, descending
 * EINVAL on bad sizes, layouts or null pointers; ENOMEM when ws_bytes is short
 * of gini_cmds_workspace_size.  Asynchronous on `stream`. */
int gini_classical_mds(const void* delta_dev, int64_t n, int layout, int dtype, int64_t ldd,
                       const float* col_scale_dev, int k, int iters, uint64_t seed,
                       float* Y_dev, double* eigvals_dev, void* ws, size_t ws_bytes,
                       void* stream);

/* Evaluation measures of an embedding (Section V-A and the heavy-tail
 * experiment).  Distances are Euclidean in both spaces; every decision that
 * turns distances into integers (the k nearest neighbours, ranks) compares
 * FP64 squared distances of the FP32 inputs (products and sums rounded
 * separately, features summed in order), ties going to the smaller index.
 * Results are written to device memory; nothing synchronises. */

/* Bytes of workspace the evaluation calls need: n points, n_labels labels
 * (silhouette), spearman != 0 for gini_distance_correlations with ranks (about
 * 40 bytes per pair of points; without, a few hundred bytes). */
size_t gini_eval_workspace_size(int64_t n, int n_labels, int spearman);

/* out_dev[0] = trustworthiness T(k_trust) = 1 - 2 / (n k (2n - 3k - 1)) *
 *   sum_i sum_{j in N_i} max(0, r(i, j) - k), N_i the k nearest neighbours of i
 *   in the embedding, r(i, j) the rank of j by distance from i in the data
 *   (1 = nearest); NaN when k_trust = 0.
 * out_dev[1] = NN(k_nn) = (1 / (n k)) sum_i #{j in N_i: label_j = label_i}
 *   (N_i the k_nn nearest embedding neighbours); NaN when k_nn = 0.
 *   X_dev n x p (row stride ldx), Y_dev n x k (k <= 8), labels_dev n int32 or
 *   NULL when k_nn = 0; 0 <= k_trust, k_nn <= 64, both < n.  One CTA per point;
 *   the data-space pass costs n^2 p FP64 multiply-adds. */
int gini_neighbour_scores(const float* X_dev, int64_t n, int64_t p, int64_t ldx,
                          const float* Y_dev, int k, const int32_t* labels_dev, int k_trust,
                          int k_nn, double* out_dev, void* ws, size_t ws_bytes, void* stream);

/* out_dev[0] = silhouette score (1/n) sum_i (b_i - a_i) / max(a_i, b_i) of the
 * embedding: a_i the mean distance from i to the other points of its label,
 * b_i the smallest mean distance to the points of another label; s_i = 0 when
 * i's label has no other point or no other label has points.  labels_dev: n
 * int32 in [0, n_labels), n_labels 1..64 (a label outside is reported as
 * GINI_ENONFINITE by gini_check and ignored). */
int gini_silhouette(const float* Y_dev, int64_t n, int k, const int32_t* labels_dev, int n_labels,
                    double* out_dev, void* ws, size_t ws_bytes, void* stream);

/* out_dev[0] = Pearson and out_dev[1] = Spearman correlation between the
 * n(n-1)/2 pairwise Euclidean distances of X and those of Y (pairs i < j;
 * Spearman = Pearson of midranks, from a device radix sort of the FP64
 * distances; NaN when spearman = 0).  2 <= n <= 65535. */
int gini_distance_correlations(const float* X_dev, int64_t n, int64_t p, int64_t ldx,
                               const float* Y_dev, int k, int spearman, double* out_dev, void* ws,
                               size_t ws_bytes, void* stream);

/* Diagnostics (no counterpart in the paper): runs the bounded wait that the
 * pipelined kernels use for their bulk copies on a barrier that nothing
 * completes.  After limit_ns (1e3 .. 1e9 ns) the wait gives up and records
 * GINI_ETIMEOUT in ws, which the next gini_check returns; the context stays
 * usable.  It shows that an expired wait ends the kernel instead of hanging
 * the GPU.  ws: at least 256 bytes. */
int gini_selftest_wait_timeout(uint64_t limit_ns, void* ws, size_t ws_bytes, void* stream);

/* Debug builds.  The library compiled with -DGINI_DEBUG_CHECKS (the Python
 * package's build(debug=True), loaded when GINI_DEBUG=1) checks the offsets its
 * hot kernels compute against the extents the call's sizes define: rows of X
 * and the weight tables in the Delta build, every stored Delta entry (FULL,
 * TILED, the FP8 strips), the bulk-copied chunks and point pairs of the fused
 * iteration, the Delta loads of the generic-k iteration, the plain form's rows,
 * the deterministic partials, the batched pool, and the scatter of the ranks.
 * A failed check skips the access it guards, sets the error bit that
 * gini_check returns as GINI_EINDEX, and keeps the first failure's site (file
 * id x 100000 + source line), index and bound, and the number of failures, in
 * the workspace header.  Release builds compile the checks away.
 *
 * gini_debug_checks: 1 in a debug build, 0 otherwise.
 * gini_debug_index_record: synchronises the device, reads the record of the
 *   workspace ws and clears it (site 0: no failure since the last read).
 * gini_selftest_index_check: (debug builds) one kernel that stores at
 *   indices 8, 12, ..., 60 of a 64-float buffer in ws, checked against a bound
 *   of 32: six stores pass, eight fail and are skipped (every index stays
 *   inside the buffer, so a broken check could not write out of bounds);
 *   gini_check then returns GINI_EINDEX.  ws: at least 512 bytes.  Release
 *   builds return GINI_EINVAL and launch nothing. */
int gini_debug_checks(void);
int gini_debug_index_record(void* ws, uint32_t* site, int64_t* index, int64_t* bound,
                            uint32_t* count);
int gini_selftest_index_check(void* ws, size_t ws_bytes, void* stream);

/* A step size for gini_mds_fit: eta0 times the inverse of a Gershgorin bound
 * on the Gauss-Newton curvature of S,
 *   eta = eta0 * sum_delta2 / (2 (n-1) k ((k/2) w_max)^2),  w_max = ((k-1)/k)^{nu-1}.
 * The paper gives no step rule; this one is the library's choice.  Host only. */
double gini_default_step(int64_t n, int k, double nu, double sum_delta2, double eta0);

#ifdef __cplusplus
}
#endif

#endif /* GINI_MDS_H */
