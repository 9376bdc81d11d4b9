/*
 * FP64 CPU oracle for Gini multidimensional scaling.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU
 * baseline / reference arm of bench.py load this library.  The product path
 * (the CUDA library and its Python binding) never calls it, and the two share
 * no code.
 *
 * Plain, slow and written to be checked against the paper by eye:
 *   - ranks by brute-force counting (Definition 1 and Eq. (rank-ties));
 *   - the generalized pseudo-distance evaluated literally as the paper writes
 *     it: D_{G,nu}(x,y) = -d sum_j z_j (Fbar^{nu-1}(z_j) - Fbar^{nu-1}(0)),
 *     z = x - y, and its symmetrization 1/2 D(x,y) + 1/2 D(y,x) (Section III-B);
 *   - the Gini norm and D_G of Section III-A (Definitions 1 and 2);
 *   - Kruskal's stress over i<j (Section IV-B) and its gradient by a double
 *     loop over all ordered pairs, ranks held fixed;
 *   - fixed-step gradient descent on the normalized stress.
 * Everything is double precision; OpenMP splits only the outer loop over rows.
 *
 * Readings where the paper is silent or garbled:
 *   - Ties get midranks (the mean of the tied positions), as the prose before
 *     Eq. (rank-ties) says; the printed fraction is garbled.
 *   - Fbar is the empirical survival function of the ranked vector,
 *     Fbar(t) = 1 - R(t)/d with midranks, and Fbar(0) = 1 - R(0)/d with
 *     R(0) = (d+1)/2 as Section III-A states.
 *   - Ranks are taken across the d components of one pair's difference
 *     vector (Definition 2; Section V-B says so explicitly).
 *   - A difference z_a = x_a - y_a is kept exactly as an FP64 TwoSum pair
 *     (hi, lo); components are compared lexicographically on (hi, lo).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct { double hi, lo; } orc_dd;

/* Exact difference a - b as hi + lo (Knuth's TwoSum applied to a and -b). */
static orc_dd two_diff(double a, double b) {
  orc_dd r;
  double nb = -b;
  double s = a + nb;
  double bb = s - a;
  r.hi = s;
  r.lo = (a - (s - bb)) + (nb - bb);
  return r;
}

static int dd_lt(orc_dd x, orc_dd y) { return x.hi < y.hi || (x.hi == y.hi && x.lo < y.lo); }
static int dd_eq(orc_dd x, orc_dd y) { return x.hi == y.hi && x.lo == y.lo; }

void orc_set_threads(int t) {
#ifdef _OPENMP
  if (t > 0) omp_set_num_threads(t);
#else
  (void)t;
#endif
}

int orc_get_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Twice the midrank of every element of v:
 *   2 R(v_a) = 2 #{b : v_b < v_a} + #{b : v_b = v_a} + 1,
 * i.e. R = #{<} + (#{=} + 1)/2 (ties share the mean of their positions).
 * Definition 1 with the midpoint rule for ties (Eq. (rank-ties)). */
void orc_midrank2(const double* v, int64_t m, int32_t* r2) {
  for (int64_t a = 0; a < m; ++a) {
    int64_t lt = 0, eq = 0;
    for (int64_t b = 0; b < m; ++b) {
      if (v[b] < v[a]) ++lt;
      else if (v[b] == v[a]) ++eq;
    }
    r2[a] = (int32_t)(2 * lt + eq + 1);
  }
}

/* Same counting rule on exact differences held as (hi, lo). */
static void midrank2_dd(const orc_dd* z, int64_t m, int32_t* r2) {
  for (int64_t a = 0; a < m; ++a) {
    int64_t lt = 0, eq = 0;
    for (int64_t b = 0; b < m; ++b) {
      if (dd_lt(z[b], z[a])) ++lt;
      else if (dd_eq(z[b], z[a])) ++eq;
    }
    r2[a] = (int32_t)(2 * lt + eq + 1);
  }
}

/* Gini norm ||x||_G = sum_j x_j (R(x_j) - R(0)), R(0) = (d+1)/2
 * (Definition 1, Eq. (Gini-norm), midranks for ties). */
double orc_gini_norm(const double* x, int64_t d) {
  int32_t* r2 = (int32_t*)malloc(sizeof(int32_t) * (size_t)d);
  orc_midrank2(x, d, r2);
  double r0 = (double)(d + 1) / 2.0, s = 0.0;
  for (int64_t j = 0; j < d; ++j) s += x[j] * (r2[j] / 2.0 - r0);
  free(r2);
  return s;
}

/* D_G(x,y) = ||x - y||_G = sum_j (x_j - y_j)(R(x_j - y_j) - R(0)) (Definition 2),
 * with the ranks of the exact differences. */
double orc_gini_dg(const double* x, const double* y, int64_t d) {
  orc_dd* z = (orc_dd*)malloc(sizeof(orc_dd) * (size_t)d);
  int32_t* r2 = (int32_t*)malloc(sizeof(int32_t) * (size_t)d);
  for (int64_t j = 0; j < d; ++j) z[j] = two_diff(x[j], y[j]);
  midrank2_dd(z, d, r2);
  double r0 = (double)(d + 1) / 2.0, s = 0.0;
  for (int64_t j = 0; j < d; ++j) s += (z[j].hi + z[j].lo) * (r2[j] / 2.0 - r0);
  free(z);
  free(r2);
  return s;
}

/* One asymmetric term D_{G,nu} for the difference vector z with midranks r2:
 *   -d sum_j z_j (Fbar(z_j)^{nu-1} - Fbar(0)^{nu-1}),  Fbar(t) = 1 - R(t)/d.
 * If dz is given, dz[j] += scale * dD/dz_j with the ranks held fixed. */
static double d_gnu(const orc_dd* z, const int32_t* r2, int64_t d, double nu,
                    double* dz, double scale) {
  double dd_ = (double)d;
  double f0 = 1.0 - ((dd_ + 1.0) / 2.0) / dd_;
  double f0p = pow(f0, nu - 1.0);
  double s = 0.0;
  for (int64_t j = 0; j < d; ++j) {
    double fb = 1.0 - (r2[j] / 2.0) / dd_;
    double w = pow(fb, nu - 1.0) - f0p;
    s += (z[j].hi + z[j].lo) * w;
    if (dz) dz[j] += scale * (-dd_ * w);
  }
  return -dd_ * s;
}

/* Symmetrized generalized Gini pseudo-distance
 *   Dbar_{G,nu}(x,y) = 1/2 D_{G,nu}(x,y) + 1/2 D_{G,nu}(y,x)   (Section III-B),
 * both terms evaluated literally, each with the ranks of its own difference
 * vector.  If dz is non-NULL it receives dDbar/dz_j for z = x - y, ranks fixed. */
static double pd_work(const double* x, const double* y, int64_t d, double nu,
                      double* dz, orc_dd* zf, orc_dd* zb, int32_t* rf, int32_t* rb) {
  for (int64_t j = 0; j < d; ++j) {
    zf[j] = two_diff(x[j], y[j]);
    zb[j] = two_diff(y[j], x[j]);
  }
  midrank2_dd(zf, d, rf);
  midrank2_dd(zb, d, rb);
  if (dz) memset(dz, 0, sizeof(double) * (size_t)d);
  double a = d_gnu(zf, rf, d, nu, dz, 0.5);
  /* D(y,x) is a function of -z: d/dz = -d/d(-z). */
  double b = d_gnu(zb, rb, d, nu, dz, -0.5);
  return 0.5 * a + 0.5 * b;
}

typedef struct {
  orc_dd* zf;
  orc_dd* zb;
  int32_t* rf;
  int32_t* rb;
  double* xi;
  double* xj;
  double* dz;
} orc_work;

static void work_alloc(orc_work* w, int64_t d) {
  w->zf = (orc_dd*)malloc(sizeof(orc_dd) * (size_t)d);
  w->zb = (orc_dd*)malloc(sizeof(orc_dd) * (size_t)d);
  w->rf = (int32_t*)malloc(sizeof(int32_t) * (size_t)d);
  w->rb = (int32_t*)malloc(sizeof(int32_t) * (size_t)d);
  w->xi = (double*)malloc(sizeof(double) * (size_t)d);
  w->xj = (double*)malloc(sizeof(double) * (size_t)d);
  w->dz = (double*)malloc(sizeof(double) * (size_t)d);
}

static void work_free(orc_work* w) {
  free(w->zf); free(w->zb); free(w->rf); free(w->rb);
  free(w->xi); free(w->xj); free(w->dz);
}

double orc_pd(const double* x, const double* y, int64_t d, double nu) {
  orc_work w;
  work_alloc(&w, d);
  double r = pd_work(x, y, d, nu, NULL, w.zf, w.zb, w.rf, w.rb);
  work_free(&w);
  return r;
}

double orc_pd_grad(const double* x, const double* y, int64_t d, double nu, double* dz) {
  orc_work w;
  work_alloc(&w, d);
  double r = pd_work(x, y, d, nu, dz, w.zf, w.zb, w.rf, w.rb);
  work_free(&w);
  return r;
}

/* Dissimilarity matrices Delta[q] = [Dbar_{G,nu_q}(x_i, x_j)] for every nu_q
 * (Algorithm 1: "Compute Gini pseudo-distances"), full symmetric n x n with a
 * zero diagonal, stored q-major.  sum_delta2[q] = sum_{i<j} delta_ij^2, the
 * denominator of Kruskal's stress (Section IV-B). */
void orc_delta(const float* X, int64_t n, int64_t p, int64_t ldx, const double* nus,
               int n_nu, double* Delta, double* sum_delta2) {
  for (int q = 0; q < n_nu; ++q) sum_delta2[q] = 0.0;
#pragma omp parallel
  {
    orc_work w;
    work_alloc(&w, p);
    double* acc = (double*)calloc((size_t)n_nu, sizeof(double));
#pragma omp for schedule(dynamic, 1)
    for (int64_t i = 0; i < n; ++i) {
      for (int64_t c = 0; c < p; ++c) w.xi[c] = (double)X[i * ldx + c];
      for (int q = 0; q < n_nu; ++q) Delta[((int64_t)q * n + i) * n + i] = 0.0;
      for (int64_t j = i + 1; j < n; ++j) {
        for (int64_t c = 0; c < p; ++c) w.xj[c] = (double)X[j * ldx + c];
        for (int q = 0; q < n_nu; ++q) {
          double v = pd_work(w.xi, w.xj, p, nus[q], NULL, w.zf, w.zb, w.rf, w.rb);
          Delta[((int64_t)q * n + i) * n + j] = v;
          Delta[((int64_t)q * n + j) * n + i] = v;
          acc[q] += v * v;
        }
      }
    }
#pragma omp critical
    for (int q = 0; q < n_nu; ++q) sum_delta2[q] += acc[q];
    free(acc);
    work_free(&w);
  }
}

/* delta for listed pairs only: out[t * n_nu + q] = Dbar_{G,nu_q}(x_I[t], x_J[t]). */
void orc_delta_pairs(const float* X, int64_t n, int64_t p, int64_t ldx, const double* nus,
                     int n_nu, const int64_t* I, const int64_t* J, int64_t npairs,
                     double* out) {
  (void)n;
#pragma omp parallel
  {
    orc_work w;
    work_alloc(&w, p);
#pragma omp for schedule(dynamic, 4)
    for (int64_t t = 0; t < npairs; ++t) {
      for (int64_t c = 0; c < p; ++c) {
        w.xi[c] = (double)X[I[t] * ldx + c];
        w.xj[c] = (double)X[J[t] * ldx + c];
      }
      for (int q = 0; q < n_nu; ++q)
        out[t * n_nu + q] = pd_work(w.xi, w.xj, p, nus[q], NULL, w.zf, w.zb, w.rf, w.rb);
    }
    work_free(&w);
  }
}

/* Embedding pseudo-distances d_ij = Dbar_{G,nu}(y_i, y_j) for listed pairs. */
void orc_embed_dist_pairs(const double* Y, int64_t n, int k, double nu, const int64_t* I,
                          const int64_t* J, int64_t npairs, double* out) {
  (void)n;
#pragma omp parallel
  {
    orc_work w;
    work_alloc(&w, k);
#pragma omp for schedule(static)
    for (int64_t t = 0; t < npairs; ++t)
      out[t] = pd_work(Y + I[t] * k, Y + J[t] * k, k, nu, NULL, w.zf, w.zb, w.rf, w.rb);
    work_free(&w);
  }
}

/* Normalized Kruskal stress S = sum_{i<j} (d_ij - delta_ij)^2 / sum_delta2 with
 * d_ij = Dbar_{G,nu}(y_i, y_j) (Section IV-B; KS = sqrt(S)).  If grad is
 * non-NULL it receives dS/dY (n x k), ranks held fixed:
 *   dS/dy_i = sum_{j != i} 2 (d_ij - delta_ij)/sum_delta2 * dDbar(y_i, y_j)/dz,
 * z = y_i - y_j, a double loop over all ordered pairs.  Delta is n x n with
 * leading dimension ldd. */
double orc_stress_grad(const double* Y, int64_t n, int k, double nu, const double* Delta,
                       int64_t ldd, double sum_delta2, double* grad) {
  double S = 0.0;
#pragma omp parallel reduction(+ : S)
  {
    orc_work w;
    work_alloc(&w, k);
#pragma omp for schedule(dynamic, 4)
    for (int64_t i = 0; i < n; ++i) {
      if (grad) for (int c = 0; c < k; ++c) grad[i * k + c] = 0.0;
      for (int64_t j = 0; j < n; ++j) {
        if (j == i) continue;
        double dij = pd_work(Y + i * k, Y + j * k, k, nu, grad ? w.dz : NULL, w.zf, w.zb,
                             w.rf, w.rb);
        double r = dij - Delta[i * ldd + j];
        if (j > i) S += r * r;
        if (grad)
          for (int c = 0; c < k; ++c) grad[i * k + c] += 2.0 * r / sum_delta2 * w.dz[c];
      }
    }
    work_free(&w);
  }
  return S / sum_delta2;
}

/* Gradient rows only: grad_rows[t] = dS/dy_{rows[t]}, with Delta_rows[t] the
 * full row rows[t] of Delta (length n). */
void orc_grad_rows(const double* Y, int64_t n, int k, double nu, const double* Delta_rows,
                   const int64_t* rows, int64_t nr, double sum_delta2, double* grad_rows) {
#pragma omp parallel
  {
    orc_work w;
    work_alloc(&w, k);
#pragma omp for schedule(dynamic, 1)
    for (int64_t t = 0; t < nr; ++t) {
      int64_t i = rows[t];
      for (int c = 0; c < k; ++c) grad_rows[t * k + c] = 0.0;
      for (int64_t j = 0; j < n; ++j) {
        if (j == i) continue;
        double dij = pd_work(Y + i * k, Y + j * k, k, nu, w.dz, w.zf, w.zb, w.rf, w.rb);
        double r = dij - Delta_rows[t * n + j];
        for (int c = 0; c < k; ++c) grad_rows[t * k + c] += 2.0 * r / sum_delta2 * w.dz[c];
      }
    }
    work_free(&w);
  }
}

/* Fixed-step gradient descent on the normalized stress ("Run MDS" of
 * Algorithm 1 read as stress minimization):
 *   Y_{t+1} = Y_t - eta * dS/dY(Y_t),  t = 0 .. T-1.
 * history[t] = S(Y_t) for t = 0..T (history[T] is the stress of the returned Y).
 * Y (n x k) is updated in place. */
void orc_fit(const double* Delta, int64_t n, int k, double nu, double sum_delta2, double eta,
             int T, double* Y, double* history) {
  double* g = (double*)malloc(sizeof(double) * (size_t)(n * k));
  for (int t = 0; t < T; ++t) {
    double S = orc_stress_grad(Y, n, k, nu, Delta, n, sum_delta2, g);
    if (history) history[t] = S;
    for (int64_t e = 0; e < n * k; ++e) Y[e] -= eta * g[e];
  }
  double S = orc_stress_grad(Y, n, k, nu, Delta, n, sum_delta2, NULL);
  if (history) history[T] = S;
  free(g);
}

/* ------------------------------------------------------------------------- *
 * Embedding losses beyond Kruskal stress with Gini distances.
 *   metric 0: d_ij = Dbar_{G,nu}(y_i, y_j)      (as above)
 *   metric 1: d_ij = ||y_i - y_j||_2            (Euclidean, Algorithm 1's KS line)
 *   loss 0 (Kruskal): S = sum_{i<j} (d_ij - delta_ij)^2 / norm, norm = sum delta^2
 *   loss 1 (Sammon):  S = sum_{i<j, delta_ij > 0} (d_ij - delta_ij)^2 / delta_ij / norm,
 *                     norm = sum_{i<j} delta_ij  (Section IV-B, Sammon loss)
 * grad[i] = dS/dy_i by a double loop over ordered pairs; the Euclidean
 * derivative (y_i - y_j)/d_ij is taken as 0 at d_ij = 0.
 * ------------------------------------------------------------------------- */
static double euclid_grad(const double* x, const double* y, int k, double* dz) {
  double s = 0.0;
  for (int c = 0; c < k; ++c) s += (x[c] - y[c]) * (x[c] - y[c]);
  double d = sqrt(s);
  if (dz)
    for (int c = 0; c < k; ++c) dz[c] = d > 0.0 ? (x[c] - y[c]) / d : 0.0;
  return d;
}

double orc_stress_grad_ex(const double* Y, int64_t n, int k, double nu, const double* Delta,
                          int64_t ldd, int metric, int loss, double norm, double* grad) {
  double S = 0.0;
#pragma omp parallel reduction(+ : S)
  {
    orc_work w;
    work_alloc(&w, k);
#pragma omp for schedule(dynamic, 4)
    for (int64_t i = 0; i < n; ++i) {
      if (grad) for (int c = 0; c < k; ++c) grad[i * k + c] = 0.0;
      for (int64_t j = 0; j < n; ++j) {
        if (j == i) continue;
        const double* yi = Y + i * k;
        const double* yj = Y + j * k;
        double dij = metric == 1 ? euclid_grad(yi, yj, k, grad ? w.dz : NULL)
                                 : pd_work(yi, yj, k, nu, grad ? w.dz : NULL, w.zf, w.zb, w.rf,
                                           w.rb);
        double delta = Delta[i * ldd + j];
        double r = dij - delta;
        double wgt = 1.0;
        if (loss == 1) {
          if (!(delta > 0.0)) continue;
          wgt = 1.0 / delta;
        }
        if (j > i) S += wgt * r * r;
        if (grad)
          for (int c = 0; c < k; ++c) grad[i * k + c] += 2.0 * wgt * r / norm * w.dz[c];
      }
    }
    work_free(&w);
  }
  return S / norm;
}
