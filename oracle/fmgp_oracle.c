/*
 * FastMuyGPs oracle: a plain, slow, obviously correct CPU restatement of the
 * posterior-mean path of "Fast Gaussian Process Posterior Mean Prediction via
 * Local Cross Validation and Precomputation" (Dunton, Priest, Muyskens).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and
 * bench.py's CPU-baseline / reference legs may load it.  It shares no code,
 * header, table or helper with the CUDA library, and the CUDA library never
 * calls it.
 *
 * Arithmetic: IEEE FP64, compiled with -O2 -ffp-contract=off (no FMA
 * contraction, no fast-math), OpenMP across independent rows only.
 *
 * Blocks guarded by ORACLE_MUTANT_* plant one mistake each; only the mutation
 * test compiles them (tests/test_oracle_mutations.py) to show that the pins
 * catch it.  The oracle proper is built without any of these macros.
 *
 * Parity pins (tests/test_oracle_pins.py): Matern closed forms against the
 * Bessel form of Eq. 3 (scipy.special.kv); kNN against an all-pairs numpy
 * lexsort on tie-heavy integer grids; blocks symmetric and SPD; k = n reduces
 * to the dense GP mean of Eq. 2 (scipy cho_solve); interpolation identity at
 * z = x_i; leave-one-out block-inverse identity linking Eq. 6 to Eq. 5;
 * sigma^2 invariance of the mean; long-double re-evaluation of the FP64
 * rounding error; the Metropolis calibration chain of Sec. 4.2 against the
 * closed-form (truncated Gaussian) posterior of a linear response, and its
 * greedy and always-accept limits.  The paper prints no worked example, so
 * no printed value pins the oracle directly.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  int kind;             /* 0 = Matern, 1 = RBF */
  double nu;            /* Matern smoothness: 0.5, 1.5 or 2.5 */
  double length_scale;  /* rho */
  double variance;      /* sigma^2 */
  double nugget;        /* tau^2 */
} fmgp_oracle_kernel;

/* ---------------------------------------------------------------- FP64 -- */
#define REAL double
#define FN(name) name##_f64
#define EXP exp
#define SQRT sqrt
#include "oracle_core.h"
#undef REAL
#undef FN
#undef EXP
#undef SQRT

/* ---------------------------------------------------------- long double -- */
#define REAL long double
#define FN(name) name##_ld
#define EXP expl
#define SQRT sqrtl
#include "oracle_core.h"
#undef REAL
#undef FN
#undef EXP
#undef SQRT

static int kernel_ok(const fmgp_oracle_kernel* kp) {
  if (!kp) return 0;
  if (kp->kind == 0 && !(kp->nu == 0.5 || kp->nu == 1.5 || kp->nu == 2.5)) return 0;
  if (kp->kind != 0 && kp->kind != 1) return 0;
  if (!(kp->length_scale > 0) || !(kp->variance > 0) || !(kp->nugget >= 0)) return 0;
  return 1;
}

/* Canonical neighbour-ranking key: D(a,b) = sum_j (a_j - b_j)^2 in FP64,
 * accumulated left to right from 0, every subtraction, product and sum
 * rounded on its own (no FMA).  Candidates are ordered by (D, index). */
double fmgp_oracle_key(const double* a, const double* b, int d) {
  double s = 0.0;
  for (int j = 0; j < d; ++j) {
    double t = a[j] - b[j];
    double t2 = t * t;
    s = s + t2;
  }
  return s;
}

/* Brute-force k-nearest-neighbour query (the neighbour queries of
 * Algorithms 1 and 2 and the test-point lookup).  For each query q, every training j (j != exclude[q] when an
 * exclusion list is given: the query's own index for self-queries) is
 * scanned in index order and kept in a sorted list of the kq smallest
 * (key, j); a later j never displaces an equal key, so ties go to the lowest
 * index.  idx_out / key_out are m x kq.  Returns 0, or 1 on bad arguments. */
int fmgp_oracle_knn(const double* X, int64_t n, int d, const double* Q, int64_t m, int kq,
                    const int64_t* exclude, int32_t* idx_out, double* key_out) {
  if (n < 1 || d < 1 || kq < 1 || m < 0) return 1;
  if (kq > n - (exclude ? 1 : 0)) return 1;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t q = 0; q < m; ++q) {
    double* best = (double*)malloc(sizeof(double) * kq);
    int32_t* bidx = (int32_t*)malloc(sizeof(int32_t) * kq);
    int cnt = 0;
    for (int64_t j = 0; j < n; ++j) {
      if (exclude && j == exclude[q]) continue;
      double D = fmgp_oracle_key(Q + q * d, X + j * d, d);
#ifdef ORACLE_MUTANT_TIE_HIGH
      if (cnt == kq && !(D <= best[kq - 1])) continue;
      int p = (cnt < kq) ? cnt : kq - 1;
      while (p > 0 && best[p - 1] >= D) {
#else
      if (cnt == kq && !(D < best[kq - 1])) continue;
      int p = (cnt < kq) ? cnt : kq - 1;
      while (p > 0 && best[p - 1] > D) {
#endif
        best[p] = best[p - 1];
        bidx[p] = bidx[p - 1];
        --p;
      }
      best[p] = D;
      bidx[p] = (int32_t)j;
      if (cnt < kq) ++cnt;
    }
    for (int a = 0; a < kq; ++a) {
      idx_out[q * kq + a] = bidx[a];
      if (key_out) key_out[q * kq + a] = best[a];
    }
    free(best);
    free(bidx);
  }
  return 0;
}

/* Kernel block over an index set, exported for the SPD / symmetry pins. */
int fmgp_oracle_assemble(const double* X, int d, const int32_t* S, int k,
                         const fmgp_oracle_kernel* kp, double* K) {
  if (!kernel_ok(kp) || k < 1) return 1;
  assemble_f64(X, d, S, k, kp, K);
  return 0;
}

/* Correlation phi at squared distances D[0..cnt), exported for the closed-form pins. */
int fmgp_oracle_phi(const fmgp_oracle_kernel* kp, const double* D, int64_t cnt, double* out) {
  if (!kernel_ok(kp)) return 1;
  for (int64_t i = 0; i < cnt; ++i) out[i] = phi_f64(kp, D[i]);
  return 0;
}

static int shape_ok(int64_t n, int d, int r, int ld, int k) {
  return n >= 1 && d >= 1 && r >= 1 && k >= 1 && k <= n && ld >= k - 1;
}

/* Algorithm 2 offline loop (Eq. 6); returns -1 on bad arguments, else the
 * number of blocks whose Cholesky failed. */
static int rows_ok(const int64_t* rows, int64_t nrows, int64_t n) {
  if (!rows) return 1;
  if (nrows < 0) return 0;
  for (int64_t q = 0; q < nrows; ++q)
    if (rows[q] < 0 || rows[q] >= n) return 0;
  return 1;
}

/* rows (nrows entries) selects the training points to process; NULL = all n. */
int64_t fmgp_oracle_precompute(const double* X, const double* Y, int64_t n, int d, int r,
                               const int32_t* nbr, int ld, int k, const fmgp_oracle_kernel* kp,
                               const int64_t* rows, int64_t nrows, double* C, int8_t* status) {
  if (!kernel_ok(kp) || !shape_ok(n, d, r, ld, k) || !rows_ok(rows, nrows, n)) return -1;
  return precompute_f64(X, Y, n, d, r, nbr, ld, k, kp, rows, nrows, C, status);
}

int64_t fmgp_oracle_precompute_ld(const double* X, const double* Y, int64_t n, int d, int r,
                                  const int32_t* nbr, int ld, int k,
                                  const fmgp_oracle_kernel* kp, const int64_t* rows,
                                  int64_t nrows, double* C, int8_t* status) {
  if (!kernel_ok(kp) || !shape_ok(n, d, r, ld, k) || !rows_ok(rows, nrows, n)) return -1;
  const int64_t cnt = rows ? nrows : n;
  long double* Cl = (long double*)malloc(sizeof(long double) * (size_t)(cnt > 0 ? cnt : 1) * k * r);
  int64_t f = precompute_ld(X, Y, n, d, r, nbr, ld, k, kp, rows, nrows, Cl, status);
  for (int64_t i = 0; i < cnt * k * r; ++i) C[i] = (double)Cl[i];
  free(Cl);
  return f;
}

/* Algorithm 2 online loop (Eq. 7): nearest training point by the canonical
 * key (ties to the lowest index), then the k-term cross-covariance dot
 * product with that point's row of C.  nearest_out (m) may be NULL. */
int fmgp_oracle_predict(const double* X, int64_t n, int d, const int32_t* nbr, int ld,
                        const double* C, int k, int r, const fmgp_oracle_kernel* kp,
                        const double* Z, int64_t m, double* Yhat, int32_t* nearest_out) {
  if (!kernel_ok(kp) || !shape_ok(n, d, r, ld, k) || m < 0) return 1;
  if (m == 0) return 0;
  int32_t* nearest = (int32_t*)malloc(sizeof(int32_t) * m);
  int rc = fmgp_oracle_knn(X, n, d, Z, m, 1, NULL, nearest, NULL);
  if (rc == 0) {
    predict_given_f64(X, d, nbr, ld, C, k, r, kp, Z, m, nearest, Yhat);
    if (nearest_out) memcpy(nearest_out, nearest, sizeof(int32_t) * m);
  }
  free(nearest);
  return rc;
}

/* Eq. 7 with j* supplied (for sampled checks at sizes where the brute-force
 * 1-NN scan is too slow); REAL = FP64 or long double. */
int fmgp_oracle_predict_given(const double* X, int d, const int32_t* nbr, int ld,
                              const double* C, int k, int r, const fmgp_oracle_kernel* kp,
                              const double* Z, int64_t m, const int32_t* nearest, double* Yhat) {
  if (!kernel_ok(kp) || d < 1 || k < 1 || r < 1 || m < 0) return 1;
  predict_given_f64(X, d, nbr, ld, C, k, r, kp, Z, m, nearest, Yhat);
  return 0;
}

/* Eq. 6 then Eq. 7 carried out entirely in long double (C never rounded to
 * FP64), for the given j*: the reference against which tests bound the FP64
 * oracle's own rounding error on ill-conditioned blocks. */
int fmgp_oracle_fit_predict_ld(const double* X, const double* Y, int64_t n, int d, int r,
                               const int32_t* nbr, int ld, int k, const fmgp_oracle_kernel* kp,
                               const double* Z, int64_t m, const int32_t* nearest, double* Yhat) {
  if (!kernel_ok(kp) || !shape_ok(n, d, r, ld, k) || m < 0) return 1;
  for (int64_t t = 0; t < m; ++t)
    if (nearest[t] < 0 || nearest[t] >= n) return 1;
  /* only the rows of C that the m predictions read */
  int64_t* rows = (int64_t*)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
  for (int64_t t = 0; t < m; ++t) rows[t] = nearest[t];
  long double* Cc = (long double*)malloc(sizeof(long double) * (size_t)(m > 0 ? m : 1) * k * r);
  long double* Cl = (long double*)calloc((size_t)n * k * r, sizeof(long double));
  long double* Yl = (long double*)malloc(sizeof(long double) * (size_t)(m > 0 ? m : 1) * r);
  precompute_ld(X, Y, n, d, r, nbr, ld, k, kp, rows, m, Cc, NULL);
  for (int64_t t = 0; t < m; ++t)
    memcpy(Cl + (size_t)nearest[t] * k * r, Cc + (size_t)t * k * r,
           sizeof(long double) * (size_t)k * r);
  predict_given_ld(X, d, nbr, ld, Cl, k, r, kp, Z, m, nearest, Yl);
  for (int64_t i = 0; i < m * r; ++i) Yhat[i] = (double)Yl[i];
  free(rows);
  free(Cc);
  free(Cl);
  free(Yl);
  return 0;
}

/* MuyGPs prediction (Eq. 8) with a brute-force kNN of each test point (k
 * nearest training points, ties to the lowest index).  nbr_out (m x k) may
 * be NULL.  Returns -1 on bad arguments, else the number of failed blocks. */
int64_t fmgp_oracle_muygps_predict(const double* X, const double* Y, int64_t n, int d, int r,
                                   const double* Z, int64_t m, int k,
                                   const fmgp_oracle_kernel* kp, double* Yhat, int32_t* nbr_out) {
  if (!kernel_ok(kp) || n < 1 || d < 1 || r < 1 || k < 1 || k > n || m < 0) return -1;
  if (m == 0) return 0;
  int32_t* N = (int32_t*)malloc(sizeof(int32_t) * (size_t)m * k);
  fmgp_oracle_knn(X, n, d, Z, m, k, NULL, N, NULL);
  int64_t f = predict_muygps_f64(X, Y, d, r, N, k, kp, Z, m, Yhat);
  if (nbr_out) memcpy(nbr_out, N, sizeof(int32_t) * (size_t)m * k);
  free(N);
  return f;
}

/* Eq. 5 LOOCV objective; returns -1 on bad arguments, else the number of
 * failed blocks.  resid (b) receives the per-point squared residuals. */
int64_t fmgp_oracle_loocv(const double* X, const double* Y, int64_t n, int d, int r,
                          const int32_t* nbr, int ld, int k, const int64_t* batch, int64_t b,
                          const fmgp_oracle_kernel* kp, double* resid, double* Q) {
  if (!kernel_ok(kp) || n < 2 || d < 1 || r < 1 || k < 1 || k > n - 1 || ld < k || b < 1)
    return -1;
  for (int64_t q = 0; q < b; ++q)
    if (batch[q] < 0 || batch[q] >= n) return -1;
  return loocv_f64(X, Y, n, d, r, nbr, ld, k, batch, b, kp, resid, Q);
}

int64_t fmgp_oracle_loocv_ld(const double* X, const double* Y, int64_t n, int d, int r,
                             const int32_t* nbr, int ld, int k, const int64_t* batch, int64_t b,
                             const fmgp_oracle_kernel* kp, double* resid, double* Q) {
  if (!kernel_ok(kp) || n < 2 || d < 1 || r < 1 || k < 1 || k > n - 1 || ld < k || b < 1)
    return -1;
  long double* rl = (long double*)malloc(sizeof(long double) * b);
  long double Ql = 0;
  int64_t f = loocv_ld(X, Y, n, d, r, nbr, ld, k, batch, b, kp, rl, &Ql);
  for (int64_t q = 0; q < b; ++q) resid[q] = (double)rl[q];
  *Q = (double)Ql;
  free(rl);
  return f;
}

/* Metropolis calibration of one input coordinate against one observation
 * (Sec. 4.2, the borehole inverse problem), with the posterior mean of Eq. 7
 * as the emulator.  The input is z0 with coordinate `dim` replaced by the
 * chain state x; the prior on x is uniform on [lo, hi]; the likelihood of
 * the observation f_obs of response column `col` is Gaussian with standard
 * deviation sigma.  Chain c starts at x0[c]; its step t proposes
 *   x' = x + step * noise[t * chains + c].
 * A proposal outside [lo, hi] has zero prior density and is rejected (its
 * margin is -inf).  Otherwise, with e = f_obs - yhat(x)[col] and e' the same
 * at x',
 *   delta = (e^2 - e'^2) / (2 sigma^2)     (the log likelihood ratio)
 * and the proposal is accepted iff margin = delta + expo[t * chains + c] > 0:
 * the Metropolis test u < exp(delta) written with expo = -log u ~ Exp(1), so
 * that no transcendental function decides a move.  samples[t * chains + c]
 * is the state after step t, accepted[c] the number of accepted moves.
 * Returns -1 on bad arguments, else 0. */
static double mcmc_emulate(const double* X, int64_t n, int d, const int32_t* nbr, int ld,
                           const double* C, int k, int r, const fmgp_oracle_kernel* kp,
                           double* z, double* yh, int col) {
  int32_t near = 0;
  fmgp_oracle_knn(X, n, d, z, 1, 1, NULL, &near, NULL);
  predict_given_f64(X, d, nbr, ld, C, k, r, kp, z, 1, &near, yh);
  return yh[col];
}

int64_t fmgp_oracle_mcmc(const double* X, int64_t n, int d, const int32_t* nbr, int ld,
                         const double* C, int k, int r, const fmgp_oracle_kernel* kp,
                         const double* z0, int dim, double lo, double hi, double f_obs, int col,
                         double sigma, double step, int chains, int64_t steps, const double* x0,
                         const double* noise, const double* expo, double* samples,
                         int64_t* accepted, double* margin) {
  if (!kernel_ok(kp) || !shape_ok(n, d, r, ld, k) || dim < 0 || dim >= d || col < 0 ||
      col >= r || !(lo <= hi) || !(sigma > 0) || chains < 0 || steps < 0)
    return -1;
  for (int c = 0; c < chains; ++c)
    if (!(x0[c] >= lo && x0[c] <= hi)) return -1;
  const double two_s2 = 2.0 * sigma * sigma;
#pragma omp parallel for schedule(dynamic, 1)
  for (int c = 0; c < chains; ++c) {
    double* z = (double*)malloc(sizeof(double) * d);
    double* yh = (double*)malloc(sizeof(double) * r);
    memcpy(z, z0, sizeof(double) * d);
    double x = x0[c];
    z[dim] = x;
    double e = f_obs - mcmc_emulate(X, n, d, nbr, ld, C, k, r, kp, z, yh, col);
    int64_t acc = 0;
    for (int64_t t = 0; t < steps; ++t) {
      const int64_t at = t * chains + c;
      const double xp = x + step * noise[at];
      double mg = -INFINITY;
      if (xp >= lo && xp <= hi) {
        z[dim] = xp;
        const double ep = f_obs - mcmc_emulate(X, n, d, nbr, ld, C, k, r, kp, z, yh, col);
#if defined(ORACLE_MUTANT_MCMC_SIGN)
        const double delta = (ep * ep - e * e) / two_s2;
#elif defined(ORACLE_MUTANT_MCMC_NO_HALF)
        const double delta = (e * e - ep * ep) / (sigma * sigma);
#else
        const double delta = (e * e - ep * ep) / two_s2;
#endif
        mg = delta + expo[at];
        if (mg > 0) {
          x = xp;
          e = ep;
          ++acc;
        }
      }
      samples[at] = x;
      if (margin) margin[at] = mg;
    }
    if (accepted) accepted[c] = acc;
    free(z);
    free(yh);
  }
  return 0;
}

void fmgp_oracle_set_threads(int t) {
#ifdef _OPENMP
  if (t > 0) omp_set_num_threads(t);
#else
  (void)t;
#endif
}

int fmgp_oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
