/*
 * Precision-generic body of the FastMuyGPs oracle.  TEST INFRASTRUCTURE ONLY:
 * only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg (and
 * bench.py --impl reference) may load this code.  It shares no code with the
 * CUDA path under paper_2205_10879_gb300/.
 *
 * fmgp_oracle.c includes this file twice: once with REAL = double (suffix
 * _f64, the oracle proper) and once with REAL = long double (suffix _ld, used
 * by tests to bound the FP64 oracle's own rounding error on ill-conditioned
 * blocks).  Neighbour selection is not in here: it always ranks on the FP64
 * canonical key (fmgp_oracle.c).
 *
 * Every loop is written in the order the method states it; nothing is
 * blocked, fused or reordered.
 */

/* Squared Euclidean distance in REAL arithmetic, summed over the features
 * left to right.  Sec. 2 (stationary isotropic kernel: k(x,x') = phi(||x-x'||)). */
static REAL FN(sqdist)(const double* a, const double* b, int d) {
  REAL s = 0;
  for (int j = 0; j < d; ++j) {
    REAL t = (REAL)a[j] - (REAL)b[j];
    s = s + t * t;
  }
  return s;
}

/* Correlation phi at squared distance D, phi(0) = 1.
 * Sec. 2, Matern kernel (Eq. 3) with u = d/rho: for half-integer nu the
 * Bessel form 2^(1-nu)/Gamma(nu) (sqrt(2 nu) u)^nu K_nu(sqrt(2 nu) u)
 * reduces to the closed forms below (Abramowitz & Stegun 10.2.15-17):
 *   nu = 1/2 : exp(-u)                                  (the exponential kernel)
 *   nu = 3/2 : (1 + sqrt3 u) exp(-sqrt3 u)
 *   nu = 5/2 : (1 + sqrt5 u + 5u^2/3) exp(-sqrt5 u)
 * RBF: the nu -> infinity limit named in Sec. 2, exp(-u^2 / 2) (same rho). */
static REAL FN(phi)(const fmgp_oracle_kernel* kp, REAL D) {
  REAL rho = (REAL)kp->length_scale;
  if (kp->kind == 1) {
#ifdef ORACLE_MUTANT_RBF_SCALE
    return EXP(-D / (rho * rho));
#endif
    return EXP(-D / (2 * rho * rho));
  }
  REAL u = SQRT(D) / rho;
  if (kp->nu == 0.5) return EXP(-u);
  if (kp->nu == 1.5) {
    REAL s3 = SQRT((REAL)3);
#ifdef ORACLE_MUTANT_MATERN_POLY
    return (1 + u) * EXP(-s3 * u);
#endif
    return (1 + s3 * u) * EXP(-s3 * u);
  }
  /* nu == 2.5 (validated by the caller) */
  REAL s5 = SQRT((REAL)5);
  return (1 + s5 * u + 5 * u * u / 3) * EXP(-s5 * u);
}

/* Kernel matrix over the index set S (k members):
 * K[a][b] = sigma^2 phi(||x_Sa - x_Sb||) for a != b and sigma^2 (1 + tau^2) on
 * the diagonal.  Eq. 3 with the nugget tau^2 on the index diagonal only. */
static void FN(assemble)(const double* X, int d, const int32_t* S, int k,
                         const fmgp_oracle_kernel* kp, REAL* K) {
  REAL s2 = (REAL)kp->variance;
  for (int a = 0; a < k; ++a) {
    for (int b = 0; b < k; ++b) {
      if (a == b) {
#ifdef ORACLE_MUTANT_NUGGET_UNSCALED
        K[a * k + b] = s2 + (REAL)kp->nugget;
        continue;
#endif
        K[a * k + b] = s2 * (1 + (REAL)kp->nugget);
      } else {
        REAL D = FN(sqdist)(X + (int64_t)S[a] * d, X + (int64_t)S[b] * d, d);
        K[a * k + b] = s2 * FN(phi)(kp, D);
      }
    }
  }
}

/* Cholesky factor K = L L^T (textbook Cholesky-Banachiewicz, row by row),
 * L stored in the lower triangle of K.  Returns 1 if a pivot is not positive. */
static int FN(cholesky)(REAL* K, int k) {
  for (int i = 0; i < k; ++i) {
    for (int j = 0; j <= i; ++j) {
      REAL s = K[i * k + j];
      for (int p = 0; p < j; ++p) s = s - K[i * k + p] * K[j * k + p];
      if (i == j) {
        if (!(s > 0)) return 1;
        K[i * k + i] = SQRT(s);
      } else {
        K[i * k + j] = s / K[j * k + j];
      }
    }
  }
  return 0;
}

/* Solve L L^T w = y in place for the r columns of y (k x r, row-major):
 * forward substitution L v = y, then back substitution L^T w = v. */
static void FN(chol_solve)(const REAL* L, int k, REAL* y, int r) {
  for (int c = 0; c < r; ++c) {
    for (int i = 0; i < k; ++i) {
      REAL s = y[i * r + c];
      for (int p = 0; p < i; ++p) s = s - L[i * k + p] * y[p * r + c];
      y[i * r + c] = s / L[i * k + i];
    }
    for (int i = k - 1; i >= 0; --i) {
      REAL s = y[i * r + c];
#ifdef ORACLE_MUTANT_BACKSOLVE_TRANSPOSE
      for (int p = i + 1; p < k; ++p) s = s - L[i * k + p] * y[p * r + c];
#else
      for (int p = i + 1; p < k; ++p) s = s - L[p * k + i] * y[p * r + c];
#endif
      y[i * r + c] = s / L[i * k + i];
    }
  }
}

/* Offline precomputation of Algorithm 2 / Eq. 6: for every training point i
 * (or for the listed rows only, C and status then follow the list order),
 * S_i = [i, N_i] with N_i its k-1 nearest neighbours (nbr row i, ascending),
 * C_i = K(X_Si, X_Si)^{-1} Y(X_Si).  C is n x k x r: C[i][a][c] pairs with
 * training point S_i[a].  A block whose Cholesky fails gets status 1 and a
 * zero row of C.  Returns the number of failed blocks. */
static int64_t FN(precompute)(const double* X, const double* Y, int64_t n, int d, int r,
                              const int32_t* nbr, int ld, int k,
                              const fmgp_oracle_kernel* kp, const int64_t* rows, int64_t nrows,
                              REAL* C, int8_t* status) {
  int64_t failed = 0;
  if (!rows) nrows = n;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : failed)
  for (int64_t q = 0; q < nrows; ++q) {
    const int64_t i = rows ? rows[q] : q;
    int32_t* S = (int32_t*)malloc(sizeof(int32_t) * k);
    REAL* K = (REAL*)malloc(sizeof(REAL) * k * k);
    REAL* w = (REAL*)malloc(sizeof(REAL) * k * r);
#ifdef ORACLE_MUTANT_SELF_LAST
    for (int a = 0; a < k - 1; ++a) S[a] = nbr[i * ld + a];
    S[k - 1] = (int32_t)i;
#else
    S[0] = (int32_t)i;
    for (int a = 1; a < k; ++a) S[a] = nbr[i * ld + (a - 1)];
#endif
    FN(assemble)(X, d, S, k, kp, K);
    int bad = FN(cholesky)(K, k);
    for (int a = 0; a < k; ++a)
      for (int c = 0; c < r; ++c) w[a * r + c] = (REAL)Y[(int64_t)S[a] * r + c];
    if (!bad) FN(chol_solve)(K, k, w, r);
    for (int a = 0; a < k; ++a)
      for (int c = 0; c < r; ++c) C[(q * k + a) * r + c] = bad ? 0 : w[a * r + c];
    if (status) status[q] = (int8_t)bad;
    failed += bad;
    free(S); free(K); free(w);
  }
  return failed;
}

/* Online prediction of Algorithm 2 / Eq. 7 for the test points whose nearest
 * training point j*(t) is given: with S = S_{j*},
 * yhat[t][c] = sum_a sigma^2 phi(||z_t - x_Sa||) C[j*][a][c], summed over a in
 * order.  The cross-covariance carries no nugget. */
static void FN(predict_given)(const double* X, int d, const int32_t* nbr, int ld,
                              const REAL* C, int k, int r, const fmgp_oracle_kernel* kp,
                              const double* Z, int64_t m, const int32_t* nearest, REAL* Yhat) {
#pragma omp parallel for schedule(static)
  for (int64_t t = 0; t < m; ++t) {
    int64_t j = nearest[t];
    const double* z = Z + t * d;
    for (int c = 0; c < r; ++c) Yhat[t * r + c] = 0;
    for (int a = 0; a < k; ++a) {
      int64_t s = (a == 0) ? j : nbr[j * ld + (a - 1)];
      REAL kz = (REAL)kp->variance * FN(phi)(kp, FN(sqdist)(z, X + s * d, d));
#ifdef ORACLE_MUTANT_CROSS_NUGGET
      if (FN(sqdist)(z, X + s * d, d) == 0) kz = kz + (REAL)kp->variance * (REAL)kp->nugget;
#endif
      for (int c = 0; c < r; ++c) Yhat[t * r + c] = Yhat[t * r + c] + kz * C[(j * k + a) * r + c];
    }
  }
}

/* LOOCV objective of Algorithm 1 / Eq. 5: for each i in the batch B, N_i =
 * the k nearest neighbours of x_i excluding i (nbr row i, first k columns),
 * yhat_i = K(x_i, X_Ni) K(X_Ni, X_Ni)^{-1} Y(X_Ni) (Eq. 4) and
 * Q = (1/b) sum_i sum_c (Y[i][c] - yhat_i[c])^2.  For r > 1 the squared
 * residuals of the r responses are summed per point and divided by b.
 * Per-point residuals go to resid (b entries) and are summed in batch order.
 * Returns the number of blocks whose Cholesky failed (their residual is NaN). */
static int64_t FN(loocv)(const double* X, const double* Y, int64_t n, int d, int r,
                         const int32_t* nbr, int ld, int k, const int64_t* batch, int64_t b,
                         const fmgp_oracle_kernel* kp, REAL* resid, REAL* Q) {
  int64_t failed = 0;
  (void)n;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : failed)
  for (int64_t q = 0; q < b; ++q) {
    int64_t i = batch[q];
    const int32_t* N = nbr + i * ld;
    REAL* K = (REAL*)malloc(sizeof(REAL) * k * k);
    REAL* w = (REAL*)malloc(sizeof(REAL) * k * r);
    FN(assemble)(X, d, N, k, kp, K);
    int bad = FN(cholesky)(K, k);
    if (bad) {
      resid[q] = NAN;
      failed += 1;
    } else {
      for (int a = 0; a < k; ++a)
        for (int c = 0; c < r; ++c) w[a * r + c] = (REAL)Y[(int64_t)N[a] * r + c];
      FN(chol_solve)(K, k, w, r);
      REAL* kx = (REAL*)malloc(sizeof(REAL) * k);
      for (int a = 0; a < k; ++a)
        kx[a] = (REAL)kp->variance *
                FN(phi)(kp, FN(sqdist)(X + i * d, X + (int64_t)N[a] * d, d));
      REAL e2 = 0;
      for (int c = 0; c < r; ++c) {
        REAL yh = 0;
        for (int a = 0; a < k; ++a) yh = yh + kx[a] * w[a * r + c];
#ifdef ORACLE_MUTANT_LOO_SIGN
        REAL e = (REAL)Y[i * r + c] + yh;
#else
        REAL e = (REAL)Y[i * r + c] - yh;
#endif
        e2 = e2 + e * e;
      }
      resid[q] = e2;
      free(kx);
    }
    free(K); free(w);
  }
  REAL s = 0;
  for (int64_t q = 0; q < b; ++q) s = s + resid[q];
  *Q = s / (REAL)b;
  return failed;
}

/* MuyGPs prediction (Eq. 8): each test point z_t is predicted from its OWN k
 * nearest training points N*_t (rows of Nz, ascending by key):
 * yhat_t = K(z_t, X_N*) K(X_N*, X_N*)^{-1} Y(X_N*), one Cholesky per test
 * point.  Returns the number of blocks whose Cholesky failed (their yhat is NaN). */
static int64_t FN(predict_muygps)(const double* X, const double* Y, int d, int r,
                                  const int32_t* Nz, int k, const fmgp_oracle_kernel* kp,
                                  const double* Z, int64_t m, REAL* Yhat) {
  int64_t failed = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : failed)
  for (int64_t t = 0; t < m; ++t) {
    const int32_t* N = Nz + t * k;
    REAL* K = (REAL*)malloc(sizeof(REAL) * k * k);
    REAL* w = (REAL*)malloc(sizeof(REAL) * k * r);
    FN(assemble)(X, d, N, k, kp, K);
    if (FN(cholesky)(K, k)) {
      for (int c = 0; c < r; ++c) Yhat[t * r + c] = NAN;
      failed += 1;
    } else {
      for (int a = 0; a < k; ++a)
        for (int c = 0; c < r; ++c) w[a * r + c] = (REAL)Y[(int64_t)N[a] * r + c];
      FN(chol_solve)(K, k, w, r);
      for (int c = 0; c < r; ++c) Yhat[t * r + c] = 0;
      for (int a = 0; a < k; ++a) {
        REAL kz = (REAL)kp->variance * FN(phi)(kp, FN(sqdist)(Z + t * d, X + (int64_t)N[a] * d, d));
        for (int c = 0; c < r; ++c) Yhat[t * r + c] = Yhat[t * r + c] + kz * w[a * r + c];
      }
    }
    free(K);
    free(w);
  }
  return failed;
}
