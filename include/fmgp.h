/*
 * fmgp.h -- C ABI of the GB300-native FastMuyGPs posterior-mean library
 * (libfmgp.so).
 *
 * Method: "Fast Gaussian Process Posterior Mean Prediction via Local Cross
 * Validation and Precomputation" (Dunton, Priest, Muyskens).  Notation:
 * training features X in R^{n x d} with responses Y in R^{n x r} (Sec. 2),
 * neighbourhood size k, test features Z in R^{m x d}, kernel hyperparameters
 * theta = [sigma, rho, nu, tau] of the Matern kernel (Eq. 3).
 *
 * Conventions shared by every entry point
 *  - All array arguments are DEVICE pointers owned by the caller, row-major
 *    and contiguous (e.g. X[i*d + j]); the library never frees or retains
 *    them.  Scalars such as Q_out that are documented as HOST pointers are the
 *    only exception.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *    enqueued asynchronously on it unless the entry point says otherwise.
 *    Internal workspace is taken stream-ordered from the device's default
 *    memory pool (cudaMallocAsync), or from the context bound to the calling
 *    thread (fmgp_context_bind), and returned on the same stream.
 *  - Argument errors are detected on the host before anything is launched:
 *    the call returns FMGP_EINVAL and launches nothing.  fmgp_last_error()
 *    returns a thread-local message describing the most recent failure.
 *  - Neighbour ranking: candidates are ordered by the canonical key
 *    D(a,b) = sum_j (a_j - b_j)^2 evaluated in IEEE FP64, left to right, each
 *    subtraction, product and sum rounded separately (FP32 inputs are widened
 *    to FP64 first), then by the candidate's index.  Results are therefore
 *    unique and deterministic: distance ties go to the lowest index.
 *  - Indices are int32: n must be below 2^31.
 */
#ifndef FMGP_H
#define FMGP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FMGP_OK = 0,
  FMGP_EINVAL = 1,       /* bad argument; nothing launched */
  FMGP_ENOMEM = 2,       /* workspace allocation failed; nothing launched */
  FMGP_ECUDA = 3,        /* a CUDA call failed (message in fmgp_last_error) */
  FMGP_ENOTSPD = 4,      /* at least one kernel block was not positive definite */
  FMGP_ETIMEOUT = 5,     /* a bounded device-side wait gave up */
  FMGP_EUNSUPPORTED = 6, /* valid request outside what this build implements */
  FMGP_EIO = 7           /* a model file could not be read or written, or is damaged */
} fmgp_status;

typedef enum { FMGP_F32 = 0, FMGP_F64 = 1 } fmgp_dtype;

/*
 * FMGP_PREC_FP64: every step in IEEE FP64 (the plain reference form).
 * FMGP_PREC_MIXED: kernel blocks assembled and Cholesky-factored in FP32,
 *   followed by iterative refinement whose residual Y - K C is formed in
 *   double-float (pairs of FP32, about 48 significant bits); blocks whose FP32
 *   factorisation fails or whose refinement does not converge are refactored
 *   in FP64.  Coefficients are stored as double-float pairs and prediction
 *   evaluates the cross-covariance in double-float.
 */
typedef enum { FMGP_PREC_FP64 = 0, FMGP_PREC_MIXED = 1 } fmgp_precision;

/*
 * Stationary isotropic kernel k(x,x') = sigma^2 phi(||x - x'||) (Sec. 2).
 * kind = FMGP_KERNEL_MATERN: Eq. 3 with nu in {0.5, 1.5, 2.5} (closed forms
 *   of the Bessel expression; nu = 0.5 is the exponential kernel).
 * kind = FMGP_KERNEL_RBF: the nu -> infinity limit, phi = exp(-d^2 / (2 rho^2)).
 * The nugget tau^2 is added, times sigma^2, to the diagonal of every training
 * block K(X_S, X_S) only; it never enters a cross-covariance.
 */
enum { FMGP_KERNEL_MATERN = 0, FMGP_KERNEL_RBF = 1 };
typedef struct {
  int32_t kind;
  double nu;            /* Matern smoothness (ignored for RBF) */
  double length_scale;  /* rho > 0 */
  double variance;      /* sigma^2 > 0 */
  double nugget;        /* tau^2 >= 0 */
} fmgp_kernel;

/* Per-neighbourhood status codes written to status_out. */
enum {
  FMGP_BLOCK_OK = 0,
  FMGP_BLOCK_NOT_SPD = 1,   /* Cholesky met a non-positive pivot; row of C is zero */
  FMGP_BLOCK_FP64_RETRY = 2, /* MIXED only: solved by the FP64 fallback */
  FMGP_BLOCK_BAD_INDEX = 3   /* a neighbour index was outside [0, n); row of C is zero */
};

/*
 * fmgp_build_knn -- self k-nearest-neighbour table of the training set: the
 * neighbour queries of Algorithm 2 (the k-1 nearest neighbours of every
 * training point) and of Algorithm 1 (the k nearest neighbours of every batch
 * point).  For every training point i, the kq nearest training points j != i,
 * ascending by (canonical key, j).  Only the index i itself is excluded; a
 * duplicate of x_i stored at another index is a neighbour at distance 0.
 *   X        n x d, FP64 or FP32 per `dtype`.
 *   kq       neighbours per row, 1 <= kq <= min(n-1, 160).  A table with
 *            kq = max(k-1, k_loocv) serves both fmgp_precompute (k-1 columns)
 *            and fmgp_loocv_objective (k columns) through nbr_ld = kq.
 *   nbr_out  n x kq int32 (row-major, leading dimension kq).
 *   dist_out n x kq FP64 canonical keys (squared distances), or NULL.
 *   flags    0 (reserved).
 * Search: a uniform grid over the bounding box for d <= 3; a tiled scan with
 * an FP32 prefilter and an exact FP64 re-rank for 4 <= d <= 15 (and for
 * d >= 16 below 4,096 points or with "tensor_cores" off); otherwise
 * candidates from a BF16 tcgen05 GEMM with FP32 accumulation (the candidate
 * selection fused into its epilogue), an exact re-rank of tc_oversample * kq
 * candidates (2 kq above kq = 64), and a certificate that every candidate
 * left out is farther than the kq-th; queries without one are redone by the
 * exhaustive scan.  The table never depends on the path taken.
 * Returns FMGP_OK, FMGP_EINVAL, FMGP_ENOMEM or FMGP_ECUDA.
 */
int fmgp_build_knn(const void* X, fmgp_dtype dtype, int64_t n, int32_t d, int32_t kq,
                   int32_t* nbr_out, double* dist_out, int32_t flags, void* stream);

/*
 * fmgp_precompute -- the offline loop of Algorithm 2 (Eq. 6).
 * For every training point i: S_i = [i, nbr[i][0..k-2]], the k x k block
 * K_i = K(X_Si, X_Si) (sigma^2 phi off the diagonal, sigma^2 (1 + tau^2) on
 * it), and C_i = K_i^{-1} Y(X_Si).
 *   Y        n x r FP64.
 *   nbr      n x nbr_ld int32 neighbour table (first k-1 columns are used),
 *            normally the output of fmgp_build_knn; entries must lie in [0, n).
 *   k        neighbourhood size |S_i|, 1 <= k <= min(n, 160), nbr_ld >= k-1.
 *            A block's FP64 factor must fit one warp's shared memory (about
 *            k <= 157 at d = 2, less for large d); larger requests return
 *            FMGP_EUNSUPPORTED (the mixed form keeps the FP64 layout for its
 *            fallback, so the same limit applies).
 *   C_out    n x k x r coefficients, C_out[(i*k + a)*r + c] pairs with point
 *            S_i[a].  FMGP_PREC_FP64: double.  FMGP_PREC_MIXED: double-float
 *            pairs (float hi, float lo; value = hi + lo), i.e. n*k*r*2 floats.
 *            Both forms take 8 bytes per coefficient.
 *   status_out n int8 FMGP_BLOCK_* codes, or NULL.
 * Returns FMGP_ENOTSPD (after completing every other row) if any block was
 * not positive definite; the status is read back with a synchronisation of
 * `stream` in that case only when status_out is NULL.  Otherwise FMGP_OK.
 * When status_out is given the call stays asynchronous and always returns
 * FMGP_OK on success; inspect status_out.
 */
int fmgp_precompute(const void* X, fmgp_dtype dtype, const double* Y, int64_t n, int32_t d,
                    int32_t r, const int32_t* nbr, int32_t nbr_ld, int32_t k,
                    const fmgp_kernel* kernel, fmgp_precision precision, void* C_out,
                    int8_t* status_out, void* stream);

/*
 * fmgp_predict -- the online loop of Algorithm 2 (Eq. 7).
 * For every test point z_t: j* = the nearest training point (canonical key,
 * ties to the lowest index), S = S_{j*} = [j*, nbr[j*][0..k-2]] and
 * Yhat[t][c] = sum_a sigma^2 phi(||z_t - x_Sa||) C[j*][a][c].  The stored row
 * C_{j*} is the single row of the nearest training point (the O(k) lookup of
 * Sec. 3).
 *   X, nbr, C, k, kernel, precision must be those given to fmgp_precompute.
 *   Z          m x d test features, same dtype as X; m >= 0 (m = 0 is a no-op).
 *   Yhat_out   m x r FP64.
 *   nearest_out m int32 j* per test point, or NULL.
 * Nearest-point search: the grid for d <= 3, a thread-per-query FP32 scan with
 * FP64 keys for the candidates it cannot separate for 4 <= d <= 15, and the
 * tensor-core search of fmgp_build_knn (kq = 1) for d >= 16; j* is exact on
 * every path.
 * Returns FMGP_OK, FMGP_EINVAL, FMGP_ENOMEM or FMGP_ECUDA.
 */
int fmgp_predict(const void* X, fmgp_dtype dtype, int64_t n, int32_t d, const int32_t* nbr,
                 int32_t nbr_ld, const void* C, int32_t k, int32_t r, const fmgp_kernel* kernel,
                 fmgp_precision precision, const void* Z, int64_t m, double* Yhat_out,
                 int32_t* nearest_out, void* stream);

/*
 * fmgp_loocv_objective -- the MuyGPs leave-one-out objective (Algorithm 1,
 * Eqs. 4-5): for each i in the batch B, N_i = nbr[i][0..k-1] (the k nearest
 * neighbours of x_i excluding i),
 * yhat_i = K(x_i, X_Ni) K(X_Ni, X_Ni)^{-1} Y(X_Ni) and
 * Q = (1/b) sum_{i in B} sum_c (Y[i][c] - yhat_i[c])^2.
 *   batch      b int64 training indices in [0, n) (device).
 *   k          1 <= k <= min(n-1, 160), nbr_ld >= k (same shared-memory limit
 *              as fmgp_precompute).
 *   Q_out      HOST pointer to one double.
 *   resid_out  b FP64 per-point squared residuals (device), or NULL.
 * The per-point residuals are summed in batch order by one deterministic
 * reduction.  This call synchronises `stream` to return Q.  Returns
 * FMGP_ENOTSPD (Q = NaN) if any block failed.
 */
int fmgp_loocv_objective(const void* X, fmgp_dtype dtype, const double* Y, int64_t n,
                         int32_t d, int32_t r, const int32_t* nbr, int32_t nbr_ld, int32_t k,
                         const int64_t* batch, int64_t b, const fmgp_kernel* kernel,
                         fmgp_precision precision, double* Q_out, double* resid_out,
                         void* stream);

/*
 * fmgp_loocv_objective_device -- fmgp_loocv_objective without synchronising:
 * Q is written to the DEVICE double Q_dev on `stream` (NaN if any block was
 * not positive definite), the number of such blocks to the device int
 * fails_dev (or nowhere when it is NULL), so that a whole step including the
 * objective can be captured into a CUDA graph and replayed.  Other arguments,
 * the reduction order and the results as fmgp_loocv_objective.  Returns
 * FMGP_OK, FMGP_EINVAL, FMGP_ENOMEM or FMGP_ECUDA.
 */
int fmgp_loocv_objective_device(const void* X, fmgp_dtype dtype, const double* Y, int64_t n,
                                int32_t d, int32_t r, const int32_t* nbr, int32_t nbr_ld,
                                int32_t k, const int64_t* batch, int64_t b,
                                const fmgp_kernel* kernel, fmgp_precision precision,
                                double* Q_dev, int32_t* fails_dev, double* resid_out,
                                void* stream);

/*
 * fmgp_muygps_predict -- plain MuyGPs prediction (Eq. 8), the method
 * FastMuyGPs accelerates: every test point z_t uses its OWN k nearest
 * training points N*_t (canonical key, ties to the lowest index) and one
 * neighbourhood solve, Yhat[t] = K(z_t, X_N*) K(X_N*, X_N*)^{-1} Y(X_N*)
 * (nugget on the block diagonal only).  O(k^3) per test point instead of
 * FastMuyGPs' O(k).
 *   X n x d, Y n x r (FP64), Z m x d (X's dtype), 1 <= k <= min(n, 160) (same
 *   shared-memory limit as fmgp_precompute).
 *   Yhat_out m x r FP64; nbr_out m x k int32 neighbour table or NULL.
 * A block that is not positive definite yields NaN predictions for its test
 * point.  Asynchronous on `stream`.
 */
int fmgp_muygps_predict(const void* X, fmgp_dtype dtype, const double* Y, int64_t n, int32_t d,
                        int32_t r, const void* Z, int64_t m, int32_t k, const fmgp_kernel* kernel,
                        fmgp_precision precision, double* Yhat_out, int32_t* nbr_out,
                        void* stream);

/*
 * fmgp_precompute_rows -- Eq. 6 for a subset of the training points (the
 * "centres"): the subsampling of the precomputed coefficients that Sec. 5
 * proposes to reduce the O(nk) memory of C.  For p < s, the block of training
 * point i = rows[p] is formed and solved exactly as fmgp_precompute does
 * (S_i = [i, nbr[i][0..k-2]]) and stored as row p of C_out.
 *   rows       s int32 training indices (device; any order, repeats allowed).
 *              An index outside [0, n) gives FMGP_BLOCK_BAD_INDEX and a zero
 *              row (counted like a non-SPD block in the return value).
 *   s          number of centres, 0 <= s < 2^31 (s = 0 is a no-op).
 *   C_out      s x k x r coefficients, element format as fmgp_precompute.
 *   status_out s int8 FMGP_BLOCK_* codes, or NULL.
 * nbr is the full table of fmgp_build_knn (rows index into it).  Other
 * arguments, precision, synchronisation and return values as fmgp_precompute.
 */
int fmgp_precompute_rows(const void* X, fmgp_dtype dtype, const double* Y, int64_t n, int32_t d,
                         int32_t r, const int32_t* nbr, int32_t nbr_ld, int32_t k,
                         const int32_t* rows, int64_t s, const fmgp_kernel* kernel,
                         fmgp_precision precision, void* C_out, int8_t* status_out,
                         void* stream);

/*
 * fmgp_predict_rows -- prediction from fmgp_precompute_rows.  Each test point
 * z_t takes the nearest centre x_{rows[p]} (canonical key; ties to the lower
 * position p) and Eq. 7 with S_{rows[p]} and row p of C:
 *   Yhat[t][c] = sum_a sigma^2 phi(||z_t - x_{S[a]}||) C[p][a][c].
 * With every training point as a centre (rows = 0..n-1) this is fmgp_predict.
 *   rows, s    as given to fmgp_precompute_rows, 1 <= s <= n.
 *   C          s x k x r from fmgp_precompute_rows (same k, kernel, precision).
 *   nearest_out m int32 training index rows[p] of each test point's centre,
 *              or NULL.
 * The rows are checked on the device before anything else runs (the call
 * synchronises `stream` once for that): an index outside [0, n) returns
 * FMGP_EINVAL with nothing written.  Otherwise asynchronous; returns FMGP_OK,
 * FMGP_EINVAL, FMGP_ENOMEM or FMGP_ECUDA.
 */
int fmgp_predict_rows(const void* X, fmgp_dtype dtype, int64_t n, int32_t d, const int32_t* nbr,
                      int32_t nbr_ld, const int32_t* rows, int64_t s, const void* C, int32_t k,
                      int32_t r, const fmgp_kernel* kernel, fmgp_precision precision,
                      const void* Z, int64_t m, double* Yhat_out, int32_t* nearest_out,
                      void* stream);

/* ------------------------------------------------------------------------
 * Resident models and the serving loop (the paper's online phase run as a
 * service: Sec. 1 motivates FastMuyGPs by applications that need many fast
 * successive predictions from a trained model, Sec. 3 gives the O(k) lookup).
 * ---------------------------------------------------------------------- */
typedef struct fmgp_model fmgp_model;

/* How fmgp_model_create holds the caller's X, nbr and C. */
enum { FMGP_MODEL_BORROW = 0, FMGP_MODEL_COPY = 1 };

/*
 * fmgp_model_create -- register a fitted model for repeated prediction.
 * X, nbr and C are as produced by fmgp_build_knn / fmgp_precompute with the
 * same k, kernel and precision.  flags = FMGP_MODEL_BORROW: they are
 * BORROWED and must stay valid and unchanged until fmgp_model_destroy.
 * flags = FMGP_MODEL_COPY: the model copies them into device memory of its
 * own (charged to the bound context, if any, like its other buffers), and the
 * caller may free or reuse them as soon as the call returns.  Any other flags
 * value returns FMGP_EINVAL.  Either way the model builds and OWNS the
 * nearest-point search grid (d <= 3), an FP32 copy of an FP64 X for the
 * nearest-point scan (4 <= d <= 15), the packed training side of the
 * tensor-core search (d >= 16) and, for FMGP_PREC_MIXED, a double-float copy
 * of X.  Synchronises `stream` before returning.  *out receives the handle.
 */
int fmgp_model_create(const void* X, fmgp_dtype dtype, int64_t n, int32_t d, const int32_t* nbr,
                      int32_t nbr_ld, const void* C, int32_t k, int32_t r,
                      const fmgp_kernel* kernel, fmgp_precision precision, int32_t flags,
                      fmgp_model** out, void* stream);

/* fmgp_predict through a model (Eq. 7): same results, no index rebuild.
 * Z (m x d device, the model's dtype), Yhat_out (m x r FP64 device),
 * nearest_out (m int32 device or NULL).  Asynchronous on `stream`. */
int fmgp_model_predict(fmgp_model* model, const void* Z, int64_t m, double* Yhat_out,
                       int32_t* nearest_out, void* stream);

/* Free the model's own buffers (waits for the device to go idle first). */
int fmgp_model_destroy(fmgp_model* model);

/* What a model was fitted with. */
typedef struct {
  int64_t n;
  int32_t d, r, k, nbr_ld;
  int32_t dtype;      /* fmgp_dtype of X */
  int32_t precision;  /* fmgp_precision of C */
  fmgp_kernel kernel;
} fmgp_model_info;
int fmgp_model_get_info(const fmgp_model* model, fmgp_model_info* out);

/*
 * fmgp_model_save / fmgp_model_load -- the fitted model of Algorithm 2 (X,
 * the neighbour table, the precomputed coefficients C of Eq. 6, k, the kernel
 * hyperparameters and the precision form) in a file, so that the online
 * phase (Eq. 7) can run in another process.
 * File: a 128-byte little-endian header (magic "FMGPMODL", version 1, shapes,
 * dtype, precision, kernel, the byte size of each array, a 64-bit FNV-1a
 * checksum over the header and the data), then X (n x d), the neighbour table
 * (n x nbr_ld int32; absent when k = 1) and C (n x k x r, 8 bytes each) as
 * stored on the device.  Arrays pass through a pinned host buffer of at most
 * 64 MB.
 * fmgp_model_save synchronises `stream`.  fmgp_model_load allocates device
 * memory for X, the table and C (owned by the model and freed by
 * fmgp_model_destroy), checks the header and the checksum, builds the model
 * as fmgp_model_create does, and synchronises `stream`.  A loaded model
 * predicts bit-identically to the one that was saved.
 * Returns FMGP_OK, FMGP_EINVAL (NULL arguments), FMGP_EIO (file cannot be
 * opened, read or written; not a model file; unsupported version;
 * inconsistent sizes; checksum mismatch), FMGP_ENOMEM or FMGP_ECUDA.
 */
int fmgp_model_save(const fmgp_model* model, const char* path, void* stream);
int fmgp_model_load(const char* path, fmgp_model** out, void* stream);

/* Device bytes owned by the model (grid and copies of X), -1 for NULL. */
int64_t fmgp_model_device_bytes(const fmgp_model* model);

/*
 * fmgp_model_mcmc -- Metropolis calibration of one model input against one
 * observation, the model's posterior mean (Eq. 7) as the emulator (Sec. 4.2:
 * recovering the borehole radius from an observed flow by MCMC).
 *
 * The emulator input of a chain in state x is z0 (d doubles, HOST) with
 * coordinate `dim` replaced by x.  Prior: uniform on [lo, hi].  Likelihood:
 * Gaussian, standard deviation sigma, of the observation f_obs of response
 * column `col`.  `chains` independent random-walk chains advance together;
 * chain c starts at x0[c] (HOST, chains doubles, each inside [lo, hi]) and its
 * step t (0 <= t < steps) does, in FP64 with every operation rounded as written:
 *   x' = x + step * noise[t * chains + c]
 *   rejected when x' < lo or x' > hi (zero prior density); otherwise
 *   e = f_obs - yhat(x)[col], e' = f_obs - yhat(x')[col],
 *   delta = (e*e - e'*e') / (2 * sigma * sigma),
 *   accepted iff delta + expo[t * chains + c] > 0.
 * With expo = -log u this is the usual test u < exp(delta).  The random draws
 * are inputs: noise (N(0,1)) and expo (Exp(1)) are DEVICE arrays of
 * steps x chains doubles, step-major.
 *
 * Outputs (DEVICE, caller-owned, each may be NULL): samples_out (steps x
 * chains doubles, the state after each step, step-major), accepted_out
 * (chains int64, accepted moves), x_out (chains doubles, final state).
 * Every step emulates all chains at once (nearest training point + gather-
 * dot), so the work per step is that of fmgp_model_predict with m = chains.
 * Errors: FMGP_EINVAL for a NULL model or z0, dim or col out of range,
 * non-finite or inverted bounds, sigma <= 0, non-finite step, f_obs or z0,
 * an x0 outside [lo, hi], missing draws; FMGP_ENOMEM for workspace.
 * Asynchronous on `stream` (x0 and z0 are read before the call returns).
 */
int fmgp_model_mcmc(fmgp_model* model, const double* z0, int32_t dim, double lo, double hi,
                    double f_obs, int32_t col, double sigma, double step, int64_t chains,
                    int64_t steps, const double* x0, const double* noise, const double* expo,
                    double* samples_out, int64_t* accepted_out, double* x_out, void* stream);

typedef struct fmgp_server fmgp_server;

typedef struct {
  int64_t device_budget_bytes;  /* admitted requests' device bytes (inputs + outputs) */
  int64_t host_staging_bytes;   /* pinned staging arena; >= the largest request */
  int32_t streams;              /* batches in flight at once (1..16) */
  int32_t max_batch_points;     /* cap on test points per launched batch; larger
                                   requests are split into pieces of this size */
} fmgp_server_config;

typedef struct {
  int64_t submitted, completed, rejected;
  int64_t batches;              /* launched batches */
  int64_t points;               /* completed test points */
  double mean_batch_requests;   /* request pieces per batch */
} fmgp_server_stats;

/*
 * fmgp_server_create -- a continuous-batching prediction service over
 * `count` resident models (borrowed; they must outlive the server).  A
 * scheduler thread admits queued requests first-come-first-served while
 * their device bytes fit the budget, splits each into pieces of at most
 * max_batch_points test points, launches the pending pieces of a model (up
 * to max_batch_points points) as one batch on the next free stream (so
 * batches of different models, later arrivals and the pieces of a large
 * request overlap on the device, and a small request waits behind at most
 * one piece of a large one), and completes a request from event polling
 * when its last piece has finished.  Staging copies and CUDA calls are made
 * outside the lock that submitters take.  Each prediction depends only on
 * its own test point, so a request's result is bit-identical alone, inside
 * any batch, or split into pieces.
 * The device current at creation is used by the scheduler thread.
 */
int fmgp_server_create(fmgp_model* const* models, int32_t count, const fmgp_server_config* cfg,
                       fmgp_server** out);

/*
 * fmgp_server_submit -- enqueue a prediction request: m test points
 * Z_host (m x d, HOST memory, the model's dtype, copied at admission so it
 * may be reused once the request completes), results written to HOST
 * buffers Yhat_host (m x r FP64) and nearest_host (m int32 or NULL) when
 * the request completes.  Returns FMGP_ENOMEM if the request alone exceeds
 * the device budget or the staging arena; *request_id identifies it.
 */
int fmgp_server_submit(fmgp_server* srv, int32_t model, const void* Z_host, int64_t m,
                       double* Yhat_host, int32_t* nearest_host, uint64_t* request_id);

/* Wait up to timeout_ms (< 0: forever) for a request: FMGP_OK when its
 * results are in the host buffers, FMGP_ETIMEOUT otherwise, or the error
 * the request failed with. */
int fmgp_server_wait(fmgp_server* srv, uint64_t request_id, int32_t timeout_ms);

/* Host-side milliseconds from submission to launch and to completion. */
int fmgp_server_request_times(fmgp_server* srv, uint64_t request_id, double* queue_ms,
                              double* total_ms);

/* Forget a finished request (its id becomes invalid). */
int fmgp_server_release(fmgp_server* srv, uint64_t request_id);

int fmgp_server_get_stats(fmgp_server* srv, fmgp_server_stats* out);

/* Stop accepting work, finish everything in flight, free the server. */
int fmgp_server_destroy(fmgp_server* srv);

/*
 * fmgp_loocv_objective_noalloc -- fmgp_loocv_objective without any device
 * allocation.  The paper has no counterpart: this is a deployment variant.
 * It is meant for callers that cannot allocate device memory while running,
 * such as an application that gives the library a fixed memory budget at
 * start-up, or a plugin whose host framework owns the device allocator and
 * does not let it call cudaMalloc.  Arguments, results and error codes are
 * those of fmgp_loocv_objective, with these differences:
 *  - Scratch (per-point residuals, the objective, a failure counter) lives in
 *    one file-scope device array of about 512 KB that every device loading
 *    the library keeps until the process exits.  Nothing is allocated or
 *    freed, by this library or by any library it calls.
 *  - b may be at most 65536; a larger batch returns FMGP_EINVAL.
 *  - Only FMGP_PREC_FP64 is accepted (FMGP_EUNSUPPORTED otherwise).
 *  - The first call on a device looks up the array's device address with
 *    that device current; make that first call before any stream capture.
 *    It is also the call at which the CUDA driver loads this library's
 *    kernels and the array onto the device (with lazy module loading, the
 *    default), which takes device memory: make it once during start-up, as
 *    a warm-up, or run with CUDA_MODULE_LOADING=EAGER.
 *  - All calls share the one array, which keeps the previous call's contents
 *    (the call clears its failure counter itself).  Calls that overlap on the
 *    GPU, from several streams or threads, race on it: serialise them.
 * When resid_out is non-NULL the residuals are written there instead of the
 * internal array.  Synchronises `stream` to return Q.
 */
int fmgp_loocv_objective_noalloc(const void* X, fmgp_dtype dtype, const double* Y, int64_t n,
                                 int32_t d, int32_t r, const int32_t* nbr, int32_t nbr_ld,
                                 int32_t k, const int64_t* batch, int64_t b,
                                 const fmgp_kernel* kernel, fmgp_precision precision,
                                 double* Q_out, double* resid_out, void* stream);

/*
 * Workspace contexts (the paper has no counterpart: memory management).
 * fmgp_context_create reserves `bytes` (rounded up to a multiple of 2 MiB) of
 * device memory on the current device in a private stream-ordered pool whose
 * size can never exceed that.
 * After fmgp_context_bind(ctx), every entry point called from this thread on
 * that device takes its internal workspace from the context instead of the
 * device's default pool, so the library's device memory use is bounded and
 * allocated up front; a call whose workspace does not fit returns
 * FMGP_ENOMEM with nothing launched that would need it.  The binding is per
 * thread (a server's scheduler thread does not inherit it); bind NULL to
 * return to the default pool.  Buffers a resident model keeps (grid, copies
 * of X) come from the context bound when it is created: destroy such models
 * before the context.
 * fmgp_context_bytes_in_use: bytes the library's buffers currently hold from
 * the context (each allocation counted in whole 256-byte units; -1 for NULL).
 * An allocation that would take it past the context's size fails.  fmgp_context_destroy waits for the device to go idle, unbinds
 * the context from the calling thread and releases its memory.
 */
typedef struct fmgp_context fmgp_context;
int fmgp_context_create(int64_t bytes, fmgp_context** out);
int fmgp_context_bind(fmgp_context* ctx);
int64_t fmgp_context_bytes_in_use(const fmgp_context* ctx);
int fmgp_context_destroy(fmgp_context* ctx);

/*
 * fmgp_peak_probe -- measured throughput of an arithmetic pipe on the current
 * device, the denominator of the roofline fractions of the neighbourhood
 * kernels (the paper has no counterpart: measurement support).
 * pipe 0 = FP32 fused multiply-add, 1 = FP64 fused multiply-add.  Every SM
 * runs 2048 threads of 8 independent FMA chains for about 30 ms per launch;
 * *flops_per_s receives the best of three timed launches after one warm-up
 * (2 flops per FMA), timed with CUDA events on `stream`.  Synchronises
 * `stream`.  Returns FMGP_OK, FMGP_EINVAL or FMGP_ECUDA.
 */
int fmgp_peak_probe(int32_t pipe, double* flops_per_s, void* stream);

/*
 * fmgp_df_eval -- diagnostic: evaluate one of the double-float primitives of
 * the mixed-precision path on the device, for testing them against FP64 (the
 * paper has no counterpart).  Each x[i] (FP64, device) is split into a pair
 * of FP32 numbers (hi = round(x), lo = round(x - hi)), the primitive is applied
 * and y[i] (FP64, device) = hi + lo of the result.
 *   fn 0: exp(-x) for x >= 0 (0 for x >= 88 or NaN); fn 1: sqrt(x) (0 for x <= 0).
 * Asynchronous on `stream`.  Returns FMGP_OK, FMGP_EINVAL or FMGP_ECUDA.
 */
int fmgp_df_eval(int32_t fn, const double* x, int64_t n, double* y, void* stream);

/* Thread-local description of the most recent error on this thread ("" if none). */
const char* fmgp_last_error(void);

/* Library version, e.g. "0.1.0". */
const char* fmgp_version(void);

/*
 * Launch-shape and path controls (results never depend on them) and three
 * checking / testing switches (check_finite, fail_alloc_after, tc_wait_ns):
 *   "grid_target"  mean training points per grid cell of the d <= 3 search (default 12)
 *   "block_warps"  warps per CTA of the neighbourhood kernels, 0 = automatic
 *   "block_panel"  Cholesky panel width of the mixed neighbourhood kernel for
 *                  k <= 64: 4 or 8 columns, 0 = the autotuner's choice or the
 *                  default (8 for k <= 32, 4 above)
 *   "block_persistent" launch form of the neighbourhood kernels: 1 = persistent
 *                  (one wave of the CTAs the SMs hold at once; each warp, or
 *                  CTA, claims its next neighbourhood from a device counter as
 *                  it becomes free), 0 = eight waves of grid-stride CTAs that
 *                  the hardware's block scheduler replaces as they finish,
 *                  -1 = the autotuner's choice, else persistent (default)
 *   "tensor_cores" 1 = tcgen05 candidate search for kNN at d >= 16 (default), 0 = off
 *   "tc_fused_select" 1 = the candidates are selected inside the tcgen05
 *                  distance kernel (default), 0 = distances go through a pass
 *                  buffer in HBM and a separate selection kernel
 *   "tc_fused_r"   candidates each epilogue thread keeps per range in the fused
 *                  selection: 0 = by kq (8 for kq <= 4, 16 for kq <= 16, 32
 *                  above; default), or 8, 16, 32 (used when kq <= 32 and
 *                  R >= kq / 4).  Above kq = 32 the lists keep 32 and the
 *                  candidates are split into at least ceil(kq / 8) ranges.
 *   "count_visits" 1 = the grid kNN (d <= 3) counts candidates examined and FP64
 *                  keys formed (diagnostic counters 3-5), 0 = off (default)
 *   "tc_oversample" candidates kept per requested neighbour for the exact
 *                  re-rank of the tensor-core search (2..4, default 4; at
 *                  least 32; at most 128 per query, or 2 kq where that is
 *                  larger, up to 320)
 *   "check_finite" 1 = every entry point first scans its floating-point
 *                  device inputs (X, Y, Z) on `stream`, synchronises it, and
 *                  returns FMGP_EINVAL naming the array if one holds a NaN or
 *                  an infinity (not while the stream is being captured into a
 *                  CUDA graph); 0 = no scan (default: the entry points stay
 *                  asynchronous; non-finite inputs then give unspecified
 *                  values, never an out-of-bounds access).  Kernel
 *                  hyperparameters are always checked on the host.
 *   "tc_wait_ns"   limit in ns of the waits in the main loop of the tensor-core
 *                  distance kernel (0 = 2 s, default).  A wait that runs out
 *                  makes the kernel stop, wait (up to 2 s) for its own copies
 *                  and matrix operations in flight, release its tensor memory
 *                  and report the abort; every query of that call is then
 *                  answered by the exhaustive exact scan (same table).  For
 *                  tests of that path.
 *   "fail_alloc_after" failure injection for tests: the next N workspace
 *                  allocations succeed and every later one fails as if the
 *                  device were out of memory (FMGP_ENOMEM); -1 = off (default)
 *   "tc_chunk_queries" queries per pass of the fused tensor-core selection
 *                  (rounded down to whole blocks of 128, at least one block;
 *                  0 = as many as keep its per-range lists within ~1 GB,
 *                  default)
 * Process-wide; returns FMGP_EINVAL for an unknown key or a value out of range.
 */
int fmgp_tune_set(const char* key, double value);
double fmgp_tune_get(const char* key);  /* -1 for an unknown key */

/*
 * Autotuner (the paper has no counterpart: launch-shape selection).
 * fmgp_autotune_precompute times the neighbourhood kernel with each feasible
 * warps-per-CTA (and, for the mixed form with k <= 64, each Cholesky panel
 * width, 4 or 8 columns), each both persistent and as eight waves (unless the
 * tuning key "block_persistent" fixes the form), on the first sample_rows
 * rows of this problem and caches the fastest for (precision, k, d, r,
 * dtype); later fmgp_precompute / fmgp_loocv_objective calls with that key
 * use it.  fmgp_autotune_choice reports the cached shape (warps and panel 0,
 * persistent -1 when none is cached: the defaults).  fmgp_autotune_knn times
 * the grid search of fmgp_build_knn at several cell occupancies and caches
 * the fastest for (d, kq) (d <= 3; for larger d it reports 0).  Results of
 * the path never depend on these choices.  Both synchronise `stream`.
 */
int fmgp_autotune_precompute(const void* X, fmgp_dtype dtype, const double* Y, int64_t n,
                             int32_t d, int32_t r, const int32_t* nbr, int32_t nbr_ld, int32_t k,
                             const fmgp_kernel* kernel, fmgp_precision precision,
                             int64_t sample_rows, int32_t* warps_out, void* stream);
int fmgp_autotune_knn(const void* X, fmgp_dtype dtype, int64_t n, int32_t d, int32_t kq,
                      double* grid_target_out, void* stream);
int fmgp_autotune_choice(fmgp_precision precision, int32_t k, int32_t d, int32_t r,
                         fmgp_dtype dtype, int32_t* warps, int32_t* panel, int32_t* persistent);
int fmgp_autotune_reset(void);

/* Diagnostic counters: 0 = kernels enqueued, 1 = tensor-core kNN calls,
 * 2 = queries of the most recent tensor-core kNN call that lacked a
 * certificate and were redone by the exact scan (valid once that call's
 * stream has completed); with the tuning key "count_visits" set, for the most
 * recent grid kNN call (d <= 3): 3 = candidates examined (FP32 lower bound
 * formed), 4 = canonical FP64 keys formed, 5 = queries (valid once that
 * call's stream has completed; -1 when unavailable). */
int64_t fmgp_diag_counter(int32_t which);

/* Number of CUDA kernels this library has enqueued since it was loaded
 * (all threads, all devices); a diagnostic counter for launch accounting. */
uint64_t fmgp_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* FMGP_H */
