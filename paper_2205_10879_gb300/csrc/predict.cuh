#pragma once
#include "common.cuh"
#include "knn.cuh"

namespace fmgp {

// A4 on a prebuilt grid (d <= 3).
int nearest_on_grid(const GridView& gv, const void* Z, fmgp_dtype dtype, int64_t m,
                    int32_t* nearest, cudaStream_t stream);

// A4: j*(t) for each test point (canonical key, ties to the lowest index).
int nearest_train(const void* X, fmgp_dtype dtype, int64_t n, int d, const void* Z, int64_t m,
                  int32_t* nearest, const TuneParams& tp, Workspace& ws, cudaStream_t stream);

// A5: Yhat[t][c] = sum_a sigma^2 phi(||z_t - x_{S_j*[a]}||) C[j*][a][c].
int gather_dot(const void* X, fmgp_dtype dtype, int64_t n, int d, const int32_t* nbr, int ld,
               const void* C, int k, int r, const KParams& kp, const fmgp_kernel& kern,
               fmgp_precision prec, const void* Z, int64_t m, const int32_t* nearest,
               double* Yhat, Workspace& ws, cudaStream_t stream, const int32_t* crow = nullptr);

// A5 with double-float coefficients and cross-covariances (mixed precision).
int gather_dot_mixed(const void* X, fmgp_dtype dtype, int64_t n, int d, const int32_t* nbr, int ld,
                     const void* C, int k, int r, const KParams& kp, const fmgp_kernel& kern,
                     const void* Z, int64_t m, const int32_t* nearest, double* Yhat,
                     Workspace& ws, cudaStream_t stream, const float2* Xdf_cached = nullptr,
                     const int32_t* crow = nullptr);

// Double-float copy of count values (FP64 or FP32 input).
int to_df(const void* in, bool f64, int64_t count, float2* out, cudaStream_t s);

}  // namespace fmgp
