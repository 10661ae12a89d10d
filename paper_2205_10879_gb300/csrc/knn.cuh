#pragma once
#include "common.cuh"
#include "grid.cuh"

namespace fmgp {

// Launch-shape choices the autotuner may change; results never depend on them.
struct TuneParams {
  double grid_target = 12.0;  // mean training points per grid cell
  int block_warps = 0;        // warps per CTA for block kernels (0 = automatic)
};

// Self kNN table (A1): nbr (n x kq), dist (n x kq canonical keys, or null).
int knn_self(const void* X, fmgp_dtype dtype, int64_t n, int d, int kq, int32_t* nbr,
             double* dist, const TuneParams& tp, Workspace& ws, cudaStream_t stream);

// kq nearest training points of each of m queries by exhaustive scan (d >= 4).
int knn_query_brute(const void* X, fmgp_dtype dtype, int64_t n, int d, const void* Q, int64_t m,
                    int kq, int32_t* idx, double* key, Workspace& ws, cudaStream_t stream);

}  // namespace fmgp
