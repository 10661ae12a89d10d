#pragma once
#include "common.cuh"
#include "grid.cuh"

namespace fmgp {

// Launch-shape choices the autotuner may change; results never depend on them.
struct TuneParams {
  double grid_target = 12.0;     // mean training points per grid cell
  int block_warps = 0;           // warps per CTA for block kernels (0 = automatic)
  int block_panel = 0;           // Cholesky panel width of the mixed kernel (0 = tuned / default)
  int block_persistent = -1;     // block kernels: 1 = persistent, 0 = 8 waves, -1 = tuned / default
  bool use_tensor_cores = true;  // tcgen05 candidate search for d >= 16
  bool tc_fused_select = true;   // candidate selection inside the tcgen05 epilogue (kq <= 32)
  int tc_oversample = 4;         // re-rank candidates per requested neighbour (2..4)
  int tc_fused_r = 0;            // per-range list length of the fused selection (0 = by kq)
  int64_t tc_chunk_queries = 0;  // queries per chunk of the fused selection (0 = ~1 GB of lists)
  bool check_finite = false;     // entry points scan X, Y, Z for NaN / Inf first (synchronising)
  int64_t tc_wait_ns = 0;        // limit of the tensor-core kernel's main-loop waits (0 = 2 s)
  bool count_visits = false;     // grid kNN counts candidates examined and FP64 keys formed
};

TuneParams& tune_params();

// Autotuner caches (0 / the default when nothing was tuned for the key).
int tuned_block_warps(int prec, int k, int d, int r, int dtype);
int tuned_block_panel(int prec, int k, int d, int r, int dtype);  // 0 = default width
// Whether the block kernels of this key run persistent (one wave of CTAs
// claiming neighbourhoods from a counter) or as eight waves of grid-stride
// CTAs: the tuning key, else the autotuner's choice, else persistent.
bool block_persistent_for(int prec, int k, int d, int r, int dtype);
double grid_target_for(int d, int kq);

// Self kNN table (A1): nbr (n x kq), dist (n x kq canonical keys, or null).
int knn_self(const void* X, fmgp_dtype dtype, int64_t n, int d, int kq, int32_t* nbr,
             double* dist, const TuneParams& tp, Workspace& ws, cudaStream_t stream);

// Exhaustive exact scan for the queries listed in qlist[0..*qcount) (count
// read on the device); self = the queries are rows of X (each excluded from
// its own list).
// Xf: an FP32 copy of X the caller already holds (null: made here for FP64).
int knn_brute_list(const void* X, fmgp_dtype dtype, int64_t n, int d, const void* Q, int64_t m,
                   int kq, bool self, const int* qlist, const int* qcount, int32_t* idx,
                   double* key, Workspace& ws, cudaStream_t stream, const float* Xf = nullptr);

// kq nearest training points of each of m query points (no exclusion):
// grid search for d <= 3, tensor-core or exhaustive search otherwise.
int knn_query(const void* X, fmgp_dtype dtype, int64_t n, int d, const void* Q, int64_t m, int kq,
              int32_t* idx, double* key, const TuneParams& tp, Workspace& ws, cudaStream_t stream);

// Tensor-core candidate search + certified exact re-rank (d >= 16).
bool tc_knn_eligible(int64_t n, int d, int64_t m, int kq);

// Training side of the tensor-core search, packed once for repeated query
// batches (resident models): BF16 rows padded to the tile, squared norms and
// rounding-error norms per row, their maxima, and FP32 rows for the re-rank.
// Buffers belong to the Workspace given to tc_pack_train.
struct TcPacked {
  const void* Xb = nullptr;
  const float* xn2 = nullptr;
  const float* xdl = nullptr;
  const unsigned int* xst = nullptr;
  const float* Xa = nullptr;
};
int tc_pack_train(const void* X, fmgp_dtype dtype, int64_t n, int d, Workspace& ws,
                  cudaStream_t s, TcPacked* out);
// As tc_knn with self = false, with the training side taken from P.
int tc_knn_query_packed(const TcPacked& P, const void* X, fmgp_dtype dtype, int64_t n, int d,
                        const void* Q, int64_t m, int kq, int32_t* idx_out, double* key_out,
                        Workspace& ws, cudaStream_t s);
int tc_knn(const void* X, fmgp_dtype dtype, int64_t n, int d, const void* Q, int64_t m, int kq,
           bool self, int32_t* idx_out, double* key_out, Workspace& ws, cudaStream_t s);

// kq nearest training points of each of m queries by exhaustive scan (d >= 4).
int knn_query_brute(const void* X, fmgp_dtype dtype, int64_t n, int d, const void* Q, int64_t m,
                    int kq, int32_t* idx, double* key, Workspace& ws, cudaStream_t stream);

// atomicMax of max |X[i]| (FP32 bits, i < count) into *mx: the magnitude bound
// whose rounding slack the exhaustive scan's FP32 lower bounds include.
// gate: optional device count; the kernel does nothing while it is 0.
int maxabs_into(const void* X, bool f64, int64_t count, unsigned int* mx, cudaStream_t s,
                const int* gate = nullptr);

// Exhaustive scan with the magnitude bound supplied: *mx must be at least
// max |coordinate| over X and all of Q (FP32 bits, rounded up).
int knn_query_brute_mx(const void* X, fmgp_dtype dtype, int64_t n, int d, const void* Q,
                       int64_t m, int kq, const unsigned int* mx, int32_t* idx, double* key,
                       Workspace& ws, cudaStream_t stream);

// Nearest training point (kq = 1) of each query by a thread-per-query scan,
// for 4 <= d <= kNn1ScanMaxD.  mx: magnitude bound as for knn_query_brute_mx,
// or null to compute it from X and Q.  Xf32: an FP32 copy of an FP64 X
// (round to nearest), or null to make one for the call.
constexpr int kNn1ScanMaxD = 15;
int nearest_scan(const void* X, fmgp_dtype dtype, int64_t n, int d, const void* Q, int64_t m,
                 const unsigned int* mx, int32_t* nearest, Workspace& ws, cudaStream_t stream,
                 const float* Xf32 = nullptr);

// FP32 copy (round to nearest) of count FP64 values.
int to_f32(const double* in, int64_t count, float* out, cudaStream_t s);

}  // namespace fmgp
