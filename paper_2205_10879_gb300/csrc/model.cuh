#pragma once
#include "common.cuh"
#include "grid.cuh"
#include "knn.cuh"

namespace fmgp {



struct Model {
  static constexpr int kMaxBufs = 32;
  const void* X = nullptr;
  fmgp_dtype dtype = FMGP_F64;
  int64_t n = 0;
  int d = 0, ld = 0, k = 0, r = 0;
  const int32_t* nbr = nullptr;
  const void* C = nullptr;
  fmgp_kernel kern{};
  fmgp_precision prec = FMGP_PREC_FP64;
  bool has_grid = false;
  GridView grid{};
  float2* Xdf = nullptr;
  float* Xf32 = nullptr;  // FP32 copy of an FP64 X for the nearest-point scan (4 <= d <= 15)
  bool has_tc = false;    // training side of the tensor-core search packed (d >= 16)
  TcPacked tc{};
  void* bufs[kMaxBufs];
  int nbufs = 0;
  size_t bytes = 0;
  fmgp_context* ctx = nullptr;  // workspace context the buffers were charged to
  int64_t ctx_bytes = 0;
  ~Model();
};

int model_predict(const Model& md, const void* Z, int64_t m, double* Yhat, int32_t* nearest,
                  cudaStream_t s);

// fmgp_model_create with the device buffers owned[0..nowned) handed to the
// model (freed with it, or at once if creation fails); with copy, X, nbr and
// C are first copied into the model's own workspace.
int model_create(const void* X, fmgp_dtype dtype, int64_t n, int32_t d, const int32_t* nbr,
                 int32_t nbr_ld, const void* C, int32_t k, int32_t r, const fmgp_kernel* kernel,
                 fmgp_precision precision, fmgp_model** out, cudaStream_t s, void* const* owned,
                 int nowned, bool copy = false);

}  // namespace fmgp
