// Per-neighbourhood block kernels (assemble + factor + solve): shared layout
// and launch helpers.
#pragma once
#include "common.cuh"

namespace fmgp {

// Byte offsets of one warp's shared-memory region.
struct BlockLayout {
  int ldl;                 // row stride of the factor (odd: conflict-free column access)
  size_t off_L, off_W, off_inv, off_X, off_S, off_flag, off_extra;
  size_t bytes_per_warp;
};

BlockLayout block_layout(int k, int d, int r, int xbytes, bool f32_factor);

struct BlockArgs {
  const double* Y;
  const int32_t* nbr;
  const int64_t* batch;  // LOOCV only
  void* C;               // precompute only
  int8_t* status;        // precompute only (may be null)
  double* resid;         // LOOCV only
  int* fail_count;       // device counter of failed blocks
  int64_t n, count;      // count = n (precompute) or b (LOOCV)
  int d, r, ld, k;
  KParams kp;
  BlockLayout layout;
};

int launch_block_f64(const BlockArgs& a, const void* X, fmgp_dtype dtype, bool loo, int warps,
                     cudaStream_t stream);
int launch_block_mixed(const BlockArgs& a, const void* X, fmgp_dtype dtype, bool loo, int warps,
                       cudaStream_t stream);
size_t block_mixed_extra_bytes(int k, int d, int r);

}  // namespace fmgp
