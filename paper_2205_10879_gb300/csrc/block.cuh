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

// What a neighbourhood kernel produces.
enum BlockMode {
  kModePrecompute = 0,  // S_i = [i, N_i] -> row C_i (Eq. 6)
  kModeLoocv = 1,       // N_i of batch points -> squared LOO residual (Eq. 5)
  kModeMuygps = 2       // N*_t of test points -> prediction (Eq. 8)
};

struct BlockArgs {
  const double* Y;
  const int32_t* nbr;
  const int64_t* batch;  // LOOCV only
  void* C;               // precompute only
  int8_t* status;        // precompute only (may be null)
  double* resid;         // LOOCV only
  const void* Zq;        // MuyGPs prediction: test points (m x d, X's dtype)
  const float2* Zdf;     // MuyGPs prediction, mixed: double-float copy of Zq
  double* yhat;          // MuyGPs prediction: m x r
  int* fail_count;       // device counter of failed blocks
  int64_t n, count;      // count = n (precompute) or b (LOOCV)
  int d, r, ld, k;
  KParams kp;
  BlockLayout layout;
  // FP64 fallback of the mixed path: process only the items list[0..*list_count)
  // (item = training point, or batch position for LOOCV) and store C as
  // double-float pairs when c_df is set.
  const int* list = nullptr;
  const int* list_count = nullptr;
  bool c_df = false;
  // Precompute over centres (subsampled precompute): item p factors the block
  // of training point rows[p] and writes C row p and status p.
  const int32_t* rows = nullptr;
  // Persistent launches: a device work counter, zero when the kernel starts.
  // The grid is then one wave of the CTAs the SMs hold at once, and every warp
  // (or CTA) claims its next neighbourhood from the counter; without one the
  // grid is several waves and the items are grid-strided.
  unsigned long long* queue = nullptr;
};

// Work distribution of the block kernels.  A warp (or CTA) starts with item
// `first` = its index in the grid and moves on to item `stride` + claim, where
// claim is the value it took from the counter (one atomic, issued when an item
// starts and read when it ends, so that its latency is hidden by the item's
// work), or its current item when there is no counter (grid stride).  With a
// counter, items are handed out in order as warps become free, so that the
// kernel ends with no wave tail.
__device__ __forceinline__ unsigned long long block_claim(unsigned long long* queue, int64_t item,
                                                          bool leader) {
  if (!queue) return (unsigned long long)item;
  return leader ? atomicAdd(queue, 1ull) : 0ull;
}

// blocks = 0 picks the grid: one wave of resident CTAs when a.queue is set (the
// launcher zeroes the counter first), else eight waves; the list mode needs an
// explicit grid and no queue.
int launch_block_f64(const BlockArgs& a, const void* X, fmgp_dtype dtype, int mode, int warps,
                     cudaStream_t stream, int blocks = 0);

// Mixed-precision form (FP32 factor + double-float refinement + FP64 fallback).
// Shared memory of one neighbourhood in the mixed form (the one-warp layout,
// or the CTA layout the large ones use; xbytes = 4 for FP32 inputs).
size_t mixed_bytes_per_warp(int k, int d, int r, int xbytes);
// panel: Cholesky panel width 4 or 8 (k <= 64 only), 0 = the default for k.
int run_block_mixed(BlockArgs a, const void* X, fmgp_dtype dtype, int mode, int warps, int panel,
                    const fmgp_kernel& kern, Workspace& ws, cudaStream_t s);

}  // namespace fmgp
