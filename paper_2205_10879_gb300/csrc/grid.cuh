// Uniform spatial grid over the training set (d <= 3) and the warp-level
// exact k-nearest-neighbour search that runs on it.
//
// Exactness: every candidate that could enter the result is compared on the
// canonical FP64 key.  FP32 arithmetic is used only to discard candidates and
// cells through LOWER bounds of their distance (with explicit rounding
// margins) compared against an UPPER bound of the current k-th key, so a
// discarded candidate is always strictly farther than the k-th result.
#pragma once
#include "common.cuh"

namespace fmgp {

constexpr int kGridMaxD = 3;

struct GridGeom {
  float lo[kGridMaxD];     // bounding-box corner (FP32)
  float w[kGridMaxD];      // cell width per dimension (FP32)
  float inv_w[kGridMaxD];
  double lo64[kGridMaxD];
  double inv_w64[kGridMaxD];
  float margin;            // absolute slack covering FP32 rounding of coordinates/bounds
  float conv_err;          // 2 u max|x|: error of rounding FP64 coordinates to FP32 (0 for FP32 input)
  int G;                   // cells per dimension
};

// Device view of a built grid.
struct GridView {
  const GridGeom* geom;    // device
  const int* cell_start;   // G^D + 1
  const double* xs64;      // n x D, cell order
  const float* xs32;       // n x D, cell order
  const int* ids;          // n, original index of each sorted point
  int64_t n;
  int D;
  int G;
  // optional device counters (diagnostics): candidates examined, FP64 keys formed
  unsigned long long* visits = nullptr;
};

// Lower bound, in FP32, of the true squared distance between q and x given
// their FP32 copies: per dimension |q - x| >= |fl(qf - xf)| (1 - 2u) - conv_err,
// and the FP32 sum of squares of D <= 3 non-negative terms is scaled by
// (1 - 8u) to absorb its own rounding.
template <int D>
__device__ __forceinline__ float dist_lower_f32(const float* qf, const float* xf, float conv_err) {
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    float t = fabsf(qf[j] - xf[j]) * (1.0f - 2.0f * 5.9604645e-8f) - conv_err;
    t = fmaxf(t, 0.f);
    s = fmaf(t, t, s);
  }
  return s * (1.0f - 16.0f * 5.9604645e-8f);
}

// Per-query slack: the FP32 copy of an FP64 query coordinate is off by at
// most u |q|; returns 2u max_j |q_j| (rounded generously).
template <int D>
__device__ __forceinline__ float query_slack(const float* qf) {
  float m = 0.f;
#pragma unroll
  for (int j = 0; j < D; ++j) m = fmaxf(m, fabsf(qf[j]));
  return 2.5f * 5.9604645e-8f * m;
}

template <int D>
__device__ __forceinline__ void cell_of(const GridGeom& g, const float* qf, int* c) {
#pragma unroll
  for (int j = 0; j < D; ++j) {
    int cj = (int)floorf((qf[j] - g.lo[j]) * g.inv_w[j]);
    c[j] = min(max(cj, 0), g.G - 1);
  }
}

// Lower bound of the squared distance from q to the box of cells
// [c0a..c0b] x {c1} x {c2}.
template <int D>
__device__ __forceinline__ float box_lower(const GridGeom& g, const float* qf, float margin,
                                           int c0a, int c0b, int c1, int c2) {
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    int ca = (j == 0) ? c0a : (j == 1 ? c1 : c2);
    int cb = (j == 0) ? c0b : ca;
    float blo = g.lo[j] + (float)ca * g.w[j];
    float bhi = g.lo[j] + (float)(cb + 1) * g.w[j];
    float gap = fmaxf(fmaxf(blo - qf[j], qf[j] - bhi), 0.f);
    gap = fmaxf(gap - margin, 0.f);
    s = fmaf(gap, gap, s);
  }
  return s * (1.0f - 1e-6f);
}

// Lower bound of the squared distance from q to any cell outside the block
// [cq - r, cq + r]^D; +inf when the block already covers the whole grid.
template <int D>
__device__ __forceinline__ float outside_lower(const GridGeom& g, const float* qf, float margin,
                                               const int* cq, int r) {
  float gap = __int_as_float(0x7f800000);
#pragma unroll
  for (int j = 0; j < D; ++j) {
    if (cq[j] - r > 0) gap = fminf(gap, qf[j] - (g.lo[j] + (float)(cq[j] - r) * g.w[j]));
    if (cq[j] + r < g.G - 1) gap = fminf(gap, (g.lo[j] + (float)(cq[j] + r + 1) * g.w[j]) - qf[j]);
  }
  if (gap == __int_as_float(0x7f800000)) return gap;
  gap = fmaxf(gap - margin, 0.f);
  return gap * gap * (1.0f - 1e-6f);
}

// Visit the cells of ring r (Chebyshev distance exactly r from cq) as
// segments of consecutive cells along dimension 0, which are contiguous in
// the sorted point array.  f(c0a, c0b, c1, c2) is called per segment.
template <int D, typename F>
__device__ __forceinline__ void for_ring_segments(int r, const int* cq, int G, F&& f) {
  if (D == 1) {
    if (r == 0) {
      f(cq[0], cq[0], 0, 0);
    } else {
      if (cq[0] - r >= 0) f(cq[0] - r, cq[0] - r, 0, 0);
      if (cq[0] + r < G) f(cq[0] + r, cq[0] + r, 0, 0);
    }
    return;
  }
  const int a0 = max(cq[0] - r, 0), b0 = min(cq[0] + r, G - 1);
  const int lo2 = (D == 3) ? max(cq[D == 3 ? 2 : 0] - r, 0) : 0;
  const int hi2 = (D == 3) ? min(cq[D == 3 ? 2 : 0] + r, G - 1) : 0;
  const int lo1 = max(cq[1] - r, 0), hi1 = min(cq[1] + r, G - 1);
  for (int c2 = lo2; c2 <= hi2; ++c2) {
    const bool edge2 = (D == 3) && (abs(c2 - cq[D == 3 ? 2 : 0]) == r);
    for (int c1 = lo1; c1 <= hi1; ++c1) {
      if (edge2 || abs(c1 - cq[1]) == r) {
        f(a0, b0, c1, c2);
      } else {
        if (cq[0] - r >= 0) f(cq[0] - r, cq[0] - r, c1, c2);
        if (cq[0] + r < G) f(cq[0] + r, cq[0] + r, c1, c2);
      }
    }
  }
}

__device__ __forceinline__ int cell_linear(int c0, int c1, int c2, int G, int D) {
  return D == 1 ? c0 : (D == 2 ? c0 + G * c1 : c0 + G * (c1 + G * c2));
}

// Host: build the grid for X (n x D, D <= 3) on `stream`, with memory from ws.
// target = mean points per cell.  Returns FMGP_OK or an error code.
int build_grid(const void* X, fmgp_dtype dtype, int64_t n, int D, double target,
               Workspace& ws, cudaStream_t stream, GridView* out);

// Cells per dimension for n points at `target` points per cell.
int grid_cells_per_dim(int64_t n, int D, double target);

}  // namespace fmgp
