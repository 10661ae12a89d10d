#include <math.h>
#include "grid.cuh"
#include "scan.cuh"

namespace fmgp {
namespace {

// Order-preserving map of doubles onto unsigned 64-bit integers.
__device__ __forceinline__ unsigned long long ord_of(double x) {
  unsigned long long b = (unsigned long long)__double_as_longlong(x);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double of_ord(unsigned long long o) {
  unsigned long long b = (o >> 63) ? (o & 0x7fffffffffffffffull) : ~o;
  return __longlong_as_double((long long)b);
}

// Bounding box and geometry in one pass.  st (zeroed before the launch)
// collects, per dimension j, max(~ord(x_j)) in st[j] (the complement of the
// minimum's ordinal) and max(ord(x_j)) in st[D + j], both by atomicMax from
// zero; st[2D] counts finished CTAs.  Each CTA reduces its points in
// registers and shared memory, and its thread 0 publishes the 2D maxima, then
// (after a fence) counts the CTA as finished; the CTA that finishes last reads
// the box and writes the geometry.  No CTA waits for another.
__device__ void write_geom(const double* lo_in, const double* hi_in, int D, int G, int f64_input,
                           GridGeom* geom) {
  GridGeom g;
  double M = 0.0, span = 0.0;
  for (int j = 0; j < kGridMaxD; ++j) {
    double lo = 0.0, hi = 1.0;
    if (j < D) {
      lo = lo_in[j];
      hi = hi_in[j];
    }
    double w = (hi - lo) / G;
    if (!(w > 0.0)) w = 1.0;
    g.lo64[j] = lo;
    g.inv_w64[j] = 1.0 / w;
    g.lo[j] = (float)lo;
    g.w[j] = (float)w;
    g.inv_w[j] = (float)(1.0 / w);
    M = fmax(M, fmax(fabs(lo), fabs(hi)));
    span = fmax(span, hi - lo);
  }
  const double u = 5.9604644775390625e-08;  // 2^-24
  g.margin = (float)(8.0 * u * (M + span) * 1.001 + 1e-30);
  g.conv_err = f64_input ? (float)(2.5 * u * M) : 0.0f;
  g.G = G;
  *geom = g;
}

constexpr int kBoxThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kBoxThreads) bbox_geom_kernel(const T* X, int64_t n, int D, int G,
                                                                int f64_input, unsigned long long* st,
                                                                GridGeom* geom) {
  __shared__ unsigned long long red[2 * kGridMaxD][kBoxThreads / 32];
  __shared__ bool last;
  // mn[j] = max of ~ord (the minimum's complement), mx[j] = max of ord; the
  // loops run to kGridMaxD so that the arrays stay in registers
  unsigned long long mn[kGridMaxD], mx[kGridMaxD];
#pragma unroll
  for (int j = 0; j < kGridMaxD; ++j) { mn[j] = 0ull; mx[j] = 0ull; }
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int j = 0; j < kGridMaxD; ++j) {
      if (j < D) {
        const unsigned long long o = ord_of((double)X[i * D + j]);
        mn[j] = ~o > mn[j] ? ~o : mn[j];
        mx[j] = o > mx[j] ? o : mx[j];
      }
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < kGridMaxD; ++j) {
#pragma unroll
    for (int off = 16; off; off >>= 1) {
      const unsigned long long a = __shfl_xor_sync(kFull, mn[j], off);
      const unsigned long long b = __shfl_xor_sync(kFull, mx[j], off);
      mn[j] = a > mn[j] ? a : mn[j];
      mx[j] = b > mx[j] ? b : mx[j];
    }
    if (lane == 0) {
      red[j][wid] = mn[j];
      red[kGridMaxD + j][wid] = mx[j];
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int j = 0; j < D; ++j) {
      unsigned long long a = red[j][0], b = red[kGridMaxD + j][0];
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
        a = red[j][w] > a ? red[j][w] : a;
        b = red[kGridMaxD + j][w] > b ? red[kGridMaxD + j][w] : b;
      }
      atomicMax(&st[j], a);
      atomicMax(&st[D + j], b);
    }
    __threadfence();
    last = atomicAdd(&st[2 * D], 1ull) == (unsigned long long)gridDim.x - 1;
    if (last) {
      __threadfence();
      double lo[kGridMaxD], hi[kGridMaxD];
      for (int j = 0; j < D; ++j) {
        lo[j] = of_ord(~atomicOr(&st[j], 0ull));
        hi[j] = of_ord(atomicOr(&st[D + j], 0ull));
      }
      write_geom(lo, hi, D, G, f64_input, geom);
    }
  }
}

// Cell of every point and the per-cell counts.  counts has cells + 1 ints,
// zero at the launch; the last one counts finished CTAs.  With fused_scan,
// the CTA that finishes last (as in bbox_geom_kernel, no waiting) turns the
// counts into the cell start offsets (exclusive prefix sum, cell_start[cells]
// = n) and clears them, so that they serve as the scatter's cursors.
constexpr int kCountThreads = 1024;
constexpr int kFusedScanCells = 8 * 4 * kCountThreads;  // at most 8 chunks for the last CTA

template <typename T>
__global__ void __launch_bounds__(kCountThreads) cell_count_kernel(const T* X, int64_t n, int D,
                                                                   const GridGeom* geom,
                                                                   int* cell_of_pt, int* counts,
                                                                   int cells, int* cell_start,
                                                                   int fused_scan) {
  const GridGeom& g = *geom;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int c[kGridMaxD] = {0, 0, 0};
    for (int j = 0; j < D; ++j) {
      double t = ((double)X[i * D + j] - g.lo64[j]) * g.inv_w64[j];
      int cj = (int)floor(t);
      c[j] = min(max(cj, 0), g.G - 1);
    }
    int cell = D == 1 ? c[0] : (D == 2 ? c[0] + g.G * c[1] : c[0] + g.G * (c[1] + g.G * c[2]));
    cell_of_pt[i] = cell;
    atomicAdd(&counts[cell], 1);
  }
  if (!fused_scan) return;
  __shared__ bool last;
  __shared__ int warp_tot[kCountThreads / 32];
  __shared__ int chunk_tot;
  __syncthreads();  // every count of this CTA is issued
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(&counts[cells], 1) == (int)gridDim.x - 1;
    if (last) __threadfence();
  }
  __syncthreads();
  if (!last) return;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  int carry = 0;
  for (int base0 = 0; base0 < cells; base0 += 4 * (int)blockDim.x) {
    const int base = base0 + 4 * threadIdx.x;
    int v[4], local = 0;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      v[t] = base + t < cells ? __ldcg(&counts[base + t]) : 0;
      local += v[t];
    }
    int incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      const int w = lane < nw ? warp_tot[lane] : 0;
      int wi = w;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, wi, o);
        if (lane >= o) wi += y;
      }
      if (lane < nw) warp_tot[lane] = wi - w;  // exclusive
      if (lane == 31) chunk_tot = wi;
    }
    __syncthreads();
    int run = carry + warp_tot[wid] + incl - local;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      if (base + t < cells) {
        cell_start[base + t] = run;
        counts[base + t] = 0;
      }
      run += v[t];
    }
    carry += chunk_tot;
    __syncthreads();  // warp_tot and chunk_tot are rewritten by the next chunk
  }
  if (threadIdx.x == 0) cell_start[cells] = carry;
}

template <typename T>
__global__ void scatter_kernel(const T* X, int64_t n, int D, const int* cell_of_pt,
                               const int* cell_start, int* cursor, double* xs64, float* xs32,
                               int* ids) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int cell = cell_of_pt[i];
    int pos = cell_start[cell] + atomicAdd(&cursor[cell], 1);
    for (int j = 0; j < D; ++j) {
      T v = X[i * D + j];
      xs64[(int64_t)pos * D + j] = (double)v;
      xs32[(int64_t)pos * D + j] = (float)v;
    }
    ids[pos] = (int)i;
  }
}

template <typename T>
int build_grid_t(const T* X, fmgp_dtype dtype, int64_t n, int D, double target, Workspace& ws,
                 cudaStream_t stream, GridView* out) {
  const int G = grid_cells_per_dim(n, D, target);
  int64_t cells = 1;
  for (int j = 0; j < D; ++j) cells *= G;
  unsigned long long* st = ws.get<unsigned long long>(2 * D + 1);
  GridGeom* geom = ws.get<GridGeom>(1);
  int* cell_of_pt = ws.get<int>(n);
  int* counts = ws.get<int>(cells + 1);
  int* cell_start = ws.get<int>(cells + 1);
  double* xs64 = ws.get<double>(n * D);
  float* xs32 = ws.get<float>(n * D);
  int* ids = ws.get<int>(n);
  if (!st || !geom || !cell_of_pt || !counts || !cell_start || !xs64 || !xs32 || !ids)
    return FMGP_ENOMEM;
  const int sms = num_sms();
  const int blocks = (int)std::min<int64_t>(ceil_div(n, 256), (int64_t)sms * 8);
  FMGP_CUDA_TRY(cudaMemsetAsync(st, 0, sizeof(unsigned long long) * (2 * D + 1), stream));
  FMGP_LAUNCH(bbox_geom_kernel<T><<<blocks, kBoxThreads, 0, stream>>>(
      X, n, D, G, dtype == FMGP_F64 ? 1 : 0, st, geom));
  FMGP_CUDA_TRY(cudaMemsetAsync(counts, 0, sizeof(int) * (cells + 1), stream));
  // up to kFusedScanCells cells the last CTA of the count kernel forms the
  // prefix sum; larger grids use the multi-CTA scan
  const bool fused = cells <= kFusedScanCells;
  const int cblocks = (int)std::min<int64_t>(ceil_div(n, kCountThreads), (int64_t)sms * 2);
  FMGP_LAUNCH(cell_count_kernel<T><<<cblocks, kCountThreads, 0, stream>>>(
      X, n, D, geom, cell_of_pt, counts, (int)cells, cell_start, fused ? 1 : 0));
  if (!fused) {
    int rc = exclusive_scan_int(counts, cell_start, (int)cells, ws, stream);
    if (rc) return rc;
    FMGP_CUDA_TRY(cudaMemsetAsync(counts, 0, sizeof(int) * cells, stream));
  }
  FMGP_LAUNCH(scatter_kernel<T><<<blocks, 256, 0, stream>>>(X, n, D, cell_of_pt, cell_start, counts, xs64,
                                                 xs32, ids));
  FMGP_CUDA_TRY(cudaGetLastError());
  out->geom = geom;
  out->cell_start = cell_start;
  out->xs64 = xs64;
  out->xs32 = xs32;
  out->ids = ids;
  out->n = n;
  out->D = D;
  out->G = G;
  return FMGP_OK;
}

}  // namespace

int grid_cells_per_dim(int64_t n, int D, double target) {
  if (target < 1.0) target = 1.0;
  double g = pow((double)n / target, 1.0 / D);
  int G = (int)floor(g);
  if (G < 1) G = 1;
  // keep G^D within the prefix-sum limit (2^24 cells)
  const int gmax = D == 1 ? (1 << 24) : (D == 2 ? 4096 : 256);
  if (G > gmax) G = gmax;
  return G;
}

int build_grid(const void* X, fmgp_dtype dtype, int64_t n, int D, double target, Workspace& ws,
               cudaStream_t stream, GridView* out) {
  if (D < 1 || D > kGridMaxD) {
    set_error("grid search supports 1 <= d <= %d, got %d", kGridMaxD, D);
    return FMGP_EUNSUPPORTED;
  }
  if (dtype == FMGP_F64)
    return build_grid_t<double>((const double*)X, dtype, n, D, target, ws, stream, out);
  return build_grid_t<float>((const float*)X, dtype, n, D, target, ws, stream, out);
}

}  // namespace fmgp
