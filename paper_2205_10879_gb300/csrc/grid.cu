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

__global__ void bbox_init(unsigned long long* bb, int D) {
  int j = threadIdx.x;
  if (j < D) {
    bb[j] = ~0ull;     // running min
    bb[D + j] = 0ull;  // running max
  }
}

template <typename T>
__global__ void bbox_kernel(const T* X, int64_t n, int D, unsigned long long* bb) {
  unsigned long long mn[kGridMaxD], mx[kGridMaxD];
  for (int j = 0; j < D; ++j) { mn[j] = ~0ull; mx[j] = 0ull; }
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    for (int j = 0; j < D; ++j) {
      unsigned long long o = ord_of((double)X[i * D + j]);
      mn[j] = o < mn[j] ? o : mn[j];
      mx[j] = o > mx[j] ? o : mx[j];
    }
  }
  for (int j = 0; j < D; ++j) {
    for (int off = 16; off; off >>= 1) {
      unsigned long long a = __shfl_xor_sync(kFull, mn[j], off);
      unsigned long long b = __shfl_xor_sync(kFull, mx[j], off);
      mn[j] = a < mn[j] ? a : mn[j];
      mx[j] = b > mx[j] ? b : mx[j];
    }
    if ((threadIdx.x & 31) == 0) {
      atomicMin(&bb[j], mn[j]);
      atomicMax(&bb[D + j], mx[j]);
    }
  }
}

__global__ void geom_kernel(const unsigned long long* bb, int D, int G, int f64_input,
                            GridGeom* geom) {
  GridGeom g;
  double M = 0.0, span = 0.0;
  for (int j = 0; j < kGridMaxD; ++j) {
    double lo = 0.0, hi = 1.0;
    if (j < D) {
      lo = of_ord(bb[j]);
      hi = of_ord(bb[D + j]);
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

template <typename T>
__global__ void cell_count_kernel(const T* X, int64_t n, int D, const GridGeom* geom,
                                  int* cell_of_pt, int* counts) {
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
  unsigned long long* bb = ws.get<unsigned long long>(2 * D);
  GridGeom* geom = ws.get<GridGeom>(1);
  int* cell_of_pt = ws.get<int>(n);
  int* counts = ws.get<int>(cells);
  int* cell_start = ws.get<int>(cells + 1);
  double* xs64 = ws.get<double>(n * D);
  float* xs32 = ws.get<float>(n * D);
  int* ids = ws.get<int>(n);
  if (!bb || !geom || !cell_of_pt || !counts || !cell_start || !xs64 || !xs32 || !ids)
    return FMGP_ENOMEM;
  const int sms = num_sms();
  const int blocks = (int)std::min<int64_t>(ceil_div(n, 256), (int64_t)sms * 8);
  FMGP_LAUNCH(bbox_init<<<1, 32, 0, stream>>>(bb, D));
  FMGP_LAUNCH(bbox_kernel<T><<<blocks, 256, 0, stream>>>(X, n, D, bb));
  FMGP_LAUNCH(geom_kernel<<<1, 1, 0, stream>>>(bb, D, G, dtype == FMGP_F64 ? 1 : 0, geom));
  FMGP_CUDA_TRY(cudaMemsetAsync(counts, 0, sizeof(int) * cells, stream));
  FMGP_LAUNCH(cell_count_kernel<T><<<blocks, 256, 0, stream>>>(X, n, D, geom, cell_of_pt, counts));
  int rc = exclusive_scan_int(counts, cell_start, (int)cells, ws, stream);
  if (rc) return rc;
  FMGP_CUDA_TRY(cudaMemsetAsync(counts, 0, sizeof(int) * cells, stream));
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
