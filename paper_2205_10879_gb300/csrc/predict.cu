// A4 (nearest training point of each test point) and A5 (gather + k-term
// cross-covariance dot product with the stored row of C), Eq. 7.
#include "knn.cuh"
#include "predict.cuh"
#include "topk.cuh"

namespace fmgp {
namespace {

// A4 on the grid: one warp per test point; lanes scan candidates, the warp
// keeps the best (key, index) and refreshes its FP32 upper bound after every
// segment of cells.
template <int D, typename T>
__global__ void __launch_bounds__(256) nn1_grid_kernel(GridView gv, const T* Z, int64_t m,
                                                       int32_t* nearest) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= m) return;
  const GridGeom g = *gv.geom;
  double q64[D];
  float qf[D];
#pragma unroll
  for (int j = 0; j < D; ++j) {
    q64[j] = (double)Z[w * D + j];
    qf[j] = (float)Z[w * D + j];
  }
  const float qs = query_slack<D>(qf);
  const float margin = g.margin + qs;
  const float cerr = g.conv_err > 0.f ? g.conv_err + qs : 0.f;
  int cq[3] = {0, 0, 0};
  cell_of<D>(g, qf, cq);
  unsigned long long bk = ~0ull, tk = ~0ull;
  int bi = INT_MAX, ti = INT_MAX;
  float t_up = __int_as_float(0x7f800000);
  for (int r = 0;; ++r) {
    for_ring_segments<D>(r, cq, g.G, [&](int c0a, int c0b, int c1, int c2) {
      if (tk != ~0ull && box_lower<D>(g, qf, margin, c0a, c0b, c1, c2) > t_up) return;
      const int s0 = gv.cell_start[cell_linear(c0a, c1, c2, g.G, D)];
      const int e0 = gv.cell_start[cell_linear(c0b, c1, c2, g.G, D) + 1];
      for (int base = s0; base < e0; base += 32) {
        const int j = base + lane;
        if (j < e0) {
          float xf[D];
#pragma unroll
          for (int t = 0; t < D; ++t) xf[t] = gv.xs32[(int64_t)j * D + t];
          if (dist_lower_f32<D>(qf, xf, cerr) <= t_up) {
            const unsigned long long ck = dbits(canon_key<double>(q64, gv.xs64 + (int64_t)j * D, D));
            const int ci = gv.ids[j];
            if (key_less(ck, ci, bk, bi)) { bk = ck; bi = ci; }
          }
        }
      }
      unsigned long long rk = bk;
      int ri = bi;
      warp_argmin(rk, ri);
      tk = rk;
      ti = ri;
      t_up = key_bits_to_float_up(tk);
    });
    if (tk != ~0ull && outside_lower<D>(g, qf, margin, cq, r) > t_up) break;
    if (r >= g.G) break;
  }
  if (lane == 0) nearest[w] = ti;
}

// A5 in FP64: one warp per test point, lane a evaluates sigma^2 phi between
// z_t and x_{S[a]} (S = S_{j*}); the products with C[j*][a][c] are summed by
// a fixed xor-butterfly, so every result depends only on its own inputs.
template <typename T>
__global__ void __launch_bounds__(256) gather_dot_f64_kernel(
    const T* X, int64_t n, int d, const int32_t* nbr, int ld, const double* C, int k, int r,
    KParams kp, const T* Z, int64_t m, const int32_t* nearest, double* Yhat,
    const int32_t* crow) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= m) return;
  const int64_t j = nearest[w];
  const int64_t cj = crow ? (int64_t)crow[w] : j;  // row of C (a position for centre subsets)
  if (j < 0 || j >= n) {  // no valid nearest point (cannot happen for n >= 1)
    if (lane == 0)
      for (int c = 0; c < r; ++c) Yhat[w * r + c] = __longlong_as_double(0x7ff8000000000000ll);
    return;
  }
  const T* z = Z + w * d;
  double kz[kMaxK / 32];
  int nslots = (k + 31) / 32;
#pragma unroll
  for (int s = 0; s < kMaxK / 32; ++s) {
    kz[s] = 0.0;
    const int a = lane + 32 * s;
    if (s < nslots && a < k) {
      int64_t idx = (a == 0) ? j : (int64_t)nbr[j * ld + a - 1];
      if (idx < 0 || idx >= n) idx = j;  // table validated by fmgp_precompute
      const T* x = X + idx * d;
      double D = 0.0;
      for (int t = 0; t < d; ++t) {
        double diff = (double)z[t] - (double)x[t];
        D = fma(diff, diff, D);
      }
      kz[s] = kp.var * phi64(kp, D);
    }
  }
  for (int c = 0; c < r; ++c) {
    double acc = 0.0;
#pragma unroll
    for (int s = 0; s < kMaxK / 32; ++s) {
      const int a = lane + 32 * s;
      if (s < nslots && a < k) acc = fma(kz[s], C[(cj * k + a) * r + c], acc);
    }
#pragma unroll
    for (int off = 16; off; off >>= 1) acc += __shfl_xor_sync(kFull, acc, off);
    if (lane == 0) Yhat[w * r + c] = acc;
  }
}

template <int D>
int launch_nn1_grid(const GridView& gv, const void* Z, fmgp_dtype dt, int64_t m, int32_t* near,
                    cudaStream_t s) {
  const int blocks = ceil_div(m * 32, 256);
  if (dt == FMGP_F64) FMGP_LAUNCH(nn1_grid_kernel<D, double><<<blocks, 256, 0, s>>>(gv, (const double*)Z, m, near));
  else FMGP_LAUNCH(nn1_grid_kernel<D, float><<<blocks, 256, 0, s>>>(gv, (const float*)Z, m, near));
  FMGP_CUDA_TRY(cudaGetLastError());
  return FMGP_OK;
}

}  // namespace

int nearest_on_grid(const GridView& gv, const void* Z, fmgp_dtype dtype, int64_t m,
                    int32_t* nearest, cudaStream_t stream) {
  if (m == 0) return FMGP_OK;
  if (gv.D == 1) return launch_nn1_grid<1>(gv, Z, dtype, m, nearest, stream);
  if (gv.D == 2) return launch_nn1_grid<2>(gv, Z, dtype, m, nearest, stream);
  return launch_nn1_grid<3>(gv, Z, dtype, m, nearest, stream);
}

int nearest_train(const void* X, fmgp_dtype dtype, int64_t n, int d, const void* Z, int64_t m,
                  int32_t* nearest, const TuneParams& tp, Workspace& ws, cudaStream_t stream) {
  if (m == 0) return FMGP_OK;
  if (d <= kGridMaxD) {
    GridView gv;
    int rc = build_grid(X, dtype, n, d, tp.grid_target, ws, stream, &gv);
    if (rc) return rc;
    if (d == 1) return launch_nn1_grid<1>(gv, Z, dtype, m, nearest, stream);
    if (d == 2) return launch_nn1_grid<2>(gv, Z, dtype, m, nearest, stream);
    return launch_nn1_grid<3>(gv, Z, dtype, m, nearest, stream);
  }
  if (d <= kNn1ScanMaxD) return nearest_scan(X, dtype, n, d, Z, m, nullptr, nearest, ws, stream);
  return knn_query_brute(X, dtype, n, d, Z, m, 1, nearest, nullptr, ws, stream);
}

int gather_dot(const void* X, fmgp_dtype dtype, int64_t n, int d, const int32_t* nbr, int ld,
               const void* C, int k, int r, const KParams& kp, const fmgp_kernel& kern,
               fmgp_precision prec, const void* Z, int64_t m, const int32_t* nearest,
               double* Yhat, Workspace& ws, cudaStream_t stream, const int32_t* crow) {
  if (m == 0) return FMGP_OK;
  const int blocks = ceil_div(m * 32, 256);
  if (prec == FMGP_PREC_FP64) {
    if (dtype == FMGP_F64)
      FMGP_LAUNCH(gather_dot_f64_kernel<double><<<blocks, 256, 0, stream>>>(
          (const double*)X, n, d, nbr, ld, (const double*)C, k, r, kp, (const double*)Z, m,
          nearest, Yhat, crow));
    else
      FMGP_LAUNCH(gather_dot_f64_kernel<float><<<blocks, 256, 0, stream>>>(
          (const float*)X, n, d, nbr, ld, (const double*)C, k, r, kp, (const float*)Z, m,
          nearest, Yhat, crow));
  } else {
    return gather_dot_mixed(X, dtype, n, d, nbr, ld, C, k, r, kp, kern, Z, m, nearest, Yhat, ws,
                            stream, nullptr, crow);
  }
  FMGP_CUDA_TRY(cudaGetLastError());
  return FMGP_OK;
}

}  // namespace fmgp
