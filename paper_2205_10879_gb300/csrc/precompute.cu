// A2 + A3 (Eq. 6) and A6 (Eqs. 4-5) in FP64: one warp per neighbourhood
// (one CTA per neighbourhood when the neighbourhood's shared memory is too
// large for several to share an SM).  The warp stages the neighbourhood's
// features and responses in shared memory, assembles the lower triangle of
// K_S there, factors it by a row-per-lane Crout Cholesky, solves
// L L^T W = Y_S by column sweeps, and either stores W as the row C_i
// (precompute) or dots it with the cross-covariance of x_i to form the
// leave-one-out residual (LOOCV) or the prediction (MuyGPs).
#include "block.cuh"
#include "knn.cuh"

namespace fmgp {
namespace {

constexpr int kMaxSlots = kMaxK / 32;

__device__ __forceinline__ void pair_of(int p, int& a, int& b) {
  int x = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)p)) * 0.5f);
  while (x * (x - 1) / 2 > p) --x;
  while ((x + 1) * x / 2 <= p) ++x;
  a = x;
  b = p - x * (x - 1) / 2;
}

template <typename T, int MODE>
__global__ void __launch_bounds__(256, 2) block_f64_kernel(BlockArgs args, const T* X) {
  constexpr bool LOO = MODE == kModeLoocv;
  extern __shared__ __align__(16) unsigned char smem[];
  const BlockLayout lay = args.layout;
  const int wpb = blockDim.x >> 5;
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* base = smem + (size_t)wid * lay.bytes_per_warp;
  double* L = (double*)(base + lay.off_L);
  double* W = (double*)(base + lay.off_W);
  double* invd = (double*)(base + lay.off_inv);
  T* XS = (T*)(base + lay.off_X);
  int* S = (int*)(base + lay.off_S);
  volatile int* flag = (int*)(base + lay.off_flag);
  const int k = args.k, d = args.d, r = args.r, ldl = lay.ldl;
  const KParams kp = args.kp;

  const int64_t total = args.list ? (int64_t)*args.list_count : args.count;
  const int64_t stride = (int64_t)gridDim.x * wpb;
  unsigned long long claim = 0;
  for (int64_t it = (int64_t)blockIdx.x * wpb + wid; it < total;
       it = stride + (int64_t)__shfl_sync(kFull, claim, 0)) {
    claim = block_claim(args.queue, it, lane == 0);
    const int64_t item = args.list ? (int64_t)args.list[it] : it;
    int64_t i = LOO ? args.batch[item]
                    : (MODE == kModePrecompute && args.rows ? (int64_t)args.rows[item] : item);
    const int64_t orow = MODE == kModePrecompute && args.rows ? item : i;  // row of C / status
    // S: precompute S_i = [i, N_i]; LOOCV N_i (self excluded); MuyGPs N*_t
    bool bad = false;
    if (MODE != kModeMuygps && (i < 0 || i >= args.n)) { bad = true; i = 0; }
    for (int a = lane; a < k; a += 32) {
      int64_t idx = MODE != kModePrecompute ? (int64_t)args.nbr[i * args.ld + a]
                                            : (a == 0 ? i : (int64_t)args.nbr[i * args.ld + a - 1]);
      if (idx < 0 || idx >= args.n) { bad = true; idx = 0; }
      S[a] = (int)idx;
    }
    bad = __any_sync(kFull, bad);
    __syncwarp();
    for (int e = lane; e < k * d; e += 32) {
      const int a = e / d, t = e - a * d;
      XS[e] = X[(int64_t)S[a] * d + t];
    }
    for (int e = lane; e < k * r; e += 32) {
      const int a = e / r, c = e - a * r;
      W[e] = args.Y[(int64_t)S[a] * r + c];
    }
    __syncwarp();
    // assemble: lower triangle off-diagonal, then the diagonal
    const int npairs = k * (k - 1) / 2;
    for (int p = lane; p < npairs; p += 32) {
      int a, b;
      pair_of(p, a, b);
      double D = 0.0;
      for (int t = 0; t < d; ++t) {
        const double diff = (double)XS[a * d + t] - (double)XS[b * d + t];
        D = fma(diff, diff, D);
      }
      L[a * ldl + b] = kp.var * phi64(kp, D);
    }
    for (int a = lane; a < k; a += 32) L[a * ldl + a] = kp.diag;
    if (lane == 0) *flag = 0;
    __syncwarp();
    // Cholesky, Crout order: step j forms column j of L
    for (int j = 0; j < k; ++j) {
      const double* lj = L + j * ldl;
      // rows lane + 32 s of column j: dot of the finished part of the row
      double dd[kMaxSlots];
#pragma unroll
      for (int s = 0; s < kMaxSlots; ++s) {
        const int row = lane + 32 * s;
        dd[s] = 0.0;
        if (row >= j && row < k) {
          const double* lr = L + row * ldl;
          for (int p = 0; p < j; ++p) dd[s] = fma(lr[p], lj[p], dd[s]);
        }
      }
      if (lane == (j & 31)) {
        const int sj = j >> 5;
        double dj = dd[0];
#pragma unroll
        for (int s = 1; s < kMaxSlots; ++s)
          if (s == sj) dj = dd[s];
        const double v = L[j * ldl + j] - dj;
        if (!(v > 0.0)) {
          *flag = 1;
        } else {
          const double ljj = sqrt(v);
          L[j * ldl + j] = ljj;
          invd[j] = 1.0 / ljj;
        }
      }
      __syncwarp();
      if (*flag) break;
      const double inv = invd[j];
#pragma unroll
      for (int s = 0; s < kMaxSlots; ++s) {
        const int row = lane + 32 * s;
        if (row > j && row < k) L[row * ldl + j] = (L[row * ldl + j] - dd[s]) * inv;
      }
      __syncwarp();
    }
    const bool fail = (*flag != 0) || bad;
    if (!fail) {
      // forward sweep: L v = y
      for (int p = 0; p < k; ++p) {
        if (lane == (p & 31))
          for (int c = 0; c < r; ++c) W[p * r + c] *= invd[p];
        __syncwarp();
#pragma unroll
        for (int s = 0; s < kMaxSlots; ++s) {
          const int row = lane + 32 * s;
          if (row > p && row < k) {
            const double l = L[row * ldl + p];
            for (int c = 0; c < r; ++c) W[row * r + c] = fma(-l, W[p * r + c], W[row * r + c]);
          }
        }
        __syncwarp();
      }
      // back sweep: L^T w = v
      for (int p = k - 1; p >= 0; --p) {
        if (lane == (p & 31))
          for (int c = 0; c < r; ++c) W[p * r + c] *= invd[p];
        __syncwarp();
#pragma unroll
        for (int s = 0; s < kMaxSlots; ++s) {
          const int row = lane + 32 * s;
          if (row < p) {
            const double l = L[p * ldl + row];
            for (int c = 0; c < r; ++c) W[row * r + c] = fma(-l, W[p * r + c], W[row * r + c]);
          }
        }
        __syncwarp();
      }
    }
    if (MODE == kModePrecompute) {
      if (args.c_df) {
        float2* Ci = (float2*)args.C + orow * (int64_t)k * r;
        for (int e = lane; e < k * r; e += 32) {
          const double v = fail ? 0.0 : W[e];
          const float hi = (float)v;
          Ci[e] = make_float2(hi, (float)(v - (double)hi));
        }
      } else {
        double* Ci = (double*)args.C + orow * (int64_t)k * r;
        for (int e = lane; e < k * r; e += 32) Ci[e] = fail ? 0.0 : W[e];
      }
      if (args.status && lane == 0)
        args.status[orow] = bad ? FMGP_BLOCK_BAD_INDEX
                             : (fail ? FMGP_BLOCK_NOT_SPD
                                     : (args.list ? FMGP_BLOCK_FP64_RETRY : FMGP_BLOCK_OK));
      if (fail && lane == 0) atomicAdd(args.fail_count, 1);
    } else {
      // cross-covariance of the query point (x_i for LOOCV, z_t for MuyGPs)
      double kx[kMaxSlots];
      const T* xi = MODE == kModeMuygps ? (const T*)args.Zq + i * d : X + i * d;
#pragma unroll
      for (int s = 0; s < kMaxSlots; ++s) {
        const int a = lane + 32 * s;
        kx[s] = 0.0;
        if (!fail && a < k) {
          double D = 0.0;
          for (int t = 0; t < d; ++t) {
            const double diff = (double)xi[t] - (double)XS[a * d + t];
            D = fma(diff, diff, D);
          }
          kx[s] = kp.var * phi64(kp, D);
        }
      }
      double e2 = 0.0;
      for (int c = 0; c < r; ++c) {
        double acc = 0.0;
#pragma unroll
        for (int s = 0; s < kMaxSlots; ++s) {
          const int a = lane + 32 * s;
          if (a < k) acc = fma(kx[s], W[a * r + c], acc);
        }
#pragma unroll
        for (int off = 16; off; off >>= 1) acc += __shfl_xor_sync(kFull, acc, off);
        if (MODE == kModeMuygps) {
          if (lane == 0)
            args.yhat[i * r + c] = fail ? __longlong_as_double(0x7ff8000000000000ll) : acc;
        } else {
          const double e = args.Y[i * r + c] - acc;
          e2 = fma(e, e, e2);
        }
      }
      if (lane == 0) {
        if (MODE == kModeLoocv) args.resid[item] = fail ? __longlong_as_double(0x7ff8000000000000ll) : e2;
        if (fail) atomicAdd(args.fail_count, 1);
      }
    }
    __syncwarp();
  }
}

// The same computation with one CTA per neighbourhood, for neighbourhoods
// too large for several warps' worth of them to share an SM (an FP64 factor
// of k = 150 needs ~190 KB): one resident warp could only use one of the
// SM's four FP64 units.  kCtaThreads threads split the work (thread t owns
// row t, so k <= kCtaThreads) with a barrier per column; every dot product
// and every update runs in the same order as in block_f64_kernel, so
// coefficients are identical to it.
constexpr int kCtaThreads = 256;
static_assert(kMaxK <= kCtaThreads, "one row per thread");

template <typename T, int MODE>
__global__ void __launch_bounds__(kCtaThreads, 1) block_f64_cta_kernel(BlockArgs args,
                                                                       const T* X) {
  constexpr bool LOO = MODE == kModeLoocv;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[kCtaThreads / 32];
  const BlockLayout lay = args.layout;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  double* L = (double*)(smem + lay.off_L);
  double* W = (double*)(smem + lay.off_W);
  double* invd = (double*)(smem + lay.off_inv);
  T* XS = (T*)(smem + lay.off_X);
  int* S = (int*)(smem + lay.off_S);
  volatile int* flag = (int*)(smem + lay.off_flag);
  const int k = args.k, d = args.d, r = args.r, ldl = lay.ldl;
  const KParams kp = args.kp;

  const int64_t total = args.list ? (int64_t)*args.list_count : args.count;
  __shared__ unsigned long long next_it;
  for (int64_t it = blockIdx.x; it < total; it = (int64_t)next_it) {
    __syncthreads();  // the previous neighbourhood is finished with shared memory and next_it
    unsigned long long claim = 0;
    if (tid == 0) claim = block_claim(args.queue, it, true);
    const int64_t item = args.list ? (int64_t)args.list[it] : it;
    int64_t i = LOO ? args.batch[item]
                    : (MODE == kModePrecompute && args.rows ? (int64_t)args.rows[item] : item);
    const int64_t orow = MODE == kModePrecompute && args.rows ? item : i;  // row of C / status
    bool bad = false;
    if (MODE != kModeMuygps && (i < 0 || i >= args.n)) { bad = true; i = 0; }
    if (tid < k) {
      int64_t idx = MODE != kModePrecompute ? (int64_t)args.nbr[i * args.ld + tid]
                                            : (tid == 0 ? i : (int64_t)args.nbr[i * args.ld + tid - 1]);
      if (idx < 0 || idx >= args.n) { bad = true; idx = 0; }
      S[tid] = (int)idx;
    }
    if (tid == 0) *flag = 0;
    bad = __syncthreads_or(bad) != 0;
    for (int e = tid; e < k * d; e += kCtaThreads) {
      const int a = e / d, t = e - a * d;
      XS[e] = X[(int64_t)S[a] * d + t];
    }
    for (int e = tid; e < k * r; e += kCtaThreads) {
      const int a = e / r, c = e - a * r;
      W[e] = args.Y[(int64_t)S[a] * r + c];
    }
    __syncthreads();
    const int npairs = k * (k - 1) / 2;
    for (int p = tid; p < npairs; p += kCtaThreads) {
      int a, b;
      pair_of(p, a, b);
      double D = 0.0;
      for (int t = 0; t < d; ++t) {
        const double diff = (double)XS[a * d + t] - (double)XS[b * d + t];
        D = fma(diff, diff, D);
      }
      L[a * ldl + b] = kp.var * phi64(kp, D);
    }
    if (tid < k) L[tid * ldl + tid] = kp.diag;
    __syncthreads();
    // Cholesky, Crout order: thread t forms row t of column j
    for (int j = 0; j < k; ++j) {
      double dd = 0.0;
      if (tid >= j && tid < k) {
        const double* lr = L + tid * ldl;
        const double* lj = L + j * ldl;
        for (int p = 0; p < j; ++p) dd = fma(lr[p], lj[p], dd);
      }
      if (tid == j) {
        const double v = L[j * ldl + j] - dd;
        if (!(v > 0.0)) {
          *flag = 1;
        } else {
          const double ljj = sqrt(v);
          L[j * ldl + j] = ljj;
          invd[j] = 1.0 / ljj;
        }
      }
      __syncthreads();
      if (*flag) break;
      if (tid > j && tid < k) L[tid * ldl + j] = (L[tid * ldl + j] - dd) * invd[j];
      __syncthreads();
    }
    const bool fail = (*flag != 0) || bad;
    if (!fail) {
      for (int p = 0; p < k; ++p) {  // forward sweep: L v = y
        for (int c = tid; c < r; c += kCtaThreads) W[p * r + c] *= invd[p];
        __syncthreads();
        if (tid > p && tid < k) {
          const double l = L[tid * ldl + p];
          for (int c = 0; c < r; ++c) W[tid * r + c] = fma(-l, W[p * r + c], W[tid * r + c]);
        }
        __syncthreads();
      }
      for (int p = k - 1; p >= 0; --p) {  // back sweep: L^T w = v
        for (int c = tid; c < r; c += kCtaThreads) W[p * r + c] *= invd[p];
        __syncthreads();
        if (tid < p) {
          const double l = L[p * ldl + tid];
          for (int c = 0; c < r; ++c) W[tid * r + c] = fma(-l, W[p * r + c], W[tid * r + c]);
        }
        __syncthreads();
      }
    }
    if (MODE == kModePrecompute) {
      if (args.c_df) {
        float2* Ci = (float2*)args.C + orow * (int64_t)k * r;
        for (int e = tid; e < k * r; e += kCtaThreads) {
          const double v = fail ? 0.0 : W[e];
          const float hi = (float)v;
          Ci[e] = make_float2(hi, (float)(v - (double)hi));
        }
      } else {
        double* Ci = (double*)args.C + orow * (int64_t)k * r;
        for (int e = tid; e < k * r; e += kCtaThreads) Ci[e] = fail ? 0.0 : W[e];
      }
      if (args.status && tid == 0)
        args.status[orow] = bad ? FMGP_BLOCK_BAD_INDEX
                                : (fail ? FMGP_BLOCK_NOT_SPD
                                        : (args.list ? FMGP_BLOCK_FP64_RETRY : FMGP_BLOCK_OK));
      if (fail && tid == 0) atomicAdd(args.fail_count, 1);
    } else {
      // cross-covariance of the query point (x_i for LOOCV, z_t for MuyGPs)
      double kx = 0.0;
      const T* xi = MODE == kModeMuygps ? (const T*)args.Zq + i * d : X + i * d;
      if (!fail && tid < k) {
        double D = 0.0;
        for (int t = 0; t < d; ++t) {
          const double diff = (double)xi[t] - (double)XS[tid * d + t];
          D = fma(diff, diff, D);
        }
        kx = kp.var * phi64(kp, D);
      }
      double e2 = 0.0;
      for (int c = 0; c < r; ++c) {
        double acc = tid < k ? kx * W[tid * r + c] : 0.0;
#pragma unroll
        for (int off = 16; off; off >>= 1) acc += __shfl_xor_sync(kFull, acc, off);
        if (lane == 0) red[wid] = acc;
        __syncthreads();
        if (tid == 0) {
          double sum = red[0];
          for (int w = 1; w < kCtaThreads / 32; ++w) sum += red[w];
          if (MODE == kModeMuygps) {
            args.yhat[i * r + c] = fail ? __longlong_as_double(0x7ff8000000000000ll) : sum;
          } else {
            const double e = args.Y[i * r + c] - sum;
            e2 = fma(e, e, e2);
          }
        }
        __syncthreads();
      }
      if (tid == 0) {
        if (MODE == kModeLoocv) args.resid[item] = fail ? __longlong_as_double(0x7ff8000000000000ll) : e2;
        if (fail) atomicAdd(args.fail_count, 1);
      }
    }
    if (tid == 0) next_it = (unsigned long long)gridDim.x + claim;
    __syncthreads();
  }
}

}  // namespace

BlockLayout block_layout(int k, int d, int r, int xbytes, bool f32_factor) {
  BlockLayout l;
  const int fb = f32_factor ? 4 : 8;
  l.ldl = (k % 2 == 0) ? k + 1 : k;
  auto up = [](size_t x) { return (x + 15) & ~(size_t)15; };
  size_t off = 0;
  l.off_L = off;    off += up((size_t)k * l.ldl * fb);
  l.off_W = off;    off += up((size_t)k * r * 8);
  l.off_inv = off;  off += up((size_t)k * 8);
  l.off_X = off;    off += up((size_t)k * d * xbytes);
  l.off_S = off;    off += up((size_t)k * 4);
  l.off_flag = off; off += 16;
  l.off_extra = off;
  l.bytes_per_warp = off;
  return l;
}

// Neighbourhoods larger than this (bytes of shared memory) take one CTA each:
// fewer than four of them would fit on an SM as one-warp blocks.
constexpr size_t kCtaBlockBytes = 56 * 1024;

int launch_block_f64(const BlockArgs& a, const void* X, fmgp_dtype dtype, int mode, int warps,
                     cudaStream_t stream, int blocks) {
  // persistent (one wave, claimed items) with a work counter, else eight whole
  // waves of the CTAs the SMs hold at once (grid stride)
  const int waves = a.queue ? 1 : 8;
  if (a.queue) FMGP_CUDA_TRY(cudaMemsetAsync(a.queue, 0, sizeof(unsigned long long), stream));
  if (a.layout.bytes_per_warp > kCtaBlockBytes) {
    const size_t smem = a.layout.bytes_per_warp;
    const void* fk = dtype == FMGP_F64
                         ? (mode == kModeLoocv    ? (const void*)block_f64_cta_kernel<double, kModeLoocv>
                            : mode == kModeMuygps ? (const void*)block_f64_cta_kernel<double, kModeMuygps>
                                                  : (const void*)block_f64_cta_kernel<double, kModePrecompute>)
                         : (mode == kModeLoocv    ? (const void*)block_f64_cta_kernel<float, kModeLoocv>
                            : mode == kModeMuygps ? (const void*)block_f64_cta_kernel<float, kModeMuygps>
                                                  : (const void*)block_f64_cta_kernel<float, kModePrecompute>);
    const int fit = std::max(1, active_ctas(fk, kCtaThreads, smem));
    const int grid = blocks > 0 ? blocks
                                : (int)std::max<int64_t>(1, std::min<int64_t>(a.count, (int64_t)num_sms() * fit * waves));
    if (dtype == FMGP_F64) {
      auto kern = mode == kModeLoocv    ? block_f64_cta_kernel<double, kModeLoocv>
                  : mode == kModeMuygps ? block_f64_cta_kernel<double, kModeMuygps>
                                        : block_f64_cta_kernel<double, kModePrecompute>;
      FMGP_CUDA_TRY(ensure_smem((const void*)kern, smem));
      FMGP_LAUNCH(kern<<<grid, kCtaThreads, smem, stream>>>(a, (const double*)X));
    } else {
      auto kern = mode == kModeLoocv    ? block_f64_cta_kernel<float, kModeLoocv>
                  : mode == kModeMuygps ? block_f64_cta_kernel<float, kModeMuygps>
                                        : block_f64_cta_kernel<float, kModePrecompute>;
      FMGP_CUDA_TRY(ensure_smem((const void*)kern, smem));
      FMGP_LAUNCH(kern<<<grid, kCtaThreads, smem, stream>>>(a, (const float*)X));
    }
    FMGP_CUDA_TRY(cudaGetLastError());
    return FMGP_OK;
  }
  const void* kern;
  if (dtype == FMGP_F64)
    kern = mode == kModeLoocv    ? (const void*)block_f64_kernel<double, kModeLoocv>
           : mode == kModeMuygps ? (const void*)block_f64_kernel<double, kModeMuygps>
                                 : (const void*)block_f64_kernel<double, kModePrecompute>;
  else
    kern = mode == kModeLoocv    ? (const void*)block_f64_kernel<float, kModeLoocv>
           : mode == kModeMuygps ? (const void*)block_f64_kernel<float, kModeMuygps>
                                 : (const void*)block_f64_kernel<float, kModePrecompute>;
  const size_t per_warp = a.layout.bytes_per_warp;
  int nb = 0;
  if (warps <= 0) {  // the CTA size with the most resident warps per SM (ties: larger)
    int best = 0;
    for (int w : {8, 6, 4, 3, 2, 1}) {
      const int c = active_ctas(kern, w * 32, (size_t)w * per_warp);
      if (c * w > best) { best = c * w; warps = w; nb = c; }
    }
    if (!best) {
      set_error("neighbourhood blocks of %zu bytes do not fit an SM", per_warp);
      return FMGP_EUNSUPPORTED;
    }
  } else {
    nb = active_ctas(kern, warps * 32, (size_t)warps * per_warp);
  }
  const size_t smem = per_warp * warps;
  const int64_t need = (a.count + warps - 1) / warps;
  // whole waves of the CTAs the SMs hold at once: no partial last wave
  if (blocks <= 0)
    blocks = (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)num_sms() * std::max(nb, 1) * waves));
  FMGP_CUDA_TRY(ensure_smem(kern, smem));
  if (dtype == FMGP_F64)
    FMGP_LAUNCH(((void (*)(BlockArgs, const double*))kern)<<<blocks, warps * 32, smem, stream>>>(a, (const double*)X));
  else
    FMGP_LAUNCH(((void (*)(BlockArgs, const float*))kern)<<<blocks, warps * 32, smem, stream>>>(a, (const float*)X));
  FMGP_CUDA_TRY(cudaGetLastError());
  return FMGP_OK;
}

}  // namespace fmgp
