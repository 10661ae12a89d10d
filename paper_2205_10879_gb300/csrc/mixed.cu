// Mixed-precision form of A2/A3/A6 and A5.
//
// Block kernel (one warp per neighbourhood):
//   1. every kernel entry K_ab = sigma^2 phi(||x_a - x_b||) is evaluated once in
//      double-float (DF, ~48 bits) and kept in shared memory (packed lower
//      triangle); its FP32 rounding fills the matrix that is factored;
//   2. FP32 Cholesky (row-per-lane Crout) and FP32 triangular solves give x0;
//   3. iterative refinement: r = y - K x in DF, delta = (L L^T)^{-1} r in FP32,
//      x += delta in DF.  At least one step is taken; further steps follow while
//      the predicted size of the next correction, |delta_s|^2 / |delta_{s-1}|
//      (relative to |x|), exceeds 1e-6, up to 6 steps;
//   4. blocks whose FP32 factorisation fails, or whose corrections stop
//      contracting, are appended to a list that the FP64 block kernel then
//      solves from scratch (status FMGP_BLOCK_FP64_RETRY).
// Coefficients are stored as DF pairs.  Prediction evaluates the
// cross-covariance and the dot product with C in DF.
#include <math.h>
#include <mutex>
#include "block.cuh"
#include "df.cuh"
#include "predict.cuh"

namespace fmgp {
namespace {

constexpr int kMaxSlots = kMaxK / 32;
constexpr int kMaxRefine = 6;

struct KParamsDF {
  int kind, nu2;
  dfl scale;   // sqrt(2 nu)/rho (Matern) or 1/(2 rho^2) (RBF)
  dfl var;     // sigma^2
  dfl diag;    // sigma^2 (1 + tau^2)
  dfl third;   // 1/3
};

dfl split(double v) {
  const float hi = (float)v;
  const float lo = (float)(v - (double)hi);
  return {hi, lo};
}

KParamsDF make_kparams_df(const KParams& p, const fmgp_kernel& k) {
  KParamsDF q;
  q.kind = p.kind;
  q.nu2 = p.nu2;
  if (p.kind == FMGP_KERNEL_RBF) q.scale = split(0.5 / (k.length_scale * k.length_scale));
  else q.scale = split(sqrt((double)p.nu2) / k.length_scale);
  q.var = split(k.variance);
  q.diag = split(k.variance * (1.0 + k.nugget));
  q.third = split(1.0 / 3.0);
  return q;
}

const DfConsts& df_consts() {
  static DfConsts c;
  static std::once_flag once;
  std::call_once(once, []() {
    const double ln2 = 0.69314718055994530942;
    c.ln2_1 = 0.693145751953125f;  // 14 significant bits
    const double rem = ln2 - (double)c.ln2_1;
    c.ln2_2 = (float)rem;
    c.ln2_3 = (float)(rem - (double)c.ln2_2);
    for (int j = -24; j <= 24; ++j) {
      const double v = exp(-(double)j / 64.0);
      c.e_hi[j + 24] = (float)v;
      c.e_lo[j + 24] = (float)(v - (double)c.e_hi[j + 24]);
    }
  });
  return c;
}

// Correlation sigma^2 phi at DF squared distance D.
__device__ __forceinline__ dfl kernel_df(const KParamsDF& p, dfl D, const DfConsts& K) {
  dfl ph;
  if (p.kind == FMGP_KERNEL_RBF) {
    ph = df_exp_neg(df_mul(D, p.scale), K);
  } else {
    const dfl a = df_mul(df_sqrt(D), p.scale);  // sqrt(2 nu) d / rho
    const dfl e = df_exp_neg(a, K);
    if (p.nu2 == 1) ph = e;
    else if (p.nu2 == 3) ph = df_mul(df_add_f(a, 1.0f), e);
    else ph = df_mul(df_add(df_add_f(a, 1.0f), df_mul(df_sqr(a), p.third)), e);
  }
  return df_mul(p.var, ph);
}

__device__ __forceinline__ dfl sqdist_df(const float2* a, const float2* b, int d) {
  dfl s = {0.0f, 0.0f};
  for (int t = 0; t < d; ++t) {
    const float2 u = a[t], v = b[t];
    const dfl diff = df_add_fast(dfl{u.x, u.y}, dfl{-v.x, -v.y});
    s = df_add_fast(s, df_sqr(diff));
  }
  return s;
}

struct MixedArgs {
  const float2* Xdf;  // n x d
  const float2* Ydf;  // n x r
  int* fb_list;       // items handed to the FP64 fallback
  int* fb_count;
  DfConsts K;
  KParamsDF kdf;
};

struct MixedLayout {
  int ldl;
  size_t off_L, off_K, off_X, off_Y, off_V, off_R, off_inv, off_S, off_flag, bytes;
};

MixedLayout mixed_layout(int k, int d, int r) {
  MixedLayout l;
  l.ldl = (k % 2 == 0) ? k + 1 : k;
  auto up = [](size_t x) { return (x + 15) & ~(size_t)15; };
  size_t o = 0;
  l.off_L = o;    o += up((size_t)k * l.ldl * 4);
  l.off_K = o;    o += up((size_t)k * (k + 1) / 2 * 8);
  l.off_X = o;    o += up((size_t)k * d * 8);
  l.off_Y = o;    o += up((size_t)k * r * 8);
  l.off_V = o;    o += up((size_t)k * r * 8);
  l.off_R = o;    o += up((size_t)k * r * 4);
  l.off_inv = o;  o += up((size_t)k * 4);
  l.off_S = o;    o += up((size_t)k * 4);
  l.off_flag = o; o += 16;
  l.bytes = o;
  return l;
}

__device__ __forceinline__ void pair_of(int p, int& a, int& b) {
  int x = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)p)) * 0.5f);
  while (x * (x - 1) / 2 > p) --x;
  while ((x + 1) * x / 2 <= p) ++x;
  a = x;
  b = p - x * (x - 1) / 2;
}

// FP32 forward and back substitution with L (row stride ldl) on R (k x r).
__device__ __forceinline__ void solve_f32(const float* L, int ldl, const float* invd, float* R,
                                          int k, int r, int lane) {
  for (int p = 0; p < k; ++p) {
    if (lane == (p & 31))
      for (int c = 0; c < r; ++c) R[p * r + c] *= invd[p];
    __syncwarp();
#pragma unroll
    for (int s = 0; s < kMaxSlots; ++s) {
      const int row = lane + 32 * s;
      if (row > p && row < k) {
        const float l = L[row * ldl + p];
        for (int c = 0; c < r; ++c) R[row * r + c] = fmaf(-l, R[p * r + c], R[row * r + c]);
      }
    }
    __syncwarp();
  }
  for (int p = k - 1; p >= 0; --p) {
    if (lane == (p & 31))
      for (int c = 0; c < r; ++c) R[p * r + c] *= invd[p];
    __syncwarp();
#pragma unroll
    for (int s = 0; s < kMaxSlots; ++s) {
      const int row = lane + 32 * s;
      if (row < p) {
        const float l = L[p * ldl + row];
        for (int c = 0; c < r; ++c) R[row * r + c] = fmaf(-l, R[p * r + c], R[row * r + c]);
      }
    }
    __syncwarp();
  }
}

template <bool LOO>
__global__ void __launch_bounds__(256) block_mixed_kernel(BlockArgs args, MixedArgs mx,
                                                          MixedLayout lay) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int wpb = blockDim.x >> 5;
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* base = smem + (size_t)wid * lay.bytes;
  float* L = (float*)(base + lay.off_L);
  dfl* KP = (dfl*)(base + lay.off_K);
  float2* XS = (float2*)(base + lay.off_X);
  dfl* YS = (dfl*)(base + lay.off_Y);
  dfl* XV = (dfl*)(base + lay.off_V);
  float* RV = (float*)(base + lay.off_R);
  float* invd = (float*)(base + lay.off_inv);
  int* S = (int*)(base + lay.off_S);
  volatile int* flag = (int*)(base + lay.off_flag);
  const int k = args.k, d = args.d, r = args.r, ldl = lay.ldl;
  const KParamsDF kp = mx.kdf;

  for (int64_t item = (int64_t)blockIdx.x * wpb + wid; item < args.count;
       item += (int64_t)gridDim.x * wpb) {
    int64_t i = LOO ? args.batch[item] : item;
    bool bad = false;
    if (i < 0 || i >= args.n) { bad = true; i = 0; }
    for (int a = lane; a < k; a += 32) {
      int64_t idx = LOO ? (int64_t)args.nbr[i * args.ld + a]
                        : (a == 0 ? i : (int64_t)args.nbr[i * args.ld + a - 1]);
      if (idx < 0 || idx >= args.n) { bad = true; idx = 0; }
      S[a] = (int)idx;
    }
    bad = __any_sync(kFull, bad);
    __syncwarp();
    for (int e = lane; e < k * d; e += 32) {
      const int a = e / d, t = e - a * d;
      XS[e] = mx.Xdf[(int64_t)S[a] * d + t];
    }
    for (int e = lane; e < k * r; e += 32) {
      const int a = e / r, c = e - a * r;
      const float2 y = mx.Ydf[(int64_t)S[a] * r + c];
      YS[e] = dfl{y.x, y.y};
    }
    __syncwarp();
    // assembly: DF entries (packed lower triangle) and their FP32 roundings
    const int npairs = k * (k - 1) / 2;
    for (int p = lane; p < npairs; p += 32) {
      int a, b;
      pair_of(p, a, b);
      const dfl kab = kernel_df(kp, sqdist_df(XS + a * d, XS + b * d, d), mx.K);
      KP[a * (a + 1) / 2 + b] = kab;
      L[a * ldl + b] = kab.hi;
    }
    for (int a = lane; a < k; a += 32) {
      KP[a * (a + 1) / 2 + a] = kp.diag;
      L[a * ldl + a] = kp.diag.hi;
    }
    if (lane == 0) *flag = 0;
    __syncwarp();
    // FP32 Cholesky (Crout order)
    for (int j = 0; j < k; ++j) {
      float dots[kMaxSlots];
#pragma unroll
      for (int s = 0; s < kMaxSlots; ++s) {
        const int row = lane + 32 * s;
        dots[s] = 0.0f;
        if (row >= j && row < k) {
          float acc = 0.0f;
          const float* lr = L + row * ldl;
          const float* lj = L + j * ldl;
          for (int q = 0; q < j; ++q) acc = fmaf(lr[q], lj[q], acc);
          dots[s] = acc;
        }
      }
      if (lane == (j & 31)) {
        float dj = dots[0];
#pragma unroll
        for (int s = 1; s < kMaxSlots; ++s)
          if (s == (j >> 5)) dj = dots[s];
        const float v = L[j * ldl + j] - dj;
        if (!(v > 0.0f)) {
          *flag = 1;
        } else {
          const float ljj = sqrtf(v);
          L[j * ldl + j] = ljj;
          invd[j] = 1.0f / ljj;
        }
      }
      __syncwarp();
      if (*flag) break;
      const float inv = invd[j];
#pragma unroll
      for (int s = 0; s < kMaxSlots; ++s) {
        const int row = lane + 32 * s;
        if (row > j && row < k) L[row * ldl + j] = (L[row * ldl + j] - dots[s]) * inv;
      }
      __syncwarp();
    }
    bool ok = (*flag == 0) && !bad;
    if (ok) {
      for (int e = lane; e < k * r; e += 32) RV[e] = YS[e].hi;
      __syncwarp();
      solve_f32(L, ldl, invd, RV, k, r, lane);
      for (int e = lane; e < k * r; e += 32) XV[e] = dfl{RV[e], 0.0f};
      __syncwarp();
      float prev = 1.0f;
      bool conv = false;
      for (int step = 1; step <= kMaxRefine; ++step) {
        // residual y - K x in DF; lane owns rows
#pragma unroll
        for (int s = 0; s < kMaxSlots; ++s) {
          const int row = lane + 32 * s;
          if (row < k) {
            for (int c = 0; c < r; ++c) {
              dfl acc = YS[row * r + c];
              for (int b = 0; b < k; ++b) {
                const dfl kab = (b <= row) ? KP[row * (row + 1) / 2 + b] : KP[b * (b + 1) / 2 + row];
                acc = df_add(acc, df_neg(df_mul(kab, XV[b * r + c])));
              }
              RV[row * r + c] = acc.hi;
            }
          }
        }
        __syncwarp();
        solve_f32(L, ldl, invd, RV, k, r, lane);
        float dmax = 0.0f, xmax = 0.0f;
        for (int e = lane; e < k * r; e += 32) {
          const dfl v = df_add_f(XV[e], RV[e]);
          XV[e] = v;
          dmax = fmaxf(dmax, fabsf(RV[e]));
          xmax = fmaxf(xmax, fabsf(v.hi));
        }
#pragma unroll
        for (int off = 16; off; off >>= 1) {
          dmax = fmaxf(dmax, __shfl_xor_sync(kFull, dmax, off));
          xmax = fmaxf(xmax, __shfl_xor_sync(kFull, xmax, off));
        }
        __syncwarp();
        const float ratio = xmax > 0.0f ? dmax / xmax : 0.0f;
        if (ratio <= 1e-7f || ratio * ratio <= 1e-6f * prev) { conv = true; break; }
        if (step >= 2 && ratio > 0.5f * prev) break;  // corrections no longer contract
        prev = ratio;
      }
      ok = conv;
    }
    if (!ok) {
      if (lane == 0) {
        const int pos = atomicAdd(mx.fb_count, 1);
        mx.fb_list[pos] = (int)item;
      }
    } else if (!LOO) {
      float2* Ci = (float2*)args.C + i * (int64_t)k * r;
      for (int e = lane; e < k * r; e += 32) Ci[e] = make_float2(XV[e].hi, XV[e].lo);
      if (args.status && lane == 0) args.status[i] = FMGP_BLOCK_OK;
    } else {
      // leave-one-out residual of x_i from its k neighbours, in DF
      dfl kx[kMaxSlots];
      const float2* xi = mx.Xdf + i * d;
#pragma unroll
      for (int s = 0; s < kMaxSlots; ++s) {
        const int a = lane + 32 * s;
        kx[s] = dfl{0.0f, 0.0f};
        if (a < k) kx[s] = kernel_df(kp, sqdist_df(xi, XS + a * d, d), mx.K);
      }
      dfl e2 = {0.0f, 0.0f};
      for (int c = 0; c < r; ++c) {
        dfl acc = {0.0f, 0.0f};
#pragma unroll
        for (int s = 0; s < kMaxSlots; ++s) {
          const int a = lane + 32 * s;
          if (a < k) acc = df_add(acc, df_mul(kx[s], XV[a * r + c]));
        }
#pragma unroll
        for (int off = 16; off; off >>= 1) {
          const dfl o = {__shfl_xor_sync(kFull, acc.hi, off), __shfl_xor_sync(kFull, acc.lo, off)};
          acc = df_add(acc, o);
        }
        const float2 y = mx.Ydf[i * r + c];
        const dfl e = df_add(dfl{y.x, y.y}, df_neg(acc));
        e2 = df_add_fast(e2, df_sqr(e));
      }
      if (lane == 0) args.resid[item] = df_to_double(e2);
    }
    __syncwarp();
  }
}

template <typename T>
__global__ void to_df_kernel(const T* in, float2* out, int64_t count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = (double)in[i];
    const float hi = (float)v;
    out[i] = make_float2(hi, (float)(v - (double)hi));
  }
}

int to_df(const void* in, bool f64, int64_t count, float2* out, cudaStream_t s) {
  if (count == 0) return FMGP_OK;
  const int blocks = (int)std::min<int64_t>(ceil_div(count, 256), (int64_t)num_sms() * 8);
  if (f64) FMGP_LAUNCH(to_df_kernel<double><<<blocks, 256, 0, s>>>((const double*)in, out, count));
  else FMGP_LAUNCH(to_df_kernel<float><<<blocks, 256, 0, s>>>((const float*)in, out, count));
  FMGP_CUDA_TRY(cudaGetLastError());
  return FMGP_OK;
}

// A5 in DF: lane a evaluates sigma^2 phi(||z - x_{S[a]}||) in DF; the k-term
// dot products with C[j*] are reduced by a fixed xor-butterfly in DF.
__global__ void __launch_bounds__(256) gather_dot_mixed_kernel(
    const float2* Xdf, int64_t n, int d, const int32_t* nbr, int ld, const float2* C, int k,
    int r, KParamsDF kp, DfConsts K, const float2* Zdf, int64_t m, const int32_t* nearest,
    double* Yhat) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= m) return;
  const int64_t j = nearest[w];
  if (j < 0 || j >= n) {
    if (lane == 0)
      for (int c = 0; c < r; ++c) Yhat[w * r + c] = __longlong_as_double(0x7ff8000000000000ll);
    return;
  }
  const float2* z = Zdf + w * d;
  dfl kz[kMaxSlots];
  const int nslots = (k + 31) / 32;
#pragma unroll
  for (int s = 0; s < kMaxSlots; ++s) {
    kz[s] = dfl{0.0f, 0.0f};
    const int a = lane + 32 * s;
    if (s < nslots && a < k) {
      int64_t idx = (a == 0) ? j : (int64_t)nbr[j * ld + a - 1];
      if (idx < 0 || idx >= n) idx = j;
      kz[s] = kernel_df(kp, sqdist_df(z, Xdf + idx * d, d), K);
    }
  }
  for (int c = 0; c < r; ++c) {
    dfl acc = {0.0f, 0.0f};
#pragma unroll
    for (int s = 0; s < kMaxSlots; ++s) {
      const int a = lane + 32 * s;
      if (s < nslots && a < k) {
        const float2 cc = C[(j * k + a) * r + c];
        acc = df_add(acc, df_mul(kz[s], dfl{cc.x, cc.y}));
      }
    }
#pragma unroll
    for (int off = 16; off; off >>= 1) {
      const dfl o = {__shfl_xor_sync(kFull, acc.hi, off), __shfl_xor_sync(kFull, acc.lo, off)};
      acc = df_add(acc, o);
    }
    if (lane == 0) Yhat[w * r + c] = df_to_double(acc);
  }
}

}  // namespace

size_t mixed_bytes_per_warp(int k, int d, int r) { return mixed_layout(k, d, r).bytes; }

int run_block_mixed(BlockArgs a, const void* X, fmgp_dtype dtype, bool loo, int warps,
                    const fmgp_kernel& kern, Workspace& ws, cudaStream_t s) {
  MixedArgs mx;
  float2* Xdf = ws.get<float2>((size_t)a.n * a.d);
  float2* Ydf = ws.get<float2>((size_t)a.n * a.r);
  int* fb_list = ws.get<int>(a.count > 0 ? a.count : 1);
  int* fb_count = ws.get<int>(1);
  if (!Xdf || !Ydf || !fb_list || !fb_count) return FMGP_ENOMEM;
  int rc = to_df(X, dtype == FMGP_F64, a.n * a.d, Xdf, s);
  if (!rc) rc = to_df(a.Y, true, a.n * a.r, Ydf, s);
  if (rc) return rc;
  FMGP_CUDA_TRY(cudaMemsetAsync(fb_count, 0, sizeof(int), s));
  mx.Xdf = Xdf;
  mx.Ydf = Ydf;
  mx.fb_list = fb_list;
  mx.fb_count = fb_count;
  mx.K = df_consts();
  mx.kdf = make_kparams_df(a.kp, kern);
  const MixedLayout lay = mixed_layout(a.k, a.d, a.r);
  const size_t smem = lay.bytes * warps;
  const int64_t need = (a.count + warps - 1) / warps;
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)num_sms() * 16));
  auto kern_fn = loo ? block_mixed_kernel<true> : block_mixed_kernel<false>;
  FMGP_CUDA_TRY(cudaFuncSetAttribute(kern_fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  FMGP_LAUNCH(kern_fn<<<blocks, warps * 32, smem, s>>>(a, mx, lay));
  FMGP_CUDA_TRY(cudaGetLastError());
  // FP64 fallback over the listed blocks (count read on the device)
  BlockArgs f = a;
  f.list = fb_list;
  f.list_count = fb_count;
  f.c_df = !loo;
  f.layout = block_layout(a.k, a.d, a.r, dtype == FMGP_F64 ? 8 : 4, false);
  int fw = (int)((200 * 1024) / f.layout.bytes_per_warp);
  fw = fw > 4 ? 4 : (fw < 1 ? 1 : fw);
  return launch_block_f64(f, X, dtype, loo, fw, s, num_sms() * 2);
}

int gather_dot_mixed(const void* X, fmgp_dtype dtype, int64_t n, int d, const int32_t* nbr, int ld,
                     const void* C, int k, int r, const KParams& kp, const fmgp_kernel& kern,
                     const void* Z, int64_t m, const int32_t* nearest, double* Yhat,
                     Workspace& ws, cudaStream_t stream) {
  if (m == 0) return FMGP_OK;
  float2* Xdf = ws.get<float2>((size_t)n * d);
  float2* Zdf = ws.get<float2>((size_t)m * d);
  if (!Xdf || !Zdf) return FMGP_ENOMEM;
  int rc = to_df(X, dtype == FMGP_F64, n * d, Xdf, stream);
  if (!rc) rc = to_df(Z, dtype == FMGP_F64, m * d, Zdf, stream);
  if (rc) return rc;
  const int blocks = ceil_div(m * 32, 256);
  FMGP_LAUNCH(gather_dot_mixed_kernel<<<blocks, 256, 0, stream>>>(
      Xdf, n, d, nbr, ld, (const float2*)C, k, r, make_kparams_df(kp, kern), df_consts(), Zdf, m,
      nearest, Yhat));
  FMGP_CUDA_TRY(cudaGetLastError());
  return FMGP_OK;
}

}  // namespace fmgp
