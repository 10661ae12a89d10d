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
#include <type_traits>
#include "block.cuh"
#include "df.cuh"
#include "predict.cuh"

namespace fmgp {
namespace {

constexpr int kMaxSlots = kMaxK / 32;
constexpr int kMaxRefine = 6;
// one-warp layouts above this size (fewer than about four neighbourhoods per
// SM) go to the CTA-per-neighbourhood kernel
constexpr size_t kMixedCtaAbove = 56 * 1024;
constexpr size_t kMixedHead = 1536;  // per-CTA shared memory before the warps' areas
static_assert(sizeof(DfConsts) <= kMixedHead, "the staged exponential table must fit the head");

// The mixed kernels work with correlations phi (sigma^2 factored out): the
// block solved is M = K / sigma^2 (diagonal 1 + tau^2), so C = M^{-1} Y / sigma^2,
// and predictions multiply the dot product by sigma^2 once.
struct KParamsDF {
  int kind, nu2;
  dfl scale;    // sqrt(2 nu)/rho (Matern) or 1/(2 rho^2) (RBF)
  dfl var;      // sigma^2
  dfl inv_var;  // 1 / sigma^2
  dfl diag;     // 1 + tau^2
  dfl third;    // 1/3
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
  q.inv_var = split(1.0 / k.variance);
  q.diag = split(1.0 + k.nugget);
  q.third = split(1.0 / 3.0);
  return q;
}

const DfConsts& df_consts() {
  static DfConsts c;
  static std::once_flag once;
  std::call_once(once, []() {
    auto put = [](float2& dst, double v) {
      const float hi = (float)v;
      dst = make_float2(hi, (float)(v - (double)hi));
    };
    for (int i = 0; i < kDfExpTable * 4; ++i) put(c.e4[i], exp(-(double)i / 4.0));
    for (int i = 0; i < 64; ++i) put(c.e256[i], exp(-(double)i / 256.0));
  });
  return c;
}

// Stage the exponential's tables in shared memory (lanes index them with
// different entries, which the constant bank would serialise).
__device__ __forceinline__ void stage_df_consts(DfConsts& dst, const DfConsts& src) {
  for (int t = threadIdx.x; t < kDfExpTable * 4; t += blockDim.x) dst.e4[t] = src.e4[t];
  for (int t = threadIdx.x; t < 64; t += blockDim.x) dst.e256[t] = src.e256[t];
}

// Correlation phi at DF squared distance D (Eq. 3 closed forms / RBF).
__device__ __forceinline__ dfl corr_df(const KParamsDF& p, dfl D, const DfConsts& K) {
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
  return ph;
}

// Squared distance in DF; the first coordinate's square starts the sum (d >= 1).
__device__ __forceinline__ dfl sqdist_df(const float2* a, const float2* b, int d) {
  float2 u = a[0], v = b[0];
  dfl s = df_sqr(df_add_fast(dfl{u.x, u.y}, dfl{-v.x, -v.y}));
  for (int t = 1; t < d; ++t) {
    u = a[t];
    v = b[t];
    const dfl diff = df_add_fast(dfl{u.x, u.y}, dfl{-v.x, -v.y});
    s = df_add_fast(s, df_sqr(diff));
  }
  return s;
}

// U kernel entries at once (pairs aa[u], bb[u] of the staged rows), the
// kernel-kind switch hoisted so that the U evaluations interleave.
template <int U>
__device__ __forceinline__ void corr_df_multi(const KParamsDF& p, const float2* XS, int d,
                                              const int* aa, const int* bb, const DfConsts& K,
                                              dfl* out) {
  dfl D[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const float2 x = XS[aa[u] * d], y = XS[bb[u] * d];
    D[u] = df_sqr(df_add_fast(dfl{x.x, x.y}, dfl{-y.x, -y.y}));
  }
  for (int t = 1; t < d; ++t) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const float2 x = XS[aa[u] * d + t], y = XS[bb[u] * d + t];
      const dfl diff = df_add_fast(dfl{x.x, x.y}, dfl{-y.x, -y.y});
      D[u] = df_add_fast(D[u], df_sqr(diff));
    }
  }
  if (p.kind == FMGP_KERNEL_RBF) {
#pragma unroll
    for (int u = 0; u < U; ++u) out[u] = df_exp_neg(df_mul(D[u], p.scale), K);
  } else if (p.nu2 == 1) {
#pragma unroll
    for (int u = 0; u < U; ++u) out[u] = df_exp_neg(df_mul(df_sqrt(D[u]), p.scale), K);
  } else if (p.nu2 == 3) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const dfl a = df_mul(df_sqrt(D[u]), p.scale);
      out[u] = df_mul(df_add_f(a, 1.0f), df_exp_neg(a, K));
    }
  } else {
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const dfl a = df_mul(df_sqrt(D[u]), p.scale);
      out[u] = df_mul(df_add(df_add_f(a, 1.0f), df_mul(df_sqr(a), p.third)), df_exp_neg(a, K));
    }
  }
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
  int ldl;  // row stride of the factor: multiple of 4 and = 4 (mod 8), so rows are
            // 16-byte aligned and float4 row reads by 8 consecutive lanes hit
            // distinct bank groups
  size_t off_L, off_LO, off_X, off_Y, off_V, off_R, off_inv, off_S, off_flag, bytes;
};

// Per-warp shared memory of the mixed block kernel.  The factor matrix M
// (k x ldl floats) holds, after assembly, hi(K_ab) in BOTH triangles; the
// Cholesky overwrites only the lower triangle and the diagonal, so hi(K_ab)
// for the residual stays available in the upper triangle, while lo(K_ab) is
// kept in a packed strict-lower array LO.
MixedLayout mixed_layout(int k, int d, int r) {
  MixedLayout l;
  int ldl = (k + 3) & ~3;
  if (ldl % 8 == 0) ldl += 4;
  l.ldl = ldl;
  auto up = [](size_t x) { return (x + 15) & ~(size_t)15; };
  size_t o = 0;
  l.off_L = o;    o += up((size_t)k * ldl * 4);
  l.off_LO = o;   o += up((size_t)k * (k - 1) / 2 * 4 + 4);
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

// L y = b then L^T x = y for column c of R (k x r), L the lower triangle of
// M (stride ldl) with inverse diagonal invd.  Rows are taken 32 at a time,
// lane = row within the block: contributions of finished blocks are
// subtracted with dot products, the block itself is solved through shuffles.
__device__ __forceinline__ void solve_f32(const float* M, int ldl, const float* invd, float* R,
                                          int k, int r, int lane) {
  const int nblk = (k + 31) >> 5;
  for (int c = 0; c < r; ++c) {
    // forward (branch-free across lanes: a row past the end works on the
    // last row, and its value is never broadcast or stored)
    for (int q = 0; q < nblk; ++q) {
      const int row = 32 * q + lane;
      const bool valid = row < k;
      const int rc = min(row, k - 1);
      float v = valid ? R[row * r + c] : 0.0f;
      const float iv = valid ? invd[row] : 0.0f;
      if (q > 0) {
        const float* mr = M + rc * ldl;
        float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
        if (r == 1) {
          for (int p = 0; p < 32 * q; p += 4) {
            const float4 a = *reinterpret_cast<const float4*>(mr + p);
            const float4 x = *reinterpret_cast<const float4*>(R + p);
            s0 = fmaf(a.x, x.x, s0); s1 = fmaf(a.y, x.y, s1);
            s2 = fmaf(a.z, x.z, s2); s3 = fmaf(a.w, x.w, s3);
          }
        } else {
          for (int p = 0; p < 32 * q; ++p) s0 = fmaf(mr[p], R[p * r + c], s0);
        }
        v -= (s0 + s1) + (s2 + s3);
      }
      const float* mb = M + rc * ldl + 32 * q;
      if (32 * q + 32 <= k) {
#pragma unroll 8
        for (int t = 0; t < 32; ++t) {
          const float mv = mb[t];
          const float m = (lane > t && valid) ? mv : 0.0f;
          const float xt = __shfl_sync(kFull, v * iv, t);
          v = (lane == t) ? xt : fmaf(-m, xt, v);
        }
      } else {
        const int tmax = k - 32 * q;
        for (int t = 0; t < tmax; ++t) {
          const float mv = mb[t];
          const float m = (lane > t && valid) ? mv : 0.0f;
          const float xt = __shfl_sync(kFull, v * iv, t);
          v = (lane == t) ? xt : fmaf(-m, xt, v);
        }
      }
      if (valid) R[row * r + c] = v;
      __syncwarp();
    }
    // backward
    for (int q = nblk - 1; q >= 0; --q) {
      const int row = 32 * q + lane;
      const bool valid = row < k;
      const int rc = min(row, k - 1);
      float v = valid ? R[row * r + c] : 0.0f;
      const float iv = valid ? invd[row] : 0.0f;
      {
        float s0 = 0.f, s1 = 0.f;
        int p = 32 * (q + 1);
        for (; p + 1 < k; p += 2) {
          s0 = fmaf(M[p * ldl + rc], R[p * r + c], s0);
          s1 = fmaf(M[(p + 1) * ldl + rc], R[(p + 1) * r + c], s1);
        }
        if (p < k) s0 = fmaf(M[p * ldl + rc], R[p * r + c], s0);
        v -= s0 + s1;
      }
      const int tmax = min(32, k - 32 * q);
      if (tmax == 32) {
#pragma unroll 8
        for (int t = 31; t >= 0; --t) {
          const float mv = M[(32 * q + t) * ldl + rc];
          const float m = (lane < t && valid) ? mv : 0.0f;
          const float xt = __shfl_sync(kFull, v * iv, t);
          v = (lane == t) ? xt : fmaf(-m, xt, v);
        }
      } else {
        for (int t = tmax - 1; t >= 0; --t) {
          const float mv = M[(32 * q + t) * ldl + rc];
          const float m = (lane < t && valid) ? mv : 0.0f;
          const float xt = __shfl_sync(kFull, v * iv, t);
          v = (lane == t) ? xt : fmaf(-m, xt, v);
        }
      }
      if (valid) R[row * r + c] = v;
      __syncwarp();
    }
  }
}

template <int MODE, int NS, int CB>
__global__ void __launch_bounds__(NS == 2 ? 192 : 256, NS >= 5 ? 1 : 2) block_mixed_kernel(BlockArgs args, MixedArgs mx,
                                                          MixedLayout lay) {
  constexpr bool LOO = MODE == kModeLoocv;
  static_assert(CB % 4 == 0, "panels start at multiples of 4 (float4 reads of finished columns)");
  extern __shared__ __align__(16) unsigned char smem[];
  const int wpb = blockDim.x >> 5;
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // the exponential's constants, staged once per CTA: lanes index the table
  // with different j, which the constant bank would serialise
  DfConsts& Ks = *reinterpret_cast<DfConsts*>(smem);
  stage_df_consts(Ks, mx.K);
  __syncthreads();
  unsigned char* base = smem + kMixedHead + (size_t)wid * lay.bytes;
  float* M = (float*)(base + lay.off_L);
  float* LO = (float*)(base + lay.off_LO);
  float2* XS = (float2*)(base + lay.off_X);
  dfl* YS = (dfl*)(base + lay.off_Y);
  dfl* XV = (dfl*)(base + lay.off_V);
  float* RV = (float*)(base + lay.off_R);
  float* invd = (float*)(base + lay.off_inv);
  int* S = (int*)(base + lay.off_S);
  volatile int* flag = (int*)(base + lay.off_flag);
  const int k = args.k, d = args.d, r = args.r, ldl = lay.ldl;
  const KParamsDF kp = mx.kdf;

  // the next item is claimed once the factorisation is done: the claim's
  // latency hides behind the solves and the refinement, and it holds no
  // registers through the assembly and the Cholesky
  const int64_t stride = (int64_t)gridDim.x * wpb;
  unsigned long long claim = 0;
  for (int64_t item = (int64_t)blockIdx.x * wpb + wid; item < args.count;
       item = stride + (int64_t)__shfl_sync(kFull, claim, 0)) {
    int64_t i = LOO ? args.batch[item]
                    : (MODE == kModePrecompute && args.rows ? (int64_t)args.rows[item] : item);
    const int64_t orow = MODE == kModePrecompute && args.rows ? item : i;  // row of C / status
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
      XS[e] = mx.Xdf[(int64_t)S[a] * d + t];
    }
    for (int e = lane; e < k * r; e += 32) {
      const int a = e / r, c = e - a * r;
      const float2 y = mx.Ydf[(int64_t)S[a] * r + c];
      YS[e] = dfl{y.x, y.y};
    }
    __syncwarp();
    // assembly: pair p = a(a-1)/2 + b (a > b), walked incrementally per lane
    {
      const int npairs = k * (k - 1) / 2;
      int a = 1, b = lane;
      while (b >= a) { b -= a; ++a; }
      // three entries per iteration, evaluated together for instruction-level
      // parallelism (out-of-range slots evaluate a dummy pair and are dropped)
      constexpr int U = 3;
      for (int p = lane; p < npairs; p += 32 * U) {
        int aa[U], bb[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const bool v = p + 32 * u < npairs;
          aa[u] = v ? a : 1;
          bb[u] = v ? b : 0;
          b += 32;
          while (b >= a) { b -= a; ++a; }
        }
        dfl kv[U];
        corr_df_multi<U>(kp, XS, d, aa, bb, Ks, kv);
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (p + 32 * u < npairs) {
            M[aa[u] * ldl + bb[u]] = kv[u].hi;
            M[bb[u] * ldl + aa[u]] = kv[u].hi;
            LO[p + 32 * u] = kv[u].lo;
          }
        }
      }
    }
    for (int a = lane; a < k; a += 32) M[a * ldl + a] = kp.diag.hi;
    __syncwarp();
    // FP32 Cholesky of the lower triangle of M, left-looking in panels of CB
    // columns: the dot products of every row with the panel's columns over
    // the finished prefix are formed in one pass (each row chunk read once
    // for CB columns), then the panel is factored in Crout order with pivots
    // broadcast by shuffle.  Rows are counted from the panel's first column:
    // lane l owns rows j0 + l, j0 + l + 32, ..., so the rows still active
    // fill the low lanes and a panel needs only ceil((k - j0) / 32) slots,
    // and the pivot row of panel column c is always lane c's first slot.
    // The loops below are branch-free across lanes: rows past the end are
    // clamped to the last row (their values are computed and never stored),
    // and only the warp-uniform slot count ns guards a slot.
    bool fail = false;
    for (int j0 = 0; j0 < k; j0 += CB) {
      const int nb = min(CB, k - j0);
      const int ns = (k - j0 + 31) >> 5;  // slots in use (warp-uniform)
      float acc[NS][CB];
      bool act[NS];
      int rr[NS];  // row of each slot, clamped into the matrix
#pragma unroll
      for (int s4 = 0; s4 < NS; ++s4) {
        const int r = j0 + lane + 32 * s4;
        act[s4] = s4 < ns && r < k;
        rr[s4] = min(r, k - 1);
#pragma unroll
        for (int c = 0; c < CB; ++c) {
          const float v = M[rr[s4] * ldl + min(j0 + c, k - 1)];
          acc[s4][c] = (c < nb && j0 + c <= r) ? v : 0.0f;
        }
      }
      for (int p = 0; p < j0; p += 4) {
        float4 bc[CB];
#pragma unroll
        for (int c = 0; c < CB; ++c)
          bc[c] = *reinterpret_cast<const float4*>(M + min(j0 + c, k - 1) * ldl + p);
#pragma unroll
        for (int s4 = 0; s4 < NS; ++s4) {
          if (s4 >= ns) break;
          const float4 a4 = *reinterpret_cast<const float4*>(M + rr[s4] * ldl + p);
#pragma unroll
          for (int c = 0; c < CB; ++c) {
            float t = acc[s4][c];
            t = fmaf(-a4.x, bc[c].x, t);
            t = fmaf(-a4.y, bc[c].y, t);
            t = fmaf(-a4.z, bc[c].z, t);
            t = fmaf(-a4.w, bc[c].w, t);
            acc[s4][c] = t;
          }
        }
      }
      // panel: columns j0 .. j0+nb-1 in order
      float lr[NS][CB];
#pragma unroll
      for (int s4 = 0; s4 < NS; ++s4)
#pragma unroll
        for (int c = 0; c < CB; ++c) lr[s4][c] = 0.0f;
#pragma unroll
      for (int c = 0; c < CB; ++c) {
        if (c >= nb) break;
        const int col = j0 + c;
        // the pivot row's finished entries L[col][j0 .. col-1] and its reduced
        // diagonal, from lane c's first slot
        float lc[CB];
#pragma unroll
        for (int c2 = 0; c2 < CB; ++c2) lc[c2] = c2 < c ? __shfl_sync(kFull, lr[0][c2], c) : 0.0f;
        float dv = __shfl_sync(kFull, acc[0][c], c);
#pragma unroll
        for (int c2 = 0; c2 < CB; ++c2)
          if (c2 < c) dv = fmaf(-lc[c2], lc[c2], dv);
        if (!(dv > 0.0f)) { fail = true; break; }
        const float inv = rsqrtf(dv);
        if (lane == c) {
          M[col * ldl + col] = dv * inv;
          invd[col] = inv;
        }
#pragma unroll
        for (int s4 = 0; s4 < NS; ++s4) {
          if (s4 >= ns) break;
          const int r = j0 + lane + 32 * s4;
          float t = acc[s4][c];
#pragma unroll
          for (int c2 = 0; c2 < CB; ++c2)
            if (c2 < c) t = fmaf(-lr[s4][c2], lc[c2], t);
          t *= inv;
          lr[s4][c] = t;  // rows at or above the pivot never read it
          if (act[s4] && r > col) M[r * ldl + col] = t;
        }
      }
      __syncwarp();
      if (fail) break;
    }
    if (lane == 0) *flag = fail ? 1 : 0;
    claim = block_claim(args.queue, item, lane == 0);
    __syncwarp();
    bool ok = (*flag == 0) && !bad;
    if (ok) {
      for (int e = lane; e < k * r; e += 32) RV[e] = YS[e].hi;
      __syncwarp();
      solve_f32(M, ldl, invd, RV, k, r, lane);
      for (int e = lane; e < k * r; e += 32) XV[e] = dfl{RV[e], 0.0f};
      __syncwarp();
      float prev = 1.0f;
      bool conv = false;
      for (int step = 1; step <= kMaxRefine; ++step) {
        // residual y - K x; lane owns rows; K_ab = (upper hi, packed lo).
        // Compensated dot product (Dot2 of Ogita, Rump & Oishi, SIAM J. Sci.
        // Comput. 26, 2005): the leading products hi * x.hi are split exactly
        // (TwoProduct by FMA) and summed with TwoSum into p; the rounding
        // errors and the small cross terms hi * x.lo + lo * x.hi collect in
        // one FP32 sum e.  The result is as accurate as if computed with twice
        // the working precision (error ~u|r| + (n u)^2 sum |K_ab x_b|), far
        // below what the FP32 correction solve can use; only fl(p + e) is
        // passed on.
        for (int c = 0; c < r; ++c) {
          float p[NS], e[NS];
#pragma unroll
          for (int s = 0; s < NS; ++s) {
            const int row = lane + 32 * s;
            p[s] = 0.0f;
            e[s] = 0.0f;
            if (row < k) {
              const dfl a = df_add(YS[row * r + c], df_neg(df_mul(kp.diag, XV[row * r + c])));
              p[s] = a.hi;
              e[s] = a.lo;
            }
          }
          int cb = 0;  // b(b-1)/2
#pragma unroll 2
          for (int b = 0; b < k; ++b) {
            const dfl xb = XV[b * r + c];
#pragma unroll
            for (int s = 0; s < NS; ++s) {
              // branch-free across lanes: a row past the end reads the last
              // row, and it and the diagonal term contribute exact zeros
              const int row = lane + 32 * s;
              const int rc = min(row, k - 1);
              const bool use = row < k && b != row;
              {
                // K_row,b = (M[b][row], LO[row(row-1)/2 + b]) below the diagonal,
                // (M[row][b], LO[b(b-1)/2 + row]) above it
                const bool below = b < rc;
                float hi = below ? M[b * ldl + rc] : M[rc * ldl + b];
                float lo = below ? LO[rc * (rc - 1) / 2 + b] : LO[cb + rc];
                hi = use ? hi : 0.0f;
                lo = use ? lo : 0.0f;
                const float h = __fmul_rn(hi, xb.hi);
                const float hr = __fmaf_rn(hi, xb.hi, -h);  // hi * x.hi = h + hr exactly
                const float t = __fadd_rn(p[s], -h);        // TwoSum(p, -h) = t + q
                const float bv = __fsub_rn(t, p[s]);
                const float q = __fadd_rn(__fsub_rn(p[s], __fsub_rn(t, bv)), __fsub_rn(-h, bv));
                p[s] = t;
                float es = __fsub_rn(e[s], hr);
                es = __fadd_rn(es, q);
                es = __fmaf_rn(-hi, xb.lo, es);
                e[s] = __fmaf_rn(-lo, xb.hi, es);
              }
            }
            cb += b;
          }
#pragma unroll
          for (int s = 0; s < NS; ++s) {
            const int row = lane + 32 * s;
            if (row < k) RV[row * r + c] = __fadd_rn(p[s], e[s]);
          }
        }
        __syncwarp();
        solve_f32(M, ldl, invd, RV, k, r, lane);
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
    } else if (MODE == kModePrecompute) {
      float2* Ci = (float2*)args.C + orow * (int64_t)k * r;
      for (int e = lane; e < k * r; e += 32) {
        const dfl cv = df_mul(XV[e], kp.inv_var);
        Ci[e] = make_float2(cv.hi, cv.lo);
      }
      if (args.status && lane == 0) args.status[orow] = FMGP_BLOCK_OK;
    } else {
      // cross-covariance of the query point (x_i for LOOCV, z_t for MuyGPs), in DF
      dfl kx[NS];
      const float2* xi = MODE == kModeMuygps ? args.Zdf + i * d : mx.Xdf + i * d;
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        const int a = lane + 32 * s;
        kx[s] = dfl{0.0f, 0.0f};
        if (a < k) kx[s] = corr_df(kp, sqdist_df(xi, XS + a * d, d), Ks);
      }
      dfl e2 = {0.0f, 0.0f};
      for (int c = 0; c < r; ++c) {
        dfl acc = {0.0f, 0.0f};
#pragma unroll
        for (int s = 0; s < NS; ++s) {
          const int a = lane + 32 * s;
          if (a < k) acc = df_add(acc, df_mul(kx[s], XV[a * r + c]));
        }
#pragma unroll
        for (int off = 16; off; off >>= 1) {
          const dfl o = {__shfl_xor_sync(kFull, acc.hi, off), __shfl_xor_sync(kFull, acc.lo, off)};
          acc = df_add(acc, o);
        }
        if (MODE == kModeMuygps) {
          // correlations times M^{-1} y; sigma^2 cancels (K = sigma^2 M)
          if (lane == 0) args.yhat[i * r + c] = df_to_double(acc);
        } else {
          const float2 y = mx.Ydf[i * r + c];
          const dfl e = df_add(dfl{y.x, y.y}, df_neg(acc));
          e2 = df_add_fast(e2, df_sqr(e));
        }
      }
      if (lane == 0 && MODE == kModeLoocv) args.resid[item] = df_to_double(e2);
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// One CTA per neighbourhood, for neighbourhoods whose one-warp layout would
// leave few warps per SM (large k, or many features): the same method as
// block_mixed_kernel with the work spread over kCtaWarps warps.
//   assembly: all threads, one kernel entry at a time, staged rows in shared
//     memory as FP32 (FP32 inputs: differences formed exactly by TwoSum) or
//     as double-float pairs (FP64 inputs);
//   FP32 Cholesky in Crout order: thread t forms row t of column j (a float4
//     dot product over the finished prefix), two barriers per column;
//   triangular solves: warp 0 (shuffle sweeps, as in the one-warp kernel);
//   refinement residual: thread t forms row t as a compensated dot product;
//   the stopping rule, the FP64 fallback list and the outputs as the one-warp
//   kernel.
constexpr int kCtaWarps = 8;

__device__ __forceinline__ void pair_index(int p, int& a, int& b) {
  int x = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)p)) * 0.5f);
  while (x * (x - 1) / 2 > p) --x;
  while ((x + 1) * x / 2 <= p) ++x;
  a = x;
  b = p - x * (x - 1) / 2;
}

// a - b as an exact pair, for FP32 or double-float coordinates.
__device__ __forceinline__ dfl coord_diff(float a, float b) { return df_two_sum(a, -b); }
__device__ __forceinline__ dfl coord_diff(float2 a, float2 b) {
  return df_add_fast(dfl{a.x, a.y}, dfl{-b.x, -b.y});
}
__device__ __forceinline__ dfl coord_diff(float2 a, float b) {
  return df_add_fast(dfl{a.x, a.y}, dfl{-b, 0.0f});
}

template <typename A, typename B>
__device__ __forceinline__ dfl sqdist_any(const A* a, const B* b, int d) {
  dfl s = df_sqr(coord_diff(a[0], b[0]));
  for (int t = 1; t < d; ++t) s = df_add_fast(s, df_sqr(coord_diff(a[t], b[t])));
  return s;
}

struct MixedCtaLayout {
  int ldl;  // multiple of 4, = 4 (mod 8): float4 row reads conflict-free
  size_t off_L, off_LO, off_X, off_Y, off_V, off_R, off_inv, off_S, off_red, bytes;
};

MixedCtaLayout mixed_cta_layout(int k, int d, int r, size_t xelem) {
  MixedCtaLayout l;
  int ldl = (k + 3) & ~3;
  if (ldl % 8 == 0) ldl += 4;
  l.ldl = ldl;
  auto up = [](size_t x) { return (x + 15) & ~(size_t)15; };
  size_t o = 0;
  l.off_L = o;   o += up((size_t)k * ldl * 4);
  l.off_LO = o;  o += up((size_t)k * (k - 1) / 2 * 4 + 4);
  l.off_X = o;   o += up((size_t)k * d * xelem);
  l.off_Y = o;   o += up((size_t)k * r * 8);
  l.off_V = o;   o += up((size_t)k * r * 8);
  l.off_R = o;   o += up((size_t)k * r * 4);
  l.off_inv = o; o += up((size_t)k * 4);
  l.off_S = o;   o += up((size_t)k * 4);
  l.off_red = o; o += up(2 * kCtaWarps * 4 + 16);
  l.bytes = o;
  return l;
}

template <int MODE, typename XT, int NW>
__global__ void __launch_bounds__(NW * 32, 2) block_mixed_cta_kernel(
    BlockArgs args, MixedArgs mx, MixedCtaLayout lay, const XT* __restrict__ Xrows) {
  constexpr bool LOO = MODE == kModeLoocv;
  constexpr int NT = NW * 32;
  extern __shared__ __align__(16) unsigned char smem[];
  DfConsts& Ks = *reinterpret_cast<DfConsts*>(smem);
  stage_df_consts(Ks, mx.K);
  unsigned char* base = smem + kMixedHead;
  float* M = (float*)(base + lay.off_L);
  float* LO = (float*)(base + lay.off_LO);
  XT* XS = (XT*)(base + lay.off_X);
  dfl* YS = (dfl*)(base + lay.off_Y);
  dfl* XV = (dfl*)(base + lay.off_V);
  float* RV = (float*)(base + lay.off_R);
  float* invd = (float*)(base + lay.off_inv);
  int* S = (int*)(base + lay.off_S);
  float* red = (float*)(base + lay.off_red);
  volatile int* flag = (int*)(red + 2 * NW);
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int k = args.k, d = args.d, r = args.r, ldl = lay.ldl;
  const KParamsDF kp = mx.kdf;

  __shared__ unsigned long long next_item;
  for (int64_t item = blockIdx.x; item < args.count; item = (int64_t)next_item) {
    __syncthreads();  // the previous neighbourhood is finished with shared memory and next_item
    unsigned long long claim = 0;
    if (tid == 0) claim = block_claim(args.queue, item, true);
    int64_t i = LOO ? args.batch[item]
                    : (MODE == kModePrecompute && args.rows ? (int64_t)args.rows[item] : item);
    const int64_t orow = MODE == kModePrecompute && args.rows ? item : i;
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
    for (int e = tid; e < k * d; e += NT) {
      const int a = e / d, t = e - a * d;
      XS[e] = Xrows[(int64_t)S[a] * d + t];
    }
    for (int e = tid; e < k * r; e += NT) {
      const int a = e / r, c = e - a * r;
      const float2 y = mx.Ydf[(int64_t)S[a] * r + c];
      YS[e] = dfl{y.x, y.y};
    }
    __syncthreads();
    // assembly: entry p = a(a-1)/2 + b (a > b) per thread
    const int npairs = k * (k - 1) / 2;
    for (int p = tid; p < npairs; p += NT) {
      int a, b;
      pair_index(p, a, b);
      const dfl kv = corr_df(kp, sqdist_any(XS + a * d, XS + b * d, d), Ks);
      M[a * ldl + b] = kv.hi;
      M[b * ldl + a] = kv.hi;
      LO[p] = kv.lo;
    }
    if (tid < k) M[tid * ldl + tid] = kp.diag.hi;
    __syncthreads();
    // FP32 Cholesky, Crout order: thread t forms row t of column j
    for (int j = 0; j < k; ++j) {
      float dd = 0.0f;
      if (tid >= j && tid < k) {
        const float* lr = M + tid * ldl;
        const float* lj = M + j * ldl;
        float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
        int p = 0;
        for (; p + 4 <= j; p += 4) {
          const float4 u = *reinterpret_cast<const float4*>(lr + p);
          const float4 v = *reinterpret_cast<const float4*>(lj + p);
          s0 = fmaf(u.x, v.x, s0); s1 = fmaf(u.y, v.y, s1);
          s2 = fmaf(u.z, v.z, s2); s3 = fmaf(u.w, v.w, s3);
        }
        for (; p < j; ++p) s0 = fmaf(lr[p], lj[p], s0);
        dd = (s0 + s1) + (s2 + s3);
      }
      if (tid == j) {
        const float v = M[j * ldl + j] - dd;
        if (!(v > 0.0f)) {
          *flag = 1;
        } else {
          const float iv = rsqrtf(v);
          M[j * ldl + j] = v * iv;
          invd[j] = iv;
        }
      }
      __syncthreads();
      if (*flag) break;
      if (tid > j && tid < k) M[tid * ldl + j] = (M[tid * ldl + j] - dd) * invd[j];
      __syncthreads();
    }
    bool ok = (*flag == 0) && !bad;
    if (ok) {
      for (int e = tid; e < k * r; e += NT) RV[e] = YS[e].hi;
      __syncthreads();
      if (wid == 0) solve_f32(M, ldl, invd, RV, k, r, lane);
      __syncthreads();
      for (int e = tid; e < k * r; e += NT) XV[e] = dfl{RV[e], 0.0f};
      __syncthreads();
      float prev = 1.0f;
      bool conv = false;
      for (int step = 1; step <= kMaxRefine; ++step) {
        // residual y - K x, row `tid`, compensated (Dot2) as in the one-warp kernel
        if (tid < k) {
          const int row = tid;
          const int rb = row * (row - 1) / 2;
          for (int c = 0; c < r; ++c) {
            const dfl a0 = df_add(YS[row * r + c], df_neg(df_mul(kp.diag, XV[row * r + c])));
            float pp = a0.hi, ee = a0.lo;
            int cb = 0;
            for (int b = 0; b < k; ++b) {
              if (b != row) {
                const dfl xb = XV[b * r + c];
                const bool below = b < row;
                const float hi = below ? M[b * ldl + row] : M[row * ldl + b];
                const float lo = below ? LO[rb + b] : LO[cb + row];
                const float h = __fmul_rn(hi, xb.hi);
                const float hr = __fmaf_rn(hi, xb.hi, -h);
                const float t = __fadd_rn(pp, -h);
                const float bv = __fsub_rn(t, pp);
                const float q = __fadd_rn(__fsub_rn(pp, __fsub_rn(t, bv)), __fsub_rn(-h, bv));
                pp = t;
                float es = __fsub_rn(ee, hr);
                es = __fadd_rn(es, q);
                es = __fmaf_rn(-hi, xb.lo, es);
                ee = __fmaf_rn(-lo, xb.hi, es);
              }
              cb += b;
            }
            RV[row * r + c] = __fadd_rn(pp, ee);
          }
        }
        __syncthreads();
        if (wid == 0) solve_f32(M, ldl, invd, RV, k, r, lane);
        __syncthreads();
        float dmax = 0.0f, xmax = 0.0f;
        for (int e = tid; e < k * r; e += NT) {
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
        if (lane == 0) {
          red[wid] = dmax;
          red[NW + wid] = xmax;
        }
        __syncthreads();
        dmax = 0.0f;
        xmax = 0.0f;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
          dmax = fmaxf(dmax, red[w]);
          xmax = fmaxf(xmax, red[NW + w]);
        }
        __syncthreads();  // red is rewritten by the next step
        const float ratio = xmax > 0.0f ? dmax / xmax : 0.0f;
        if (ratio <= 1e-7f || ratio * ratio <= 1e-6f * prev) { conv = true; break; }
        if (step >= 2 && ratio > 0.5f * prev) break;  // corrections no longer contract
        prev = ratio;
      }
      ok = conv;
    }
    if (!ok) {
      if (tid == 0) {
        const int pos = atomicAdd(mx.fb_count, 1);
        mx.fb_list[pos] = (int)item;
      }
    } else if (MODE == kModePrecompute) {
      float2* Ci = (float2*)args.C + orow * (int64_t)k * r;
      for (int e = tid; e < k * r; e += NT) {
        const dfl cv = df_mul(XV[e], kp.inv_var);
        Ci[e] = make_float2(cv.hi, cv.lo);
      }
      if (args.status && tid == 0) args.status[orow] = FMGP_BLOCK_OK;
    } else {
      // cross-covariance of the query point with row `lane` (+32 s) in warp 0
      if (wid == 0) {
        constexpr int NSL = kMaxK / 32;
        dfl kx[NSL];
        const float2* xi = MODE == kModeMuygps ? args.Zdf + i * d : mx.Xdf + i * d;
#pragma unroll
        for (int s2 = 0; s2 < NSL; ++s2) {
          const int a = lane + 32 * s2;
          kx[s2] = dfl{0.0f, 0.0f};
          if (a < k) kx[s2] = corr_df(kp, sqdist_any(xi, XS + a * d, d), Ks);
        }
        dfl e2 = {0.0f, 0.0f};
        for (int c = 0; c < r; ++c) {
          dfl acc = {0.0f, 0.0f};
#pragma unroll
          for (int s2 = 0; s2 < NSL; ++s2) {
            const int a = lane + 32 * s2;
            if (a < k) acc = df_add(acc, df_mul(kx[s2], XV[a * r + c]));
          }
#pragma unroll
          for (int off = 16; off; off >>= 1) {
            const dfl o = {__shfl_xor_sync(kFull, acc.hi, off), __shfl_xor_sync(kFull, acc.lo, off)};
            acc = df_add(acc, o);
          }
          if (MODE == kModeMuygps) {
            if (lane == 0) args.yhat[i * r + c] = df_to_double(acc);
          } else {
            const float2 y = mx.Ydf[i * r + c];
            const dfl e = df_add(dfl{y.x, y.y}, df_neg(acc));
            e2 = df_add_fast(e2, df_sqr(e));
          }
        }
        if (lane == 0 && MODE == kModeLoocv) args.resid[item] = df_to_double(e2);
      }
    }
    if (tid == 0) next_item = (unsigned long long)gridDim.x + claim;
    __syncthreads();
  }
}

// A5 in DF: lane a evaluates sigma^2 phi(||z - x_{S[a]}||) in DF; the k-term
// dot products with C[j*] are reduced by a fixed xor-butterfly in DF.
__global__ void __launch_bounds__(256) gather_dot_mixed_kernel(
    const float2* Xdf, int64_t n, int d, const int32_t* nbr, int ld, const float2* C, int k,
    int r, KParamsDF kp, DfConsts K, const float2* Zdf, int64_t m, const int32_t* nearest,
    double* Yhat, const int32_t* crow) {
  // the exponential's constants in shared memory (lanes index the table
  // with different j, which the constant bank would serialise)
  __shared__ DfConsts Ks;
  stage_df_consts(Ks, K);
  __syncthreads();
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= m) return;
  const int64_t j = nearest[w];
  if (j < 0 || j >= n) {
    if (lane == 0)
      for (int c = 0; c < r; ++c) Yhat[w * r + c] = __longlong_as_double(0x7ff8000000000000ll);
    return;
  }
  const int64_t cj = crow ? (int64_t)crow[w] : j;  // row of C (a position for centre subsets)
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
      kz[s] = corr_df(kp, sqdist_df(z, Xdf + idx * d, d), Ks);
    }
  }
  for (int c = 0; c < r; ++c) {
    dfl acc = {0.0f, 0.0f};
#pragma unroll
    for (int s = 0; s < kMaxSlots; ++s) {
      const int a = lane + 32 * s;
      if (s < nslots && a < k) {
        const float2 cc = C[(cj * k + a) * r + c];
        acc = df_add(acc, df_mul(kz[s], dfl{cc.x, cc.y}));
      }
    }
#pragma unroll
    for (int off = 16; off; off >>= 1) {
      const dfl o = {__shfl_xor_sync(kFull, acc.hi, off), __shfl_xor_sync(kFull, acc.lo, off)};
      acc = df_add(acc, o);
    }
    if (lane == 0) Yhat[w * r + c] = df_to_double(df_mul(acc, kp.var));
  }
}

}  // namespace

// Evaluate a double-float primitive on FP64 inputs split into DF pairs:
// fn 0: exp(-x) (df_exp_neg), fn 1: sqrt(x) (df_sqrt).
__global__ void df_eval_kernel(int fn, const double* x, int64_t n, double* y, DfConsts K) {
  __shared__ DfConsts Ks;
  stage_df_consts(Ks, K);
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = x[i];
    const float hi = (float)v;
    const dfl a = {hi, (float)(v - (double)hi)};
    const dfl r = fn == 0 ? df_exp_neg(a, Ks) : df_sqrt(a);
    y[i] = df_to_double(r);
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

size_t mixed_bytes_per_warp(int k, int d, int r, int xbytes) {
  const size_t w = mixed_layout(k, d, r).bytes;
  return w > kMixedCtaAbove ? mixed_cta_layout(k, d, r, xbytes == 4 ? 4 : 8).bytes : w;
}

// FP64 fallback over the blocks the mixed kernels listed (count read on the device).
static int mixed_fallback(const BlockArgs& a, const void* X, fmgp_dtype dtype, int mode, bool loo,
                          int* fb_list, int* fb_count, cudaStream_t s) {
  BlockArgs f = a;
  f.list = fb_list;
  f.list_count = fb_count;
  f.queue = nullptr;  // a fixed grid over the device-counted list
  f.c_df = !loo;
  f.layout = block_layout(a.k, a.d, a.r, dtype == FMGP_F64 ? 8 : 4, false);
  int fw = (int)((200 * 1024) / f.layout.bytes_per_warp);
  fw = fw > 4 ? 4 : (fw < 1 ? 1 : fw);
  return launch_block_f64(f, X, dtype, mode, fw, s, num_sms() * 2);
}

int run_block_mixed(BlockArgs a, const void* X, fmgp_dtype dtype, int mode, int warps, int panel,
                    const fmgp_kernel& kern, Workspace& ws, cudaStream_t s) {
  const bool loo = mode != kModePrecompute;
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
  // persistent (one wave, claimed items) with a work counter, else eight
  // whole waves of the CTAs the SMs hold at once (grid stride)
  const int waves = a.queue ? 1 : 8;
  if (a.queue) FMGP_CUDA_TRY(cudaMemsetAsync(a.queue, 0, sizeof(unsigned long long), s));
  mx.Xdf = Xdf;
  mx.Ydf = Ydf;
  mx.fb_list = fb_list;
  mx.fb_count = fb_count;
  mx.K = df_consts();
  mx.kdf = make_kparams_df(a.kp, kern);
  const MixedLayout lay = mixed_layout(a.k, a.d, a.r);
  if (lay.bytes > kMixedCtaAbove) {
    // few one-warp neighbourhoods would fit an SM: one CTA per neighbourhood
    const bool f32 = dtype == FMGP_F32;
    const MixedCtaLayout cl = mixed_cta_layout(a.k, a.d, a.r, f32 ? 4 : 8);
    const size_t smem = kMixedHead + cl.bytes;
    auto pick = [&](auto xt) {
      using XT = typename decltype(xt)::type;
      return mode == kModeLoocv    ? block_mixed_cta_kernel<kModeLoocv, XT, kCtaWarps>
             : mode == kModeMuygps ? block_mixed_cta_kernel<kModeMuygps, XT, kCtaWarps>
                                   : block_mixed_cta_kernel<kModePrecompute, XT, kCtaWarps>;
    };
    struct TF { using type = float; };
    struct TD { using type = float2; };
    const void* fn = f32 ? (const void*)pick(TF{}) : (const void*)pick(TD{});
    const int fit = active_ctas(fn, kCtaWarps * 32, smem);
    if (!fit) {
      set_error("neighbourhood blocks of %zu bytes do not fit an SM", cl.bytes);
      return FMGP_EUNSUPPORTED;
    }
    const int blocks = (int)std::max<int64_t>(
        1, std::min<int64_t>(a.count, (int64_t)num_sms() * fit * waves));
    FMGP_CUDA_TRY(ensure_smem(fn, smem));
    if (f32)
      FMGP_LAUNCH(pick(TF{})<<<blocks, kCtaWarps * 32, smem, s>>>(a, mx, cl, (const float*)X));
    else
      FMGP_LAUNCH(pick(TD{})<<<blocks, kCtaWarps * 32, smem, s>>>(a, mx, cl, (const float2*)Xdf));
    FMGP_CUDA_TRY(cudaGetLastError());
    return mixed_fallback(a, X, dtype, mode, loo, fb_list, fb_count, s);
  }
  // rows per lane (k <= 32 S) and the Cholesky panel width are compile-time:
  // 8 columns for k <= 32 and 4 above by default; for k <= 64 the other
  // width is instantiated too (panel = 4 or 8 picks it, 0 the default)
  auto pick = [&](auto sconst, auto cbconst) {
    constexpr int SS = decltype(sconst)::value;
    constexpr int CB = decltype(cbconst)::value;
    return mode == kModeLoocv    ? block_mixed_kernel<kModeLoocv, SS, CB>
           : mode == kModeMuygps ? block_mixed_kernel<kModeMuygps, SS, CB>
                                 : block_mixed_kernel<kModePrecompute, SS, CB>;
  };
  using I4 = std::integral_constant<int, 4>;
  using I8 = std::integral_constant<int, 8>;
  const int S = (a.k + 31) / 32;
  auto kern_fn = S == 1 ? (panel == 4 ? pick(std::integral_constant<int, 1>{}, I4{})
                                      : pick(std::integral_constant<int, 1>{}, I8{}))
               : S == 2 ? (panel == 8 ? pick(std::integral_constant<int, 2>{}, I8{})
                                      : pick(std::integral_constant<int, 2>{}, I4{}))
               : S == 3 ? pick(std::integral_constant<int, 3>{}, I4{})
               : S == 4 ? pick(std::integral_constant<int, 4>{}, I4{})
                        : pick(std::integral_constant<int, 5>{}, I4{});
  int nb = 0;
  {
    // the 2-slot instantiation is compiled for at most 192 threads (6 warps)
    cudaFuncAttributes fa;
    FMGP_CUDA_TRY(cudaFuncGetAttributes(&fa, (const void*)kern_fn));
    const int maxw = fa.maxThreadsPerBlock / 32;
    if (warps > maxw) warps = maxw;
    if (warps <= 0) {  // the CTA size with the most resident warps per SM (ties: larger)
      int best = 0;
      for (int w : {8, 6, 4, 3, 2, 1}) {
        if (w > maxw) continue;
        const int c = active_ctas((const void*)kern_fn, w * 32, kMixedHead + lay.bytes * w);
        if (c * w > best) { best = c * w; warps = w; nb = c; }
      }
      if (!best) {
        set_error("neighbourhood blocks of %zu bytes do not fit an SM", lay.bytes);
        return FMGP_EUNSUPPORTED;
      }
    } else {
      nb = active_ctas((const void*)kern_fn, warps * 32, kMixedHead + lay.bytes * warps);
    }
  }
  const size_t smem = kMixedHead + lay.bytes * warps;
  const int64_t need = (a.count + warps - 1) / warps;
  // whole waves of the CTAs the SMs hold at once: no partial last wave
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)num_sms() * std::max(nb, 1) * waves));
  FMGP_CUDA_TRY(ensure_smem((const void*)kern_fn, smem));
  FMGP_LAUNCH(kern_fn<<<blocks, warps * 32, smem, s>>>(a, mx, lay));
  FMGP_CUDA_TRY(cudaGetLastError());
  return mixed_fallback(a, X, dtype, mode, loo, fb_list, fb_count, s);
}

int gather_dot_mixed(const void* X, fmgp_dtype dtype, int64_t n, int d, const int32_t* nbr, int ld,
                     const void* C, int k, int r, const KParams& kp, const fmgp_kernel& kern,
                     const void* Z, int64_t m, const int32_t* nearest, double* Yhat,
                     Workspace& ws, cudaStream_t stream, const float2* Xdf_cached,
                     const int32_t* crow) {
  if (m == 0) return FMGP_OK;
  float2* Xdf = Xdf_cached ? nullptr : ws.get<float2>((size_t)n * d);
  float2* Zdf = ws.get<float2>((size_t)m * d);
  if ((!Xdf && !Xdf_cached) || !Zdf) return FMGP_ENOMEM;
  int rc = Xdf_cached ? FMGP_OK : to_df(X, dtype == FMGP_F64, n * d, Xdf, stream);
  if (Xdf_cached) Xdf = (float2*)Xdf_cached;
  if (!rc) rc = to_df(Z, dtype == FMGP_F64, m * d, Zdf, stream);
  if (rc) return rc;
  const int blocks = ceil_div(m * 32, 256);
  FMGP_LAUNCH(gather_dot_mixed_kernel<<<blocks, 256, 0, stream>>>(
      Xdf, n, d, nbr, ld, (const float2*)C, k, r, make_kparams_df(kp, kern), df_consts(), Zdf, m,
      nearest, Yhat, crow));
  FMGP_CUDA_TRY(cudaGetLastError());
  return FMGP_OK;
}

}  // namespace fmgp

using namespace fmgp;

extern "C" int fmgp_df_eval(int32_t fn, const double* x, int64_t n, double* y, void* stream) {
  clear_error();
  if ((fn != 0 && fn != 1) || n < 0 || (n > 0 && (!x || !y))) {
    set_error("fmgp_df_eval: fn must be 0 or 1, x and y non-NULL");
    return FMGP_EINVAL;
  }
  if (n == 0) return FMGP_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const int blocks = (int)std::min<int64_t>(ceil_div(n, 256), (int64_t)num_sms() * 8);
  FMGP_LAUNCH(df_eval_kernel<<<blocks, 256, 0, s>>>(fn, x, n, y, df_consts()));
  FMGP_CUDA_TRY(cudaGetLastError());
  return FMGP_OK;
}
