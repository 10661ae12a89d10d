// Tensor-core candidate search for the kNN steps (A1, A4) at d >= 16.
//
// 1. pack: X and the queries are rounded to BF16 (rows padded to the tile,
//    features to a multiple of 64), with each row's squared norm of the
//    rounded vector and its rounding error norm ||x - x_bf16||.
// 2. tc_dist_kernel: a tcgen05 GEMM.  A CTA owns 128 queries and sweeps all
//    candidate tiles of 256 rows: a TMA producer thread streams 64-wide
//    feature chunks of both operands (128-byte swizzle) through a 4-stage
//    shared-memory ring, one thread issues tcgen05.mma (kind::f16, BF16 in,
//    FP32 accumulate in tensor memory, M=128 N=256 K=16), and four epilogue
//    warps read the double-buffered accumulator with tcgen05.ld and write the
//    approximate squared distances ||q||^2 + ||x||^2 - 2 q.x to a pass buffer.
// 3. select: one warp per query keeps the L smallest approximate distances.
// 4. rerank: the L candidates get their canonical FP64 keys; the kq best are
//    the result if a certificate holds: every candidate outside the list has
//    approximate distance >= the list's largest, whose rigorous lower bound
//    (BF16 rounding of both vectors, FP32 accumulation) exceeds the kq-th
//    exact key.  Queries without a certificate are redone by the exhaustive
//    exact scan.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <mutex>
#include "knn.cuh"
#include "topk.cuh"

namespace fmgp {
namespace {

constexpr int kTM = 128;        // queries per CTA (TMEM lanes)
constexpr int kTN = 256;        // candidates per tile (accumulator columns)
constexpr int kTK = 64;         // BF16 features per stage (128 bytes: one swizzle row)
constexpr int kStages = 4;
constexpr int kABytes = kTM * kTK * 2;   // 16 KB
constexpr int kBBytes = kTN * kTK * 2;   // 32 KB
constexpr int kStageBytes = kABytes + kBBytes;
constexpr int kTcThreads = 192;          // warps 0-3 epilogue, 4 producer, 5 MMA
constexpr size_t kTcSmem = (size_t)kStages * kStageBytes + 1024 + 256;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t global_timer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// Wait for the phase of `parity` to complete; gives up after ~2 s or when
// another role has raised the abort flag.  Returns false if it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort) {
  const uint32_t addr = smem_u32(bar);
  const uint64_t t0 = global_timer();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done) : "r"(addr), "r"(parity) : "memory");
    if (done) return true;
    if (*abort) return false;
    if (global_timer() - t0 > 2000000000ull) return false;
  }
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1)
      : "memory");
}
// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row
// groups 1024 bytes apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
// Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N = kTN, M = kTM.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTN >> 3) << 17) |
                            ((uint32_t)(kTM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t* v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
      "%28, %29, %30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
        "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
        "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
        "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
        "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Approximate squared distances for query blocks [qb0, qb0 + gridDim.x) against
// every candidate tile.  out row (qb - qb0)*128 + i holds query qb*128 + i.
__global__ void __launch_bounds__(kTcThreads, 1) tc_dist_kernel(
    const __grid_constant__ CUtensorMap tmQ, const __grid_constant__ CUtensorMap tmX,
    const float* __restrict__ qnorm, const float* __restrict__ xnorm, int qb0, int n_tiles,
    int k_chunks, int64_t ld_out, float* __restrict__ out, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + (size_t)kStages * kStageBytes);
  uint64_t* empty = full + kStages;
  uint64_t* tfull = empty + kStages;
  uint64_t* tempty = tfull + 2;
  uint32_t* tmem_slot = (uint32_t*)(tempty + 2);
  volatile int* abort = (volatile int*)(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int qb = qb0 + blockIdx.x;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 4);
    }
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 5) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(2 * kTN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 4) {
    if (lane == 0) {  // TMA producer
      int it = 0;
      for (int t = 0; t < n_tiles && !*abort; ++t) {
        for (int kc = 0; kc < k_chunks; ++kc, ++it) {
          const int s = it % kStages;
          const uint32_t ph = (uint32_t)(it / kStages) & 1u;
          if (!mbar_wait(&empty[s], ph ^ 1u, abort)) { *abort = 1; break; }
          unsigned char* a = smem + (size_t)s * kStageBytes;
          mbar_expect_tx(&full[s], kStageBytes);
          tma_load_2d(a, &tmQ, &full[s], kc * kTK, qb * kTM);
          tma_load_2d(a + kABytes, &tmX, &full[s], kc * kTK, t * kTN);
        }
      }
    }
  } else if (warp == 5) {
    if (lane == 0) {  // MMA issuer
      int it = 0;
      for (int t = 0; t < n_tiles && !*abort; ++t) {
        const int b = t & 1;
        const uint32_t u = (uint32_t)(t >> 1);
        if (!mbar_wait(&tempty[b], (u & 1u) ^ 1u, abort)) { *abort = 1; break; }
        tc_fence_after();
        const uint32_t dacc = tmem + (uint32_t)(b * kTN);
        for (int kc = 0; kc < k_chunks; ++kc, ++it) {
          const int s = it % kStages;
          const uint32_t ph = (uint32_t)(it / kStages) & 1u;
          if (!mbar_wait(&full[s], ph, abort)) { *abort = 1; break; }
          tc_fence_after();
          const uint32_t a = smem_u32(smem + (size_t)s * kStageBytes);
          const uint64_t ad = sw128_desc(a), bd = sw128_desc(a + kABytes);
#pragma unroll
          for (int kk = 0; kk < kTK / 16; ++kk)
            mma_bf16(dacc, ad + (uint64_t)(2 * kk), bd + (uint64_t)(2 * kk),
                     (kc > 0 || kk > 0) ? 1u : 0u);
          mma_commit(&empty[s]);
        }
        if (*abort) break;
        mma_commit(&tfull[b]);
      }
    }
  } else {  // epilogue warps 0-3: TMEM lanes 32*warp .. 32*warp+31
    const int row = warp * 32 + lane;
    const float qn = qnorm[(int64_t)qb * kTM + row];
    float* orow = out + ((int64_t)blockIdx.x * kTM + row) * ld_out;
    for (int t = 0; t < n_tiles; ++t) {
      const int b = t & 1;
      const uint32_t u = (uint32_t)(t >> 1);
      if (!mbar_wait(&tfull[b], u & 1u, abort)) { *abort = 1; break; }
      tc_fence_after();
      for (int c = 0; c < kTN / 32; ++c) {
        uint32_t v[32];
        tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(b * kTN + c * 32), v);
        const int col0 = t * kTN + c * 32;
        const float* xn = xnorm + col0;
        float4* dst = reinterpret_cast<float4*>(orow + col0);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          float4 o;
          o.x = qn + xn[4 * q + 0] - 2.0f * __uint_as_float(v[4 * q + 0]);
          o.y = qn + xn[4 * q + 1] - 2.0f * __uint_as_float(v[4 * q + 1]);
          o.z = qn + xn[4 * q + 2] - 2.0f * __uint_as_float(v[4 * q + 2]);
          o.w = qn + xn[4 * q + 3] - 2.0f * __uint_as_float(v[4 * q + 3]);
          dst[q] = o;
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[b]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (*abort && threadIdx.x == 0) atomicExch(err, 1);
  if (warp == 5) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(2 * kTN));
  }
}

// One warp per row: BF16 copy (padded), squared norm of the rounded row, and
// the norm of its rounding error; running maxima in stats (float bits).
template <typename T>
__global__ void pack_bf16_kernel(const T* __restrict__ X, int64_t rows, int d, int64_t rows_pad,
                                 int d_pad, __nv_bfloat16* __restrict__ Xb,
                                 float* __restrict__ norm2, float* __restrict__ delta,
                                 unsigned int* stats) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= rows_pad) return;
  float n2 = 0.f, e2 = 0.f;
  for (int j = lane; j < d_pad; j += 32) {
    float xb = 0.f;
    if (w < rows && j < d) {
      const double v = (double)X[w * d + j];
      const __nv_bfloat16 h = __double2bfloat16(v);
      xb = __bfloat162float(h);
      Xb[w * d_pad + j] = h;
      const float e = (float)(v - (double)xb);
      e2 = fmaf(e, e, e2);
    } else {
      Xb[w * d_pad + j] = __float2bfloat16(0.f);
    }
    n2 = fmaf(xb, xb, n2);
  }
  for (int o = 16; o; o >>= 1) {
    n2 += __shfl_xor_sync(kFull, n2, o);
    e2 += __shfl_xor_sync(kFull, e2, o);
  }
  if (lane == 0) {
    // generous rounding: the bound only needs to be an upper bound
    const float dl = sqrtf(e2) * 1.0001f + 1e-30f;
    norm2[w] = n2;
    delta[w] = dl;
    if (w < rows) {
      atomicMax(&stats[0], __float_as_uint(sqrtf(n2) * 1.0001f));
      atomicMax(&stats[1], __float_as_uint(dl));
    }
  }
}

// One warp per query row of the pass buffer: the L smallest approximate
// distances (negative values clamp to 0; ties by index).
template <int S>
__global__ void __launch_bounds__(256) select_kernel(const float* __restrict__ Dp, int64_t ld,
                                                     int64_t q0, int64_t rows, int64_t n, int L,
                                                     int exclude_self, int32_t* __restrict__ cand,
                                                     float* __restrict__ dL) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= rows) return;
  const int64_t q = q0 + w;
  const float* row = Dp + w * ld;
  WarpTopK<S> top;
  top.init(L);
  for (int64_t base = 0; base < n; base += 32) {
    const int64_t j = base + lane;
    unsigned long long ck = ~0ull;
    int ci = INT_MAX;
    if (j < n && !(exclude_self && j == q)) {
      // keys are the FP32 bit patterns of non-negative values (ordered like integers)
      const unsigned long long v = (unsigned long long)__float_as_uint(fmaxf(row[j], 0.0f));
      if (v <= top.tk) {
        ck = v;
        ci = (int)j;
      }
    }
    top.offer(ck, ci, lane);
  }
  top.store(L, lane, cand + q * L, nullptr);
  // largest approximate distance in the list (position L-1); +inf if not full
  if (lane == 0)
    dL[q] = top.full() ? __uint_as_float((unsigned int)top.tk) : __int_as_float(0x7f800000);
}

// Exact re-rank with certificate; uncertified queries go to the fallback list.
template <typename T, int S>
__global__ void __launch_bounds__(256) rerank_kernel(
    const T* __restrict__ X, const T* __restrict__ Q, int d, int64_t m, int L, int kq,
    const int32_t* __restrict__ cand, const float* __restrict__ dL,
    const float* __restrict__ qnorm2, const float* __restrict__ qdelta,
    const unsigned int* __restrict__ xstats, const unsigned int* __restrict__ qstats,
    const int* __restrict__ err, int32_t* __restrict__ idx_out, double* __restrict__ key_out,
    int* fb_list, int* fb_count) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= m) return;
  const T* qr = Q + w * d;
  WarpTopK<S> top;
  top.init(kq);
  for (int base = 0; base < L; base += 32) {
    const int a = base + lane;
    unsigned long long ck = ~0ull;
    int ci = INT_MAX;
    if (a < L) {
      const int j = cand[w * L + a];
      if (j >= 0 && j != INT_MAX) {
        const T* xr = X + (int64_t)j * d;
        double t = __dsub_rn((double)qr[0], (double)xr[0]);
        double s = __dmul_rn(t, t);
        for (int p = 1; p < d; ++p) {
          t = __dsub_rn((double)qr[p], (double)xr[p]);
          s = __dadd_rn(s, __dmul_rn(t, t));
        }
        ck = dbits(s);
        ci = j;
      }
    }
    top.offer(ck, ci, lane);
  }
  // certificate: lower bound of the true distance of any candidate outside
  // the list (approximate distance >= dL) must exceed the kq-th exact key.
  const float xmaxn = __uint_as_float(xstats[0]), xdel = __uint_as_float(xstats[1]);
  const float qn = sqrtf(qnorm2[w]) * 1.0001f;
  const float u = 5.9604645e-8f;
  const float E = 2.0f * d * 4.0f * u * qn * xmaxn + d * u * (qn * qn + xmaxn * xmaxn) + 1e-30f;
  const float Dl = dL[w];
  float lo = sqrtf(fmaxf(Dl - E, 0.0f)) - qdelta[w] - xdel;
  lo = fmaxf(lo, 0.0f);
  lo = lo * lo * (1.0f - 1e-5f);
  const float kth_up = key_bits_to_float_up(top.tk);
  // a distance pass that gave up (err) certifies nothing: every query is redone
  const bool cert = (*err == 0) && top.full() && (Dl == __int_as_float(0x7f800000) || lo > kth_up);
  if (cert) {
    top.store(kq, lane, idx_out + w * kq, key_out ? key_out + w * kq : nullptr);
  } else if (lane == 0) {
    const int pos = atomicAdd(fb_count, 1);
    fb_list[pos] = (int)w;
  }
  (void)qstats;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, []() {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  });
  return fn;
}

int make_map(CUtensorMap* map, const void* base, int64_t rows, int d_pad, int box_rows) {
  auto fn = encode_fn();
  if (!fn) {
    set_error("cuTensorMapEncodeTiled is unavailable");
    return FMGP_ECUDA;
  }
  cuuint64_t dims[2] = {(cuuint64_t)d_pad, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)d_pad * 2};
  cuuint32_t box[2] = {(cuuint32_t)kTK, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides,
                  box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
    return FMGP_ECUDA;
  }
  return FMGP_OK;
}

template <typename T>
int pack(const T* X, int64_t rows, int d, int64_t rows_pad, int d_pad, Workspace& ws,
         cudaStream_t s, __nv_bfloat16** Xb, float** n2, float** dl, unsigned int** stats) {
  *Xb = ws.get<__nv_bfloat16>((size_t)rows_pad * d_pad);
  *n2 = ws.get<float>(rows_pad);
  *dl = ws.get<float>(rows_pad);
  *stats = ws.get<unsigned int>(2);
  if (!*Xb || !*n2 || !*dl || !*stats) return FMGP_ENOMEM;
  FMGP_CUDA_TRY(cudaMemsetAsync(*stats, 0, 2 * sizeof(unsigned int), s));
  FMGP_LAUNCH(pack_bf16_kernel<T><<<ceil_div(rows_pad * 32, 256), 256, 0, s>>>(
      X, rows, d, rows_pad, d_pad, *Xb, *n2, *dl, *stats));
  FMGP_CUDA_TRY(cudaGetLastError());
  return FMGP_OK;
}

template <typename T>
int tc_knn_t(const T* X, int64_t n, int d, const T* Q, int64_t m, int kq, bool self,
             int32_t* idx_out, double* key_out, Workspace& ws, cudaStream_t s) {
  const int L = std::min(128, (std::max(4 * kq, 32) + 31) / 32 * 32);
  const int S = L / 32;
  const int d_pad = (d + kTK - 1) / kTK * kTK;
  const int64_t n_pad = (n + kTN - 1) / kTN * kTN;
  const int64_t m_pad = (m + kTM - 1) / kTM * kTM;
  __nv_bfloat16 *Xb, *Qb;
  float *xn2, *xdl, *qn2, *qdl;
  unsigned int *xst, *qst;
  int rc = pack<T>(X, n, d, n_pad, d_pad, ws, s, &Xb, &xn2, &xdl, &xst);
  if (rc) return rc;
  if (self && m_pad <= n_pad) {
    Qb = Xb; qn2 = xn2; qdl = xdl; qst = xst;
  } else {
    rc = pack<T>(Q, m, d, m_pad, d_pad, ws, s, &Qb, &qn2, &qdl, &qst);
    if (rc) return rc;
  }
  CUtensorMap tmQ, tmX;
  rc = make_map(&tmQ, Qb, self && m_pad <= n_pad ? n_pad : m_pad, d_pad, kTM);
  if (!rc) rc = make_map(&tmX, Xb, n_pad, d_pad, kTN);
  if (rc) return rc;
  // pass buffer: at most ~1 GB of approximate distances
  int64_t qblocks = m_pad / kTM;
  int64_t pass_blocks = std::max<int64_t>(1, (int64_t)(1ll << 30) / (n_pad * 4 * kTM));
  pass_blocks = std::min(pass_blocks, qblocks);
  float* Dp = ws.get<float>((size_t)pass_blocks * kTM * n_pad);
  int32_t* cand = ws.get<int32_t>((size_t)m * L);
  float* dL = ws.get<float>(m);
  int* err = ws.get<int>(1);
  int* fb_list = ws.get<int>(m);
  int* fb_count = ws.get<int>(1);
  if (!Dp || !cand || !dL || !err || !fb_list || !fb_count) return FMGP_ENOMEM;
  FMGP_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), s));
  FMGP_CUDA_TRY(cudaMemsetAsync(fb_count, 0, sizeof(int), s));
  FMGP_CUDA_TRY(cudaFuncSetAttribute(tc_dist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kTcSmem));
  const int n_tiles = (int)(n_pad / kTN), k_chunks = d_pad / kTK;
  for (int64_t qb0 = 0; qb0 < qblocks; qb0 += pass_blocks) {
    const int nb = (int)std::min(pass_blocks, qblocks - qb0);
    FMGP_LAUNCH(tc_dist_kernel<<<nb, kTcThreads, kTcSmem, s>>>(
        tmQ, tmX, qn2, xn2, (int)qb0, n_tiles, k_chunks, n_pad, Dp, err));
    const int64_t q0 = qb0 * kTM;
    const int64_t rows = std::min<int64_t>((int64_t)nb * kTM, m - q0);
    if (rows > 0) {
      const int blocks = ceil_div(rows * 32, 256);
      switch (S) {
        case 1: FMGP_LAUNCH(select_kernel<1><<<blocks, 256, 0, s>>>(Dp, n_pad, q0, rows, n, L, self, cand, dL)); break;
        case 2: FMGP_LAUNCH(select_kernel<2><<<blocks, 256, 0, s>>>(Dp, n_pad, q0, rows, n, L, self, cand, dL)); break;
        case 3: FMGP_LAUNCH(select_kernel<3><<<blocks, 256, 0, s>>>(Dp, n_pad, q0, rows, n, L, self, cand, dL)); break;
        default: FMGP_LAUNCH(select_kernel<4><<<blocks, 256, 0, s>>>(Dp, n_pad, q0, rows, n, L, self, cand, dL)); break;
      }
    }
  }
  FMGP_CUDA_TRY(cudaGetLastError());
  const int blocks = ceil_div(m * 32, 256);
  const int KS = (kq + 31) / 32;
  switch (KS) {
    case 1: FMGP_LAUNCH((rerank_kernel<T, 1><<<blocks, 256, 0, s>>>(X, Q, d, m, L, kq, cand, dL, qn2, qdl, xst, qst, err, idx_out, key_out, fb_list, fb_count))); break;
    case 2: FMGP_LAUNCH((rerank_kernel<T, 2><<<blocks, 256, 0, s>>>(X, Q, d, m, L, kq, cand, dL, qn2, qdl, xst, qst, err, idx_out, key_out, fb_list, fb_count))); break;
    case 3: FMGP_LAUNCH((rerank_kernel<T, 3><<<blocks, 256, 0, s>>>(X, Q, d, m, L, kq, cand, dL, qn2, qdl, xst, qst, err, idx_out, key_out, fb_list, fb_count))); break;
    default: FMGP_LAUNCH((rerank_kernel<T, 4><<<blocks, 256, 0, s>>>(X, Q, d, m, L, kq, cand, dL, qn2, qdl, xst, qst, err, idx_out, key_out, fb_list, fb_count))); break;
  }
  FMGP_CUDA_TRY(cudaGetLastError());
  diag_record_tc(fb_count, s);
  // exhaustive exact scan for uncertified queries
  return knn_brute_list(X, sizeof(T) == 8 ? FMGP_F64 : FMGP_F32, n, d, Q, m, kq, self, fb_list,
                        fb_count, idx_out, key_out, ws, s);
}

}  // namespace

bool tc_knn_eligible(int64_t n, int d, int64_t m, int kq) {
  const TuneParams& tp = tune_params();
  if (!tp.use_tensor_cores) return false;
  const int L = std::min(128, (std::max(4 * kq, 32) + 31) / 32 * 32);
  return d >= 16 && kq <= 96 && n > 2 * L && n >= 4096 && m >= 128;
}

int tc_knn(const void* X, fmgp_dtype dtype, int64_t n, int d, const void* Q, int64_t m, int kq,
           bool self, int32_t* idx_out, double* key_out, Workspace& ws, cudaStream_t s) {
  if (dtype == FMGP_F64)
    return tc_knn_t<double>((const double*)X, n, d, (const double*)Q, m, kq, self, idx_out,
                            key_out, ws, s);
  return tc_knn_t<float>((const float*)X, n, d, (const float*)Q, m, kq, self, idx_out, key_out,
                         ws, s);
}

}  // namespace fmgp
