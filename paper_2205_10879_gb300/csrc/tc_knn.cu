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
//    warps read the double-buffered accumulator with tcgen05.ld and form the
//    approximate squared distances ||q||^2 + ||x||^2 - 2 q.x.  For kq <= 32
//    each epilogue thread (one query) keeps the R smallest of its CTA's
//    candidate range in registers (the fused form: nothing but R candidates
//    per query and range reaches HBM); otherwise the distances go to a pass
//    buffer.
// 3. select: one warp per query keeps the L smallest approximate distances
//    (of the per-range lists, or of the pass buffer).  With per-range lists,
//    every candidate a range dropped is no closer than that range's R-th, so
//    the smallest such R-th joins the list's L-th in the certificate bound.
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
#include "df.cuh"

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
// fused selection: a second epilogue warpgroup (warps 6-9) takes the upper
// half of each tile's columns, so two warps per SM sub-partition hide the
// latency of the TMEM loads and the per-chunk filtering
constexpr int kTcSelThreads = 320;
// longest candidate list of the re-rank (2 kq for kq = 160)
constexpr int kMaxTcList = 320;
constexpr int kTcEpiWarps(int R) { return R > 0 ? 8 : 4; }
constexpr size_t kTcSmem = (size_t)kStages * kStageBytes + 1024 + 256;
// fused selection: per epilogue thread a 32-float row of the current chunk's
// values, written as 16-byte slots swizzled by the row's low 3 bits (slot
// q at q ^ (row & 7): the 8 rows of a store phase hit distinct banks) and
// read back at the bits the thread pops
constexpr int kScrStride = 32;
constexpr size_t kTcSelSmem = kTcSmem + (size_t)2 * kTM * kScrStride * sizeof(float);
static_assert(kTcSelSmem <= 232448, "fused tensor-core kernel exceeds 227 KB of shared memory");

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
// Limit of the bounded waits after an abort (the drains below), in ns.
constexpr uint64_t kDrainWaitNs = 2000000000ull;

// Wait for the phase of `parity` to complete; gives up after limit_ns or when
// another role has raised the abort flag.  Returns false if it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort,
                                          uint64_t limit_ns = kDrainWaitNs) {
  const uint32_t addr = smem_u32(bar);
  const uint64_t t0 = global_timer();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done) : "r"(addr), "r"(parity) : "memory");
    if (done) return true;
    if (abort && *abort) return false;
    if (global_timer() - t0 > limit_ns) return false;
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
// Issue a 32x32b.x32 TMEM load without waiting: v must not be read before
// tmem_wait_regs(v).
__device__ __forceinline__ void tmem_ld32_issue(uint32_t taddr, uint32_t (&v)[32]) {
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
}
// Wait for the thread's TMEM loads; v passes through the wait so that no use
// of it is moved above it.
__device__ __forceinline__ void tmem_wait_regs(uint32_t (&v)[32]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]),
                 "+r"(v[6]), "+r"(v[7]), "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]),
                 "+r"(v[12]), "+r"(v[13]), "+r"(v[14]), "+r"(v[15]), "+r"(v[16]), "+r"(v[17]),
                 "+r"(v[18]), "+r"(v[19]), "+r"(v[20]), "+r"(v[21]), "+r"(v[22]), "+r"(v[23]),
                 "+r"(v[24]), "+r"(v[25]), "+r"(v[26]), "+r"(v[27]), "+r"(v[28]), "+r"(v[29]),
                 "+r"(v[30]), "+r"(v[31])
               :
               : "memory");
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

// Insert (dv, col) into the ascending list bk/bi of R entries (static
// indices only, so the list stays in registers).  Equal keys keep their
// arrival order: columns arrive in increasing order, so ties go to the lower
// index.
template <int R>
__device__ __forceinline__ void sorted_insert(float (&bk)[R], int (&bi)[R], float dv, int col) {
#pragma unroll
  for (int s = R - 1; s > 0; --s) {
    const bool a = dv < bk[s - 1];
    const bool b = dv < bk[s];
    bi[s] = a ? bi[s - 1] : (b ? col : bi[s]);
    bk[s] = a ? bk[s - 1] : (b ? dv : bk[s]);
  }
  if (dv < bk[0]) { bk[0] = dv; bi[0] = col; }
}

// Fused selection of one 32-column chunk (TMEM values v, column norms xv):
// w = ||x||^2 - 2 q.x, the lane's hits below its R-th value as a bit mask
// (sign of w - threshold shifted in by a funnel shift per column), then each
// lane pops its own hits into its sorted list; the warp pays for its busiest
// lane, not for the union of all lanes' hits.
template <int R>
__device__ __forceinline__ void select_chunk(const uint32_t (&v)[32], const float4 (&xv)[8],
                                             float (&bk)[R], int (&bi)[R], float* scr, int sw,
                                             int64_t gcol, int64_t n_valid, int self,
                                             int64_t qrow) {
  float4* scr4 = reinterpret_cast<float4*>(scr);
  const float thr = bk[R - 1];
  float w[32];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const float4 x = xv[q];
    float4 o;
    o.x = w[4 * q + 0] = fmaf(-2.0f, __uint_as_float(v[4 * q + 0]), x.x);
    o.y = w[4 * q + 1] = fmaf(-2.0f, __uint_as_float(v[4 * q + 1]), x.y);
    o.z = w[4 * q + 2] = fmaf(-2.0f, __uint_as_float(v[4 * q + 2]), x.z);
    o.w = w[4 * q + 3] = fmaf(-2.0f, __uint_as_float(v[4 * q + 3]), x.w);
    scr4[q ^ sw] = o;
  }
  // bit j = (w_j < thr) = sign bit of w_j - thr (thr = +inf gives -inf:
  // set), shifted in from the top column of each 8-column group down
  unsigned int g8[4];
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    unsigned int mg = 0;
#pragma unroll
    for (int e = 7; e >= 0; --e) mg = __funnelshift_l(__float_as_uint(w[8 * g + e] - thr), mg, 1);
    g8[g] = mg;
  }
  unsigned int mask = g8[0] | (g8[1] << 8) | (g8[2] << 16) | (g8[3] << 24);
  const int64_t lim = n_valid - gcol;
  if (lim < 32) mask &= lim <= 0 ? 0u : ((1u << lim) - 1u);
  if (self) {
    const int64_t sj = qrow - gcol;
    if (sj >= 0 && sj < 32) mask &= ~(1u << sj);
  }
  while (__any_sync(kFull, mask != 0u)) {
    if (mask) {
      const int j = __ffs(mask) - 1;
      mask &= mask - 1u;
      const float wj = scr[(((j >> 2) ^ sw) << 2) | (j & 3)];
      if (wj < bk[R - 1]) sorted_insert<R>(bk, bi, wj, (int)(gcol + j));
    }
  }
  __syncwarp();
}

__device__ __forceinline__ void load_norms(const float* xnorm, int64_t gcol, float4 (&xv)[8]) {
  const float4* xn4 = reinterpret_cast<const float4*>(xnorm + gcol);
#pragma unroll
  for (int q = 0; q < 8; ++q) xv[q] = xn4[q];
}

// Approximate squared distances of query block qb0 + blockIdx.x against
// candidate tiles tile0 + blockIdx.y*tpc .. (at most tpc tiles, not past
// tile_end).  Query q below is counted from the first query of block qb0.
// R == 0: out row q (query q), column (t - tile0)*256 + j holds candidate
//   t*256 + j.
// R > 0: for each half h of the tile columns, the R smallest (clamped at 0;
//   candidates >= n_valid and, with self, the query itself left out) as an
//   ascending list at pkey/pidx[(q * 2 gridDim.y + 2 blockIdx.y + h) * R ..],
//   INT_MAX past the end.  The thread ranks w = ||x||^2 - 2 q.x (FP32) and
//   reports ||q||^2 + w: the sum is monotone in w, so the kept set and the
//   range's R-th value are those of the reported distances.
template <int R>
__global__ void __launch_bounds__(R > 0 ? kTcSelThreads : kTcThreads, 1) tc_dist_kernel(
    const __grid_constant__ CUtensorMap tmQ, const __grid_constant__ CUtensorMap tmX,
    const float* __restrict__ qnorm, const float* __restrict__ xnorm, int qb0, int tile0,
    int tile_end, int tpc, int k_chunks, int64_t ld_out, float* __restrict__ out,
    int64_t n_valid, int self, float* __restrict__ pkey, int32_t* __restrict__ pidx,
    int* __restrict__ err, uint64_t wait_ns) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + (size_t)kStages * kStageBytes);
  uint64_t* empty = full + kStages;
  uint64_t* tfull = empty + kStages;
  uint64_t* tempty = tfull + 2;
  uint32_t* tmem_slot = (uint32_t*)(tempty + 2);
  volatile int* abort = (volatile int*)(tmem_slot + 1);
  uint64_t* drain = (uint64_t*)(tmem_slot + 2);  // MMA completion after an abort
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int qb = qb0 + (int)blockIdx.x;
  const int t_first = tile0 + blockIdx.y * tpc;
  const int n_tiles = max(0, min(tpc, tile_end - t_first));
  int it_issued = 0;  // stages the producer filled (its thread only)

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], kTcEpiWarps(R));
    }
    mbar_init(drain, 1);
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
          if (!mbar_wait(&empty[s], ph ^ 1u, abort, wait_ns)) { *abort = 1; break; }
          unsigned char* a = smem + (size_t)s * kStageBytes;
          mbar_expect_tx(&full[s], kStageBytes);
          tma_load_2d(a, &tmQ, &full[s], kc * kTK, qb * kTM);
          tma_load_2d(a + kABytes, &tmX, &full[s], kc * kTK, (t_first + t) * kTN);
        }
      }
      it_issued = it;
    }
  } else if (warp == 5) {
    if (lane == 0) {  // MMA issuer
      int it = 0;
      for (int t = 0; t < n_tiles && !*abort; ++t) {
        const int b = t & 1;
        const uint32_t u = (uint32_t)(t >> 1);
        if (!mbar_wait(&tempty[b], (u & 1u) ^ 1u, abort, wait_ns)) { *abort = 1; break; }
        tc_fence_after();
        const uint32_t dacc = tmem + (uint32_t)(b * kTN);
        for (int kc = 0; kc < k_chunks; ++kc, ++it) {
          const int s = it % kStages;
          const uint32_t ph = (uint32_t)(it / kStages) & 1u;
          if (!mbar_wait(&full[s], ph, abort, wait_ns)) { *abort = 1; break; }
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
  } else if constexpr (R > 0) {  // epilogue warps 0-3 and 6-9, fused selection
    // TMEM lane quarter of a warp = its index mod 4; half h of the columns
    const int quarter = warp & 3, h = warp >= 6 ? 1 : 0;
    const int row = quarter * 32 + lane;
    const int64_t qrow = (int64_t)qb * kTM + row;
    const float qn = qnorm[qrow];
    float* scr = reinterpret_cast<float*>(smem + (size_t)kStages * kStageBytes + 256) +
                 (h * kTM + row) * kScrStride;
    const int sw = row & 7;
    float bk[R];  // ascending w values of the kept candidates
    int bi[R];
#pragma unroll
    for (int s = 0; s < R; ++s) { bk[s] = __int_as_float(0x7f800000); bi[s] = INT_MAX; }
    for (int t = 0; t < n_tiles; ++t) {
      const int b = t & 1;
      const uint32_t u = (uint32_t)(t >> 1);
      const bool ok = mbar_wait(&tfull[b], u & 1u, abort, wait_ns);
      if (!__all_sync(kFull, ok)) { *abort = 1; break; }
      tc_fence_after();
      const uint32_t tbase = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * kTN);
      const int c0 = h * (kTN / 64);  // this warpgroup's 4 chunks: c0 .. c0 + 3
      const int64_t g0 = (int64_t)(t_first + t) * kTN + c0 * 32;
      if constexpr (R <= 16) {
        // software pipelined: chunk c+1's TMEM load and norms are in flight
        // while chunk c is filtered
        uint32_t va[32], vb[32];
        float4 xa[8], xb[8];
        load_norms(xnorm, g0, xa);
        __syncwarp();
        tmem_ld32_issue(tbase + (uint32_t)(c0 * 32), va);
        tmem_wait_regs(va);
        load_norms(xnorm, g0 + 32, xb);
        tmem_ld32_issue(tbase + (uint32_t)(c0 * 32 + 32), vb);
        select_chunk<R>(va, xa, bk, bi, scr, sw, g0, n_valid, self, qrow);
        tmem_wait_regs(vb);
        load_norms(xnorm, g0 + 64, xa);
        tmem_ld32_issue(tbase + (uint32_t)(c0 * 32 + 64), va);
        select_chunk<R>(vb, xb, bk, bi, scr, sw, g0 + 32, n_valid, self, qrow);
        tmem_wait_regs(va);
        load_norms(xnorm, g0 + 96, xb);
        tmem_ld32_issue(tbase + (uint32_t)(c0 * 32 + 96), vb);
        select_chunk<R>(va, xa, bk, bi, scr, sw, g0 + 64, n_valid, self, qrow);
        tmem_wait_regs(vb);
        select_chunk<R>(vb, xb, bk, bi, scr, sw, g0 + 96, n_valid, self, qrow);
      } else {
        // R = 32: the list leaves no registers for a second chunk in flight
        for (int c = 0; c < kTN / 64; ++c) {
          uint32_t v[32];
          float4 xv[8];
          __syncwarp();
          tmem_ld32_issue(tbase + (uint32_t)((c0 + c) * 32), v);
          tmem_wait_regs(v);
          load_norms(xnorm, g0 + c * 32, xv);
          select_chunk<R>(v, xv, bk, bi, scr, sw, g0 + c * 32, n_valid, self, qrow);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[b]);
    }
    const int64_t seg = (qrow - (int64_t)qb0 * kTM) * 2 * gridDim.y + 2 * blockIdx.y + h;
    float* okey = pkey + seg * R;
    int32_t* oidx = pidx + seg * R;
#pragma unroll
    for (int s = 0; s < R; ++s) {
      okey[s] = bi[s] == INT_MAX ? __int_as_float(0x7f800000) : fmaxf(qn + bk[s], 0.0f);
      oidx[s] = bi[s];
    }
  } else {  // epilogue warps 0-3: TMEM lanes 32*warp .. 32*warp+31
    const int row = warp * 32 + lane;
    const float qn = qnorm[(int64_t)qb * kTM + row];
    float* orow = out + ((int64_t)(qb - qb0) * kTM + row) * ld_out;
    for (int t = 0; t < n_tiles; ++t) {
      const int b = t & 1;
      const uint32_t u = (uint32_t)(t >> 1);
      if (!mbar_wait(&tfull[b], u & 1u, abort, wait_ns)) { *abort = 1; break; }
      tc_fence_after();
      for (int c = 0; c < kTN / 32; ++c) {
        uint32_t v[32];
        tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(b * kTN + c * 32), v);
        const int gcol = (t_first + t) * kTN + c * 32;
        const float* xn = xnorm + gcol;
        float4* dst = reinterpret_cast<float4*>(orow + (gcol - tile0 * kTN));
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
  const bool aborted = *abort != 0;
  if (aborted && threadIdx.x == 0) atomicExch(err, 1);
  // After an abort, wait (bounded, whatever the flag) for this CTA's own
  // asynchronous work: the producer for the copies it issued, so none lands in
  // shared memory after the CTA is gone; the MMA thread for its MMAs, before
  // the accumulator is freed.
  if (aborted && warp == 4 && lane == 0) {
    for (int j = max(0, it_issued - kStages); j < it_issued; ++j)
      mbar_wait(&full[j % kStages], (uint32_t)(j / kStages) & 1u, nullptr);
  }
  if (warp == 5) {
    if (aborted && lane == 0) {
      mma_commit(drain);
      mbar_wait(drain, 0u, nullptr);
    }
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(2 * kTN));
  }
}

// One warp per row (grid-strided): BF16 copy (padded), squared norm of the
// rounded row, and the norm of its rounding error; the running maxima over
// the real rows go to stats (float bits), one pair of atomics per CTA.
constexpr int kPackThreads = 256;
template <typename T>
__global__ void __launch_bounds__(kPackThreads) pack_bf16_kernel(
    const T* __restrict__ X, int64_t rows, int d, int64_t rows_pad, int d_pad,
    __nv_bfloat16* __restrict__ Xb, float* __restrict__ norm2, float* __restrict__ delta,
    unsigned int* stats) {
  __shared__ float red[2][kPackThreads / 32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t nwarps = (int64_t)gridDim.x * (kPackThreads / 32);
  float mnorm = 0.f, mdel = 0.f;
  for (int64_t w = (int64_t)blockIdx.x * (kPackThreads / 32) + wib; w < rows_pad; w += nwarps) {
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
    // generous rounding: the bound only needs to be an upper bound
    const float dl = sqrtf(e2) * 1.0001f + 1e-30f;
    if (lane == 0) {
      norm2[w] = n2;
      delta[w] = dl;
    }
    if (w < rows) {
      mnorm = fmaxf(mnorm, sqrtf(n2) * 1.0001f);
      mdel = fmaxf(mdel, dl);
    }
  }
  if (lane == 0) {
    red[0][wib] = mnorm;
    red[1][wib] = mdel;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < kPackThreads / 32; ++i) {
      mnorm = fmaxf(mnorm, red[0][i]);
      mdel = fmaxf(mdel, red[1][i]);
    }
    atomicMax(&stats[0], __float_as_uint(mnorm));
    atomicMax(&stats[1], __float_as_uint(mdel));
  }
}

// One warp per query: merge the chunk of approximate distances (columns
// col0 .. col0+ncols of the global candidate range, row q of Dc) into the
// query's running list of the L smallest (FP32 keys as bits, ties by index;
// negative values clamp to 0).  first = no previous list.
template <int S>
__global__ void __launch_bounds__(256) select_merge_kernel(
    const float* __restrict__ Dc, int64_t ld, int64_t m, int64_t col0, int64_t ncols, int64_t n,
    int L, int exclude_self, int first, int32_t* __restrict__ cand, float* __restrict__ ckey,
    float* __restrict__ dL) {
  const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (q >= m) return;
  WarpTopK32<S> top;
  top.init(L);
  if (!first) {
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const int g = lane * S + s;
      const int j = g < L ? cand[q * L + g] : INT_MAX;
      top.k[s] = j == INT_MAX ? ~0u : __float_as_uint(ckey[q * L + g]);
      top.i[s] = j;
    }
    top.refresh_threshold();
  }
  const float* row = Dc + q * ld;
  const int64_t cols = min(ncols, n - col0);
  for (int64_t base = 0; base < cols; base += 128) {
    float v4[4];
    const int64_t c = base + 4 * lane;
    if (c + 3 < cols) {
      const float4 f = *reinterpret_cast<const float4*>(row + c);
      v4[0] = f.x; v4[1] = f.y; v4[2] = f.z; v4[3] = f.w;
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) v4[e] = c + e < cols ? row[c + e] : 0.f;
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int64_t j = col0 + c + e;
      unsigned int ck = ~0u;
      int ci = INT_MAX;
      if (c + e < cols && !(exclude_self && j == q)) {
        const unsigned int v = __float_as_uint(fmaxf(v4[e], 0.0f));
        if (v <= top.tk) { ck = v; ci = (int)j; }
      }
      top.offer(ck, ci, lane);
    }
  }
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int g = lane * S + s;
    if (g < L) {
      cand[q * L + g] = top.i[s];
      ckey[q * L + g] = top.i[s] == INT_MAX ? 0.f : __uint_as_float(top.k[s]);
    }
  }
  // largest approximate distance in the list (position L-1); +inf if not full
  if (lane == 0)
    dL[q] = top.full() ? __uint_as_float(top.tk) : __int_as_float(0x7f800000);
}

// One warp per query: the L smallest of the per-range lists of the fused
// distance pass (nseg ranges of R ascending entries each, INT_MAX past a
// range's end).  dL = the smaller of the list's L-th key (+inf if not full)
// and the smallest R-th key of a full range: every candidate outside the
// list is at least that far.
template <int S>
__global__ void __launch_bounds__(256) select_parts_kernel(
    const float* __restrict__ pkey, const int32_t* __restrict__ pidx, int64_t m, int nseg, int R,
    int L, int32_t* __restrict__ cand, float* __restrict__ ckey, float* __restrict__ dL) {
  const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (q >= m) return;
  WarpTopK32<S> top;
  top.init(L);
  const int tot = nseg * R;
  const float* kq_ = pkey + q * tot;
  const int32_t* iq = pidx + q * tot;
  float bound = __int_as_float(0x7f800000);
  for (int base = 0; base < tot; base += 32) {
    const int e = base + lane;
    unsigned int ck = ~0u;
    int ci = INT_MAX;
    if (e < tot) {
      const int j = iq[e];
      if (j != INT_MAX) {
        const float v = kq_[e];
        ck = __float_as_uint(v);
        ci = j;
        if (e % R == R - 1) bound = fminf(bound, v);
      }
    }
    top.offer(ck, ci, lane);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) bound = fminf(bound, __shfl_xor_sync(kFull, bound, o));
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int g = lane * S + s;
    if (g < L) {
      cand[q * L + g] = top.i[s];
      ckey[q * L + g] = top.i[s] == INT_MAX ? 0.f : __uint_as_float(top.k[s]);
    }
  }
  if (lane == 0)
    dL[q] = fminf(bound, top.full() ? __uint_as_float(top.tk) : __int_as_float(0x7f800000));
}

// As select_parts_kernel for at most 32*PER entries per query, without a
// running list: the L-th smallest key T is found by bisection on the key
// bits (warp counts of keys <= mid), the members are the keys < T and, of
// those equal to T, the lowest indices; they are written unordered (the
// re-rank needs the set, not its order).
template <int PER>
__global__ void __launch_bounds__(256) select_parts_bisect_kernel(
    const float* __restrict__ pkey, const int32_t* __restrict__ pidx, int64_t m, int nseg, int R,
    int L, int32_t* __restrict__ cand, float* __restrict__ ckey, float* __restrict__ dL) {
  const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (q >= m) return;
  const int tot = nseg * R;
  const float* kq_ = pkey + q * tot;
  const int32_t* iq = pidx + q * tot;
  unsigned int kk[PER];
  int ii[PER];
  float bound = __int_as_float(0x7f800000);
  int nvalid = 0;
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int e = p * 32 + lane;
    kk[p] = ~0u;
    ii[p] = INT_MAX;
    if (e < tot) {
      const int j = iq[e];
      if (j != INT_MAX) {
        const float v = kq_[e];
        kk[p] = __float_as_uint(v) & 0x7fffffffu;  // v >= 0; -0 counts as +0
        ii[p] = j;
        ++nvalid;
        if (e % R == R - 1) bound = fminf(bound, v);
      }
    }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) bound = fminf(bound, __shfl_xor_sync(kFull, bound, o));
  nvalid = __reduce_add_sync(kFull, (unsigned)nvalid);
  const bool full = nvalid >= L;
  // T = smallest key with at least L keys <= T (all valid keys if not full)
  unsigned int T = 0x7f800000u;
  if (full) {
    unsigned int lo = 0, hi = 0x7f800000u;
    while (lo < hi) {
      const unsigned int mid = lo + ((hi - lo) >> 1);
      int c = 0;
#pragma unroll
      for (int p = 0; p < PER; ++p) c += kk[p] <= mid ? 1 : 0;
      if ((int)__reduce_add_sync(kFull, (unsigned)c) >= L) hi = mid; else lo = mid + 1;
    }
    T = lo;
  }
  bool mem[PER];
  int nlt = 0;
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    mem[p] = full ? kk[p] < T : ii[p] != INT_MAX;
    nlt += mem[p] ? 1 : 0;
  }
  if (full) {
    // keys equal to T by increasing index until the list holds L
    int need = L - (int)__reduce_add_sync(kFull, (unsigned)nlt);
    while (need > 0) {
      unsigned int best = ~0u;
#pragma unroll
      for (int p = 0; p < PER; ++p)
        if (kk[p] == T && !mem[p]) best = min(best, (unsigned int)ii[p]);
      best = __reduce_min_sync(kFull, best);
#pragma unroll
      for (int p = 0; p < PER; ++p)
        if (kk[p] == T && (unsigned int)ii[p] == best) mem[p] = true;
      --need;
    }
  }
  int base = 0;
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const unsigned int bal = __ballot_sync(kFull, mem[p]);
    if (mem[p]) {
      const int pos = base + __popc(bal & ((1u << lane) - 1u));
      cand[q * L + pos] = ii[p];
      ckey[q * L + pos] = __uint_as_float(kk[p]);
    }
    base += __popc(bal);
  }
  for (int g = base + lane; g < L; g += 32) cand[q * L + g] = INT_MAX;
  if (lane == 0)
    dL[q] = fminf(bound, full ? __uint_as_float(T) : __int_as_float(0x7f800000));
}

// Exact re-rank with certificate; uncertified queries go to the fallback list.
// One warp per query.  Candidate rows are read through a shared-memory tile
// (32 rows x 64 features, padded) so every global read is coalesced and each
// lane then walks its own row.
//   A: FP32 squared distances of the L candidates with rigorous bounds
//      (relative (d+4)u for the FP32 sum, plus the FP64->FP32 conversion of
//      both vectors); U = the kq-th smallest upper bound.
//   B: only candidates whose lower bound does not exceed U can be among the
//      kq nearest: they are compacted and get their canonical FP64 keys.
constexpr int kRrWarps = 4;
constexpr int kRrChunk = 32;

template <typename T>
__device__ __forceinline__ void load_rows(const T* X, int d, const int* rows, int nrows, int c0,
                                          int cw, T* tile, int lane) {
  // tile: 32 rows x (kRrChunk + 1).  Full 16-byte-aligned chunks are read with
  // 16-byte loads, several rows per warp instruction.
  constexpr int V = 16 / sizeof(T);            // elements per 16-byte load
  constexpr int PER_ROW = kRrChunk / V;        // loads per row chunk
  if (cw == kRrChunk && (d % V) == 0 && (reinterpret_cast<uintptr_t>(X) & 15) == 0) {
    for (int e = lane; e < nrows * PER_ROW; e += 32) {
      const int r = e / PER_ROW, v = e - r * PER_ROW;
      const int j = rows[r];
      if (j < 0) continue;
      const T* src = X + (int64_t)j * d + c0 + v * V;
      const float4 f = *reinterpret_cast<const float4*>(src);
      const T* fv = reinterpret_cast<const T*>(&f);
#pragma unroll
      for (int t = 0; t < V; ++t) tile[r * (kRrChunk + 1) + v * V + t] = fv[t];
    }
    return;
  }
  for (int r = 0; r < nrows; ++r) {
    const int j = rows[r];
    if (j < 0) continue;
    const T* src = X + (int64_t)j * d + c0;
    for (int p = lane; p < cw; p += 32) tile[r * (kRrChunk + 1) + p] = src[p];
  }
}

// Dynamic shared memory of rerank_kernel<T, S, KS>: per warp a row tile
// (32 candidate rows and the query row, kRrChunk features each), and two
// candidate-slot lists and two FP32 interval bounds of 32*S entries.
template <typename T>
constexpr size_t rr_smem_bytes(int S) {
  return (size_t)kRrWarps * 33 * (kRrChunk + 1) * sizeof(T) +
         (size_t)kRrWarps * 2 * 32 * S * (sizeof(int) + sizeof(float));
}

// Xa, Qa: FP32 copies of the rows for the bounds pass A (X, Q themselves for
// FP32 inputs; for FP64 inputs converted once, not per candidate visit).
// At most 32*S candidates per query (L <= 32*S), kq <= 32*KS.
template <typename T, int S, int KS>
__global__ void __launch_bounds__(kRrWarps * 32, 1) rerank_kernel(
    const T* __restrict__ X, const T* __restrict__ Q, const float* __restrict__ Xa,
    const float* __restrict__ Qa, int d, int64_t m, int L, int kq,
    const int32_t* __restrict__ cand, const float* __restrict__ ckey,
    const float* __restrict__ xdl, const float* __restrict__ dL,
    const float* __restrict__ qnorm2, const float* __restrict__ qdelta,
    const unsigned int* __restrict__ xstats, const int* __restrict__ err,
    int32_t* __restrict__ idx_out, double* __restrict__ key_out, int* fb_list, int* fb_count) {
  constexpr int LCAP = 32 * S;
  extern __shared__ __align__(16) unsigned char rr_smem[];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t w = (int64_t)blockIdx.x * kRrWarps + wid;
  if (w >= m) return;  // warps are independent: no CTA-wide barrier below
  T* tile = reinterpret_cast<T*>(rr_smem) + (size_t)wid * 33 * (kRrChunk + 1);
  int* lists0 = reinterpret_cast<int*>(rr_smem + (size_t)kRrWarps * 33 * (kRrChunk + 1) * sizeof(T)) +
                (size_t)wid * 2 * LCAP;
  // ivl0[0..LCAP) / ivl0[LCAP..2 LCAP): FP32 interval (lo, hi) per candidate slot
  float* ivl0 = reinterpret_cast<float*>(
                    rr_smem + (size_t)kRrWarps * 33 * (kRrChunk + 1) * sizeof(T) +
                    (size_t)kRrWarps * 2 * LCAP * sizeof(int)) +
                (size_t)wid * 2 * LCAP;
  T* qrow = tile + 32 * (kRrChunk + 1);
  int* rowlist = lists0;
  int* keep = lists0 + LCAP;
  const T* qr = Q + w * d;
  const float u = 5.9604645e-8f;
  const float gam = (d + 4) * u * 1.1f;
  const float xmaxn = __uint_as_float(xstats[0]);
  const float qnrm = sqrtf(qnorm2[w]) * 1.0001f + qdelta[w];
  const float econv = (sizeof(T) == 8) ? 1.01f * u * (qnrm + xmaxn + __uint_as_float(xstats[1])) : 0.f;
  float lo[S], hi[S];
  // A0: the tensor-core distance of each candidate with its rigorous error
  // (FP32 accumulation E, BF16 rounding of both vectors) bounds the exact
  // distance; candidates whose lower bound exceeds the kq-th smallest upper
  // bound cannot be among the kq nearest and skip the FP32 pass.  The others
  // are compacted into the slot list.
  int nsurv = L;
  {
    const float qn0 = sqrtf(qnorm2[w]) * 1.0001f;
    const float E0 =
        2.0f * d * 4.0f * u * qn0 * xmaxn + d * u * (qn0 * qn0 + xmaxn * xmaxn) + 1e-30f;
    const float qd = qdelta[w];
    int jg[S];
    WarpTopK<KS> u0;
    u0.init(kq);
#pragma unroll
    for (int g = 0; g < S; ++g) {
      const int a = 32 * g + lane;
      jg[g] = a < L ? cand[w * L + a] : INT_MAX;
      const bool valid = jg[g] != INT_MAX;
      const float D = valid ? ckey[w * L + a] : 0.0f;
      const float xd = valid ? xdl[jg[g]] : 0.0f;
      const float l = fmaxf(sqrtf(fmaxf(D - E0, 0.0f)) - qd - xd, 0.0f);
      const float h = sqrtf(D + E0) + qd + xd;
      lo[g] = valid ? l * l * (1.0f - 1e-5f) : __int_as_float(0x7f800000);
      u0.offer(valid ? (unsigned long long)__float_as_uint(h * h * (1.0f + 1e-5f)) : ~0ull,
               valid ? a : INT_MAX, lane);
    }
    const float Ub = u0.full() ? __uint_as_float((unsigned int)u0.tk) : __int_as_float(0x7f800000);
    nsurv = 0;
#pragma unroll
    for (int g = 0; g < S; ++g) {
      const bool take = jg[g] != INT_MAX && lo[g] <= Ub;
      const unsigned bal = __ballot_sync(kFull, take);
      if (take) keep[nsurv + __popc(bal & ((1u << lane) - 1u))] = jg[g];
      nsurv += __popc(bal);
    }
    __syncwarp();
  }
  // A: FP32 bounds for the surviving candidates (slots 0 .. nsurv-1)
  WarpTopK<KS> ub;
  ub.init(kq);
#pragma unroll
  for (int g = 0; g < S; ++g) {
    const int a = 32 * g + lane;
    if (32 * g >= nsurv) {  // warp-uniform: no candidate left in this group
      lo[g] = hi[g] = __int_as_float(0x7f800000);
      continue;
    }
    const int j = a < nsurv ? keep[a] : INT_MAX;
    rowlist[lane] = (j == INT_MAX) ? -1 : j;
    __syncwarp();
    float acc = 0.f;
    float* tilef = reinterpret_cast<float*>(tile);
    float* qrowf = tilef + 32 * (kRrChunk + 1);
    const float* qra = Qa + w * d;
    for (int c0 = 0; c0 < d; c0 += kRrChunk) {
      const int cw = min(kRrChunk, d - c0);
      load_rows<float>(Xa, d, rowlist, 32, c0, cw, tilef, lane);
      for (int p = lane; p < cw; p += 32) qrowf[p] = qra[c0 + p];
      __syncwarp();
      const float* myrow = tilef + lane * (kRrChunk + 1);
      for (int p = 0; p < cw; ++p) {
        const float t = qrowf[p] - myrow[p];
        acc = fmaf(t, t, acc);
      }
      __syncwarp();
    }
    const bool valid = rowlist[lane] >= 0;
    const float l = fmaxf(sqrtf(acc * (1.0f - gam)) - econv, 0.0f);
    const float h = sqrtf(acc * (1.0f + gam)) + econv;
    lo[g] = valid ? l * l * (1.0f - 1e-6f) : __int_as_float(0x7f800000);
    hi[g] = valid ? h * h * (1.0f + 1e-6f) : __int_as_float(0x7f800000);
    if (a < LCAP) {
      ivl0[a] = lo[g];
      ivl0[LCAP + a] = hi[g];
      keep[a] = rowlist[lane];
    }
    ub.offer(valid ? (unsigned long long)__float_as_uint(hi[g]) : ~0ull, valid ? a : INT_MAX, lane);
    __syncwarp();
  }
  const float U = ub.full() ? __uint_as_float((unsigned int)ub.tk) : __int_as_float(0x7f800000);
  __syncwarp();
  // Below, a slot can hold a candidate only if a < nsurv (the survivors were
  // packed to the front): testing lo <= U alone would admit the empty slots
  // (lo = U = +inf) when fewer than kq candidates survive, e.g. after a
  // distance pass that gave up.
  // Without requested distances, FP64 keys are needed only when the FP32
  // intervals leave membership or order open.  If exactly kq candidates have
  // lower bound <= U (the kq-th smallest upper bound) and, ordered by
  // midpoint, consecutive intervals are disjoint, that order is the exact one.
  if (key_out == nullptr) {
    int cnt = 0;
#pragma unroll
    for (int g = 0; g < S; ++g)
      cnt += __popc(__ballot_sync(kFull, 32 * g + lane < nsurv && lo[g] <= U));
    if (cnt == kq) {
      WarpTopK<KS> ord;
      ord.init(kq);
#pragma unroll
      for (int g = 0; g < S; ++g) {
        const int a = 32 * g + lane;
        const bool in = a < nsurv && lo[g] <= U;
        const float mid = 0.5f * lo[g] + 0.5f * hi[g];
        ord.offer(in ? (unsigned long long)__float_as_uint(mid) : ~0ull, in ? a : INT_MAX, lane);
      }
      // positions lane*KS + s hold candidate slots ord.i[s]; check each
      // position's interval against the next position's
      bool ok = true;
      const int nxt0 = __shfl_down_sync(kFull, ord.i[0], 1);
#pragma unroll
      for (int s2 = 0; s2 < KS; ++s2) {
        const int pos = lane * KS + s2;
        if (pos + 1 < kq) {
          const int a = ord.i[s2];
          const int b = (s2 + 1 < KS) ? ord.i[(s2 + 1 < KS) ? s2 + 1 : s2] : nxt0;
          if (!(ivl0[LCAP + a] < ivl0[b])) ok = false;
        }
      }
      if (__all_sync(kFull, ok)) {
        float hk = 0.0f;
#pragma unroll
        for (int s2 = 0; s2 < KS; ++s2) {
          const int pos = lane * KS + s2;
          if (pos < kq) idx_out[w * kq + pos] = keep[ord.i[s2]];
          if (pos == kq - 1) hk = ivl0[LCAP + ord.i[s2]];
        }
        hk = __shfl_sync(kFull, hk, (kq - 1) / KS);
        // certificate with the kq-th member's upper bound
        const float xdel0 = __uint_as_float(xstats[1]);
        const float qn0 = sqrtf(qnorm2[w]) * 1.0001f;
        const float E0 =
            2.0f * d * 4.0f * u * qn0 * xmaxn + d * u * (qn0 * qn0 + xmaxn * xmaxn) + 1e-30f;
        const float Dl0 = dL[w];
        float lb0 = fmaxf(sqrtf(fmaxf(Dl0 - E0, 0.0f)) - qdelta[w] - xdel0, 0.0f);
        lb0 = lb0 * lb0 * (1.0f - 1e-5f);
        const bool cert0 = (*err == 0) && (Dl0 == __int_as_float(0x7f800000) || lb0 > hk);
        if (!cert0 && lane == 0) {
          const int pos = atomicAdd(fb_count, 1);
          fb_list[pos] = (int)w;
        }
        return;
      }
    }
  }
  // FP32 inputs: when at most 32 candidates can still be among the kq nearest
  // (lower bound <= U), rank them by double-float distance (relative error
  // <= (d+8) 2^-45, which also covers the canonical FP64 key's rounding).  If
  // every neighbouring gap up to rank kq exceeds both values' error bounds,
  // membership and order are those of the canonical keys.
  if (key_out == nullptr && sizeof(T) == 4 && kq <= 32) {
    int cnt = 0;
#pragma unroll
    for (int g = 0; g < S; ++g)
      cnt += __popc(__ballot_sync(kFull, 32 * g + lane < nsurv && lo[g] <= U));
    if (cnt <= 32) {
      int my_slot = -1, base = 0;
#pragma unroll
      for (int g = 0; g < S; ++g) {
        const int a = 32 * g + lane;
        const bool in = a < nsurv && lo[g] <= U;
        const unsigned bal = __ballot_sync(kFull, in);
        const int pos = base + __popc(bal & ((1u << lane) - 1u));
        // member with position pos is held by lane pos
        for (int src = 0; src < 32; ++src) {
          const int ps = __shfl_sync(kFull, pos, src);
          const int inn = __shfl_sync(kFull, (int)in, src);
          if (inn && ps == lane) my_slot = 32 * g + src;
        }
        base += __popc(bal);
      }
      rowlist[lane] = my_slot >= 0 ? keep[my_slot] : -1;
      __syncwarp();
      dfl acc = {0.0f, 0.0f};
      for (int c0 = 0; c0 < d; c0 += kRrChunk) {
        const int cw = min(kRrChunk, d - c0);
        load_rows<T>(X, d, rowlist, 32, c0, cw, tile, lane);
        for (int p = lane; p < cw; p += 32) qrow[p] = qr[c0 + p];
        __syncwarp();
        if (my_slot >= 0) {
          const T* myrow = tile + lane * (kRrChunk + 1);
          for (int p = 0; p < cw; ++p) {
            const dfl t = df_two_sum((float)qrow[p], -(float)myrow[p]);
            acc = df_add_fast(acc, df_sqr(t));
          }
        }
        __syncwarp();
      }
      const float eps = (d + 8) * 2.85e-14f;
      WarpTopK<1> o2;
      o2.init(cnt);
      o2.offer(my_slot >= 0 ? (unsigned long long)__float_as_uint(acc.hi) : ~0ull,
               my_slot >= 0 ? lane : INT_MAX, lane);
      const int src = o2.i[0] < 32 ? o2.i[0] : 0;  // lane holding the member ranked here
      const dfl mine = {__shfl_sync(kFull, acc.hi, src), __shfl_sync(kFull, acc.lo, src)};
      const dfl next = {__shfl_down_sync(kFull, mine.hi, 1), __shfl_down_sync(kFull, mine.lo, 1)};
      bool ok2 = true;
      if (lane < kq && lane + 1 < cnt) {
        const dfl gap = df_add(next, df_neg(mine));
        ok2 = gap.hi > eps * (mine.hi + next.hi) + 1e-37f;
      }
      if (cnt >= kq && __all_sync(kFull, ok2)) {
        const int slot = __shfl_sync(kFull, my_slot, src);
        if (lane < kq) idx_out[w * kq + lane] = keep[slot];
        float hk = __shfl_sync(kFull, mine.hi + fabsf(mine.lo), kq - 1);
        hk = hk * (1.0f + 1e-6f) + 1e-37f;  // upper bound of the kq-th canonical key
        const float xdel0 = __uint_as_float(xstats[1]);
        const float qn0 = sqrtf(qnorm2[w]) * 1.0001f;
        const float E0 =
            2.0f * d * 4.0f * u * qn0 * xmaxn + d * u * (qn0 * qn0 + xmaxn * xmaxn) + 1e-30f;
        const float Dl0 = dL[w];
        float lb0 = fmaxf(sqrtf(fmaxf(Dl0 - E0, 0.0f)) - qdelta[w] - xdel0, 0.0f);
        lb0 = lb0 * lb0 * (1.0f - 1e-5f);
        const bool cert0 = (*err == 0) && (Dl0 == __int_as_float(0x7f800000) || lb0 > hk);
        if (!cert0 && lane == 0) {
          const int pos = atomicAdd(fb_count, 1);
          fb_list[pos] = (int)w;
        }
        return;
      }
    }
  }
  // B: compact the candidates that can still be among the kq nearest
  int nkeep = 0;
#pragma unroll
  for (int g = 0; g < S; ++g) {
    const int a = 32 * g + lane;
    const bool take = a < nsurv && lo[g] <= U;
    const unsigned bal = __ballot_sync(kFull, take);
    const int cj = take ? keep[a] : 0;
    __syncwarp();
    if (take) keep[nkeep + __popc(bal & ((1u << lane) - 1u))] = cj;
    __syncwarp();
    nkeep += __popc(bal);
  }
  __syncwarp();
  WarpTopK<KS> top;
  top.init(kq);
  for (int base = 0; base < nkeep; base += 32) {
    const int cnt = min(32, nkeep - base);
    rowlist[lane] = lane < cnt ? keep[base + lane] : -1;
    __syncwarp();
    double s = 0.0;
    for (int c0 = 0; c0 < d; c0 += kRrChunk) {
      const int cw = min(kRrChunk, d - c0);
      load_rows<T>(X, d, rowlist, cnt, c0, cw, tile, lane);
      for (int p = lane; p < cw; p += 32) qrow[p] = qr[c0 + p];
      __syncwarp();
      if (lane < cnt) {
        const T* myrow = tile + lane * (kRrChunk + 1);
        int p = 0;
        if (c0 == 0) {  // canonical key: first term t0*t0, then left-to-right rounded sums
          const double t = __dsub_rn((double)qrow[0], (double)myrow[0]);
          s = __dmul_rn(t, t);
          p = 1;
        }
        for (; p < cw; ++p) {
          const double t = __dsub_rn((double)qrow[p], (double)myrow[p]);
          s = __dadd_rn(s, __dmul_rn(t, t));
        }
      }
      __syncwarp();
    }
    top.offer(lane < cnt ? dbits(s) : ~0ull, lane < cnt ? rowlist[lane] : INT_MAX, lane);
    __syncwarp();
  }
  // certificate for candidates outside the list (approximate distance >= dL)
  const float xdel = __uint_as_float(xstats[1]);
  const float qn = sqrtf(qnorm2[w]) * 1.0001f;
  const float E = 2.0f * d * 4.0f * u * qn * xmaxn + d * u * (qn * qn + xmaxn * xmaxn) + 1e-30f;
  const float Dl = dL[w];
  float lb = fmaxf(sqrtf(fmaxf(Dl - E, 0.0f)) - qdelta[w] - xdel, 0.0f);
  lb = lb * lb * (1.0f - 1e-5f);
  const float kth_up = key_bits_to_float_up(top.tk);
  // a distance pass that gave up (err) certifies nothing: every query is redone
  const bool cert =
      (*err == 0) && top.full() && (Dl == __int_as_float(0x7f800000) || lb > kth_up);
  if (cert) {
    top.store(kq, lane, idx_out + w * kq, key_out ? key_out + w * kq : nullptr);
  } else if (lane == 0) {
    const int pos = atomicAdd(fb_count, 1);
    fb_list[pos] = (int)w;
  }
}

template <typename T, int S, int KS>
int launch_rerank_t(const T* X, const T* Q, const float* Xa, const float* Qa, int d, int64_t m,
                    int L, int kq, const int32_t* cand, const float* ckey, const float* xdl,
                    const float* dL, const float* qn2, const float* qdl, const unsigned int* xst,
                    const int* err, int32_t* idx, double* key, int* fbl, int* fbc,
                    cudaStream_t s) {
  const int blocks = ceil_div(m, kRrWarps);
  constexpr size_t smem = rr_smem_bytes<T>(S);
  FMGP_CUDA_TRY(ensure_smem((const void*)rerank_kernel<T, S, KS>, smem));
  FMGP_LAUNCH((rerank_kernel<T, S, KS><<<blocks, kRrWarps * 32, smem, s>>>(
      X, Q, Xa, Qa, d, m, L, kq, cand, ckey, xdl, dL, qn2, qdl, xst, err, idx, key, fbl, fbc)));
  FMGP_CUDA_TRY(cudaGetLastError());
  return FMGP_OK;
}

// The instance for L candidates (L <= 32*S) and kq results (kq <= 32*KS).
// Lists of up to 128 candidates come in every (S, KS); longer ones only for
// L = round_up(2 kq, 32), i.e. S = 6, 8, 10 with KS = S / 2 (a shorter L or
// kq rounds up to the next instance).
template <typename T>
int launch_rerank(const T* X, const T* Q, const float* Xa, const float* Qa, int d, int64_t m,
                  int L, int kq, const int32_t* cand, const float* ckey, const float* xdl,
                  const float* dL, const float* qn2, const float* qdl, const unsigned int* xst,
                  const int* err, int32_t* idx, double* key, int* fbl, int* fbc,
                  cudaStream_t s) {
  const int S = (L + 31) / 32, KS = (kq + 31) / 32;
#define FMGP_RR(SS, KK)                                                                       \
  return launch_rerank_t<T, SS, KK>(X, Q, Xa, Qa, d, m, L, kq, cand, ckey, xdl, dL, qn2, qdl, \
                                    xst, err, idx, key, fbl, fbc, s)
  if (S <= 4) {
    const int si = S * 4 + KS;
    switch (si) {
      case 1 * 4 + 1: FMGP_RR(1, 1);
      case 2 * 4 + 1: FMGP_RR(2, 1);
      case 2 * 4 + 2: FMGP_RR(2, 2);
      case 3 * 4 + 1: FMGP_RR(3, 1);
      case 3 * 4 + 2: FMGP_RR(3, 2);
      case 3 * 4 + 3: FMGP_RR(3, 3);
      case 4 * 4 + 1: FMGP_RR(4, 1);
      case 4 * 4 + 2: FMGP_RR(4, 2);
      case 4 * 4 + 3: FMGP_RR(4, 3);
      default: FMGP_RR(4, 4);
    }
  }
  if (S <= 6 && KS <= 3) FMGP_RR(6, 3);
  if (S <= 8 && KS <= 4) FMGP_RR(8, 4);
  FMGP_RR(10, 5);
#undef FMGP_RR
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
  const int blocks = (int)std::min<int64_t>(ceil_div(rows_pad, kPackThreads / 32),
                                            (int64_t)num_sms() * 8);
  FMGP_LAUNCH(pack_bf16_kernel<T><<<blocks, kPackThreads, 0, s>>>(
      X, rows, d, rows_pad, d_pad, *Xb, *n2, *dl, *stats));
  FMGP_CUDA_TRY(cudaGetLastError());
  return FMGP_OK;
}

// Candidates kept per query for the re-rank, in whole warps: the tuned
// multiple of kq (at least 32) up to 128, and above that 2 kq (at most 320,
// i.e. kq <= 160).
int tc_list_len(int kq) {
  const int want = std::max(32, std::min(tune_params().tc_oversample * kq, std::max(128, 2 * kq)));
  return std::min(kMaxTcList, (want + 31) / 32 * 32);
}

// Per-range list length of the fused selection for kq neighbours (0 = the
// pass-buffer form); the tc_fused_r tuning key overrides it (R >= kq / 4).
// Above kq = 32 the lists keep 32 and the candidates are split into more
// ranges instead (tc_fused_ranges_min).
int tc_fused_r(int kq) {
  if (!tune_params().tc_fused_select) return 0;
  const int o = tune_params().tc_fused_r;
  if (o && kq <= 32 && (o == 8 || o == 16 || o == 32) && kq <= 4 * o) return o;
  return kq <= 4 ? 8 : kq <= 16 ? 16 : 32;
}

// Fewest candidate ranges per query block for the fused selection: with 2
// column halves per range, 2 * ranges * R list entries hold at least four
// times kq, so no half-range is expected to hold more than an eighth of the
// kq nearest and every range's R-th value lies well beyond the kq-th.
int tc_fused_ranges_min(int kq, int R) {
  if (kq <= 32) return R >= 16 ? 4 : 2;
  return std::max(4, (4 * kq + 2 * R - 1) / (2 * R));
}

// FP32 rows of X for the re-rank's bounds pass: X itself, or a copy of an
// FP64 X.
template <typename T>
int f32_rows(const T* X, int64_t n, int d, Workspace& ws, cudaStream_t s, const float** out) {
  if (sizeof(T) == 4) {
    *out = reinterpret_cast<const float*>(X);
    return FMGP_OK;
  }
  float* f = ws.get<float>((size_t)n * d);
  if (!f) return FMGP_ENOMEM;
  *out = f;
  return to_f32(reinterpret_cast<const double*>(X), n * d, f, s);
}

// pre: the training side packed by tc_pack_train (null: packed here).
template <typename T>
int tc_knn_t(const T* X, int64_t n, int d, const T* Q, int64_t m, int kq, bool self,
             int32_t* idx_out, double* key_out, Workspace& ws, cudaStream_t s,
             const TcPacked* pre = nullptr) {
  const int L = tc_list_len(kq);
  const int S = L / 32;
  const int d_pad = (d + kTK - 1) / kTK * kTK;
  const int64_t n_pad = (n + kTN - 1) / kTN * kTN;
  const int64_t m_pad = (m + kTM - 1) / kTM * kTM;
  __nv_bfloat16 *Xb, *Qb;
  float *xn2, *xdl, *qn2, *qdl;
  unsigned int *xst, *qst;
  int rc = FMGP_OK;
  if (pre) {
    Xb = reinterpret_cast<__nv_bfloat16*>(const_cast<void*>(pre->Xb));
    xn2 = const_cast<float*>(pre->xn2);
    xdl = const_cast<float*>(pre->xdl);
    xst = const_cast<unsigned int*>(pre->xst);
  } else {
    rc = pack<T>(X, n, d, n_pad, d_pad, ws, s, &Xb, &xn2, &xdl, &xst);
    if (rc) return rc;
  }
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
  const int n_tiles = (int)(n_pad / kTN), k_chunks = d_pad / kTK;
  const int64_t qblocks = m_pad / kTM;
  int32_t* cand = ws.get<int32_t>((size_t)m * L);
  float* ckey = ws.get<float>((size_t)m * L);
  float* dL = ws.get<float>(m);
  int* err = ws.get<int>(1);
  int* fb_list = ws.get<int>(m);
  int* fb_count = ws.get<int>(1);
  if (!cand || !ckey || !dL || !err || !fb_list || !fb_count) return FMGP_ENOMEM;
  FMGP_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), s));
  FMGP_CUDA_TRY(cudaMemsetAsync(fb_count, 0, sizeof(int), s));
  const int sblocks = ceil_div(m * 32, 256);
  // limit of the distance kernel's main-loop waits (the drains after an
  // abort keep kDrainWaitNs)
  const uint64_t main_wait = tune_params().tc_wait_ns > 0 ? (uint64_t)tune_params().tc_wait_ns
                                                          : kDrainWaitNs;
  const int R = tc_fused_r(kq);
  if (R > 0) {
    // candidate ranges per query block: the split with the shortest
    // makespan (whole waves of one CTA per SM x tiles per CTA, plus a tile's
    // worth of start-up), with at least tc_fused_ranges_min ranges so the
    // ranges' R-th keys lie well beyond the kq nearest.  Up to kq = 32 the
    // per-range lists of all queries stay within ~1 GB; above it the ranges
    // are at most 12 (768 list entries per query) and the query blocks are
    // processed in chunks whose lists take at most ~1 GB.
    const int sms = num_sms();
    const int ys_lo = std::min(n_tiles, tc_fused_ranges_min(kq, R));
    const int64_t per_range = 2 * m_pad * R * (int64_t)(sizeof(float) + sizeof(int32_t));
    const int ys_hi =
        kq <= 32 ? (int)std::max<int64_t>(
                       ys_lo, std::min<int64_t>(std::min(n_tiles, 128), (1ll << 30) / per_range))
                 : std::max(ys_lo, std::min(n_tiles, 12));
    int nseg = ys_lo;
    int64_t best = INT64_MAX;
    for (int ys = ys_lo; ys <= ys_hi; ++ys) {
      const int tpc = ceil_div(n_tiles, ys);
      if (ceil_div(n_tiles, tpc) != ys) continue;  // same ranges as a smaller split
      const int64_t cost = ceil_div(qblocks * ys, sms) * (int64_t)(tpc + 2);
      if (cost < best) { best = cost; nseg = ys; }
    }
    const int tpc = ceil_div(n_tiles, nseg);
    const int64_t lists_per_qb = (int64_t)kTM * 2 * nseg * R;  // entries per query block
    const int64_t cq = tune_params().tc_chunk_queries;
    const int64_t chunk_qb = std::max<int64_t>(
        1, std::min<int64_t>(qblocks, cq > 0 ? cq / kTM : (1ll << 30) / (lists_per_qb * 8)));
    float* pkey = ws.get<float>((size_t)(chunk_qb * lists_per_qb));
    int32_t* pidx = ws.get<int32_t>((size_t)(chunk_qb * lists_per_qb));
    if (!pkey || !pidx) return FMGP_ENOMEM;
    const void* kfn = R == 8 ? (const void*)tc_dist_kernel<8>
                    : R == 16 ? (const void*)tc_dist_kernel<16> : (const void*)tc_dist_kernel<32>;
    FMGP_CUDA_TRY(ensure_smem(kfn, kTcSelSmem));
    const int tot = 2 * nseg * R;
    for (int64_t qb0 = 0; qb0 < qblocks; qb0 += chunk_qb) {
      const int64_t nqb = std::min(chunk_qb, qblocks - qb0);
      const int64_t q0 = qb0 * kTM;
      const int64_t mc = std::min<int64_t>(m, (qb0 + nqb) * kTM) - q0;  // queries of the chunk
      const dim3 grid((unsigned)nqb, (unsigned)nseg);
      if (R == 8)
        FMGP_LAUNCH(tc_dist_kernel<8><<<grid, kTcSelThreads, kTcSelSmem, s>>>(
            tmQ, tmX, qn2, xn2, (int)qb0, 0, n_tiles, tpc, k_chunks, 0, nullptr, n, self ? 1 : 0,
            pkey, pidx, err, main_wait));
      else if (R == 16)
        FMGP_LAUNCH(tc_dist_kernel<16><<<grid, kTcSelThreads, kTcSelSmem, s>>>(
            tmQ, tmX, qn2, xn2, (int)qb0, 0, n_tiles, tpc, k_chunks, 0, nullptr, n, self ? 1 : 0,
            pkey, pidx, err, main_wait));
      else
        FMGP_LAUNCH(tc_dist_kernel<32><<<grid, kTcSelThreads, kTcSelSmem, s>>>(
            tmQ, tmX, qn2, xn2, (int)qb0, 0, n_tiles, tpc, k_chunks, 0, nullptr, n, self ? 1 : 0,
            pkey, pidx, err, main_wait));
      const int cblocks = (int)ceil_div(mc * 32, 256);
      int32_t* cc = cand + q0 * L;
      float* ck = ckey + q0 * L;
      float* cd = dL + q0;
      if (tot <= 128)
        FMGP_LAUNCH(select_parts_bisect_kernel<4><<<cblocks, 256, 0, s>>>(pkey, pidx, mc, 2 * nseg, R, L, cc, ck, cd));
      else if (tot <= 256)
        FMGP_LAUNCH(select_parts_bisect_kernel<8><<<cblocks, 256, 0, s>>>(pkey, pidx, mc, 2 * nseg, R, L, cc, ck, cd));
      else if (tot <= 512)
        FMGP_LAUNCH(select_parts_bisect_kernel<16><<<cblocks, 256, 0, s>>>(pkey, pidx, mc, 2 * nseg, R, L, cc, ck, cd));
      else if (tot <= 768)
        FMGP_LAUNCH(select_parts_bisect_kernel<24><<<cblocks, 256, 0, s>>>(pkey, pidx, mc, 2 * nseg, R, L, cc, ck, cd));
      else switch (S) {  // kq <= 32 here: L <= 128
        case 1: FMGP_LAUNCH(select_parts_kernel<1><<<cblocks, 256, 0, s>>>(pkey, pidx, mc, 2 * nseg, R, L, cc, ck, cd)); break;
        case 2: FMGP_LAUNCH(select_parts_kernel<2><<<cblocks, 256, 0, s>>>(pkey, pidx, mc, 2 * nseg, R, L, cc, ck, cd)); break;
        case 3: FMGP_LAUNCH(select_parts_kernel<3><<<cblocks, 256, 0, s>>>(pkey, pidx, mc, 2 * nseg, R, L, cc, ck, cd)); break;
        default: FMGP_LAUNCH(select_parts_kernel<4><<<cblocks, 256, 0, s>>>(pkey, pidx, mc, 2 * nseg, R, L, cc, ck, cd)); break;
      }
    }
  } else {
    // candidate range in chunks of whole tiles; the chunk buffer holds ~1 GB
    int chunk_tiles = (int)std::max<int64_t>(1, (int64_t)(1ll << 30) / (m_pad * 4 * kTN));
    chunk_tiles = std::min(chunk_tiles, n_tiles);
    // tiles per CTA: enough CTAs for two waves over the SMs
    const int64_t want = 2ll * num_sms();
    int tpc = chunk_tiles;
    while (tpc > 1 && qblocks * ((chunk_tiles + tpc - 1) / tpc) < want) tpc = (tpc + 1) / 2;
    const int ysplit = (chunk_tiles + tpc - 1) / tpc;
    float* Dc = ws.get<float>((size_t)m_pad * chunk_tiles * kTN);
    if (!Dc) return FMGP_ENOMEM;
    FMGP_CUDA_TRY(ensure_smem((const void*)tc_dist_kernel<0>, kTcSmem));
    const int64_t ldc = (int64_t)chunk_tiles * kTN;
    for (int t0 = 0; t0 < n_tiles; t0 += chunk_tiles) {
      const int t1 = std::min(n_tiles, t0 + chunk_tiles);
      FMGP_LAUNCH(tc_dist_kernel<0><<<dim3((unsigned)qblocks, (unsigned)ysplit), kTcThreads, kTcSmem, s>>>(
          tmQ, tmX, qn2, xn2, 0, t0, t1, tpc, k_chunks, ldc, Dc, n, 0, nullptr, nullptr, err, main_wait));
      const int64_t col0 = (int64_t)t0 * kTN, ncols = (int64_t)(t1 - t0) * kTN;
      const int first = t0 == 0 ? 1 : 0;
      switch (S <= 4 ? S : S <= 6 ? 6 : S <= 8 ? 8 : 10) {  // list slots per lane >= L / 32
        case 1: FMGP_LAUNCH(select_merge_kernel<1><<<sblocks, 256, 0, s>>>(Dc, ldc, m, col0, ncols, n, L, self, first, cand, ckey, dL)); break;
        case 2: FMGP_LAUNCH(select_merge_kernel<2><<<sblocks, 256, 0, s>>>(Dc, ldc, m, col0, ncols, n, L, self, first, cand, ckey, dL)); break;
        case 3: FMGP_LAUNCH(select_merge_kernel<3><<<sblocks, 256, 0, s>>>(Dc, ldc, m, col0, ncols, n, L, self, first, cand, ckey, dL)); break;
        case 4: FMGP_LAUNCH(select_merge_kernel<4><<<sblocks, 256, 0, s>>>(Dc, ldc, m, col0, ncols, n, L, self, first, cand, ckey, dL)); break;
        case 6: FMGP_LAUNCH(select_merge_kernel<6><<<sblocks, 256, 0, s>>>(Dc, ldc, m, col0, ncols, n, L, self, first, cand, ckey, dL)); break;
        case 8: FMGP_LAUNCH(select_merge_kernel<8><<<sblocks, 256, 0, s>>>(Dc, ldc, m, col0, ncols, n, L, self, first, cand, ckey, dL)); break;
        default: FMGP_LAUNCH(select_merge_kernel<10><<<sblocks, 256, 0, s>>>(Dc, ldc, m, col0, ncols, n, L, self, first, cand, ckey, dL)); break;
      }
    }
  }
  FMGP_CUDA_TRY(cudaGetLastError());
  // FP32 rows for the re-rank's bounds pass
  const float* Xa = nullptr;
  const float* Qa = nullptr;
  if (pre) Xa = pre->Xa;
  else if ((rc = f32_rows<T>(X, n, d, ws, s, &Xa))) return rc;
  if (self) Qa = Xa;
  else if ((rc = f32_rows<T>(Q, m, d, ws, s, &Qa))) return rc;
  rc = launch_rerank<T>(X, Q, Xa, Qa, d, m, L, kq, cand, ckey, xdl, dL, qn2, qdl, xst, err,
                        idx_out, key_out, fb_list, fb_count, s);
  if (rc) return rc;
  FMGP_CUDA_TRY(cudaGetLastError());
  diag_record_tc(fb_count, s);
  // exhaustive exact scan for uncertified queries
  return knn_brute_list(X, sizeof(T) == 8 ? FMGP_F64 : FMGP_F32, n, d, Q, m, kq, self, fb_list,
                        fb_count, idx_out, key_out, ws, s, Xa);
}

}  // namespace

bool tc_knn_eligible(int64_t n, int d, int64_t m, int kq) {
  const TuneParams& tp = tune_params();
  if (!tp.use_tensor_cores) return false;
  const int L = tc_list_len(kq);
  return d >= 16 && kq <= kMaxK && n > 2 * L && n >= 4096 && m >= 128;
}

int tc_pack_train(const void* X, fmgp_dtype dtype, int64_t n, int d, Workspace& ws,
                  cudaStream_t s, TcPacked* out) {
  const int d_pad = (d + kTK - 1) / kTK * kTK;
  const int64_t n_pad = (n + kTN - 1) / kTN * kTN;
  __nv_bfloat16* Xb;
  float *xn2, *xdl;
  unsigned int* xst;
  const float* Xa;
  int rc;
  if (dtype == FMGP_F64) {
    rc = pack<double>((const double*)X, n, d, n_pad, d_pad, ws, s, &Xb, &xn2, &xdl, &xst);
    if (!rc) rc = f32_rows<double>((const double*)X, n, d, ws, s, &Xa);
  } else {
    rc = pack<float>((const float*)X, n, d, n_pad, d_pad, ws, s, &Xb, &xn2, &xdl, &xst);
    if (!rc) rc = f32_rows<float>((const float*)X, n, d, ws, s, &Xa);
  }
  if (rc) return rc;
  out->Xb = Xb;
  out->xn2 = xn2;
  out->xdl = xdl;
  out->xst = xst;
  out->Xa = Xa;
  return FMGP_OK;
}

int tc_knn_query_packed(const TcPacked& P, const void* X, fmgp_dtype dtype, int64_t n, int d,
                        const void* Q, int64_t m, int kq, int32_t* idx_out, double* key_out,
                        Workspace& ws, cudaStream_t s) {
  if (dtype == FMGP_F64)
    return tc_knn_t<double>((const double*)X, n, d, (const double*)Q, m, kq, false, idx_out,
                            key_out, ws, s, &P);
  return tc_knn_t<float>((const float*)X, n, d, (const float*)Q, m, kq, false, idx_out, key_out,
                         ws, s, &P);
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
