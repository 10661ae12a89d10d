// Arithmetic-pipe throughput probe: the FP32 and FP64 fused multiply-add
// peaks that the roofline fractions of the neighbourhood kernels are quoted
// against (their bound is the ALU pipe, not HBM or the tensor cores).
//
// Every thread runs kChains independent FMA chains x = x * a + b for `iters`
// rounds; the grid fills every SM with 2 CTAs of 1024 threads, so issue, not
// latency, bounds the kernel.  Work = 2 * kChains * iters flops per thread.
// The result is written only when it equals an impossible sentinel, which
// keeps the chains live without a store per thread.
#include <algorithm>
#include "common.cuh"

namespace fmgp {
namespace {

constexpr int kChains = 8;
constexpr int kProbeThreads = 1024;

// Target of the never-taken store that keeps the chains live.
__device__ double g_probe_sink;

template <typename T>
__global__ void __launch_bounds__(kProbeThreads) fma_probe_kernel(T a, T b, int iters) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == (T)-1.2345e30) g_probe_sink = (double)s;
}

template <typename T>
int run_probe(int iters, double* flops_per_s, cudaStream_t s) {
  const int blocks = 2 * num_sms();
  cudaEvent_t e0, e1;
  FMGP_CUDA_TRY(cudaEventCreate(&e0));
  FMGP_CUDA_TRY(cudaEventCreate(&e1));
  // a < 1 and b > 0: every chain converges to b / (1 - a), no overflow or denormals
  const T a = (T)0.9990234375, b = (T)1.0e-3;
  double best = 0.0;
  int rc = FMGP_OK;
  for (int rep = 0; rep < 4 && rc == FMGP_OK; ++rep) {  // the first launch warms up
    cudaError_t e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) {
      FMGP_LAUNCH(fma_probe_kernel<T><<<blocks, kProbeThreads, 0, s>>>(a, b, iters));
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "peak probe");
      break;
    }
    if (rep > 0 && ms > 0.0f) {
      const double fl = 2.0 * kChains * (double)iters * (double)blocks * kProbeThreads;
      best = std::max(best, fl / (ms * 1e-3));
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc == FMGP_OK) *flops_per_s = best;
  return rc;
}

}  // namespace
}  // namespace fmgp

using namespace fmgp;

extern "C" int fmgp_peak_probe(int32_t pipe, double* flops_per_s, void* stream) {
  clear_error();
  if (!flops_per_s || (pipe != 0 && pipe != 1)) {
    set_error("fmgp_peak_probe: pipe must be 0 (FP32) or 1 (FP64) and flops_per_s non-NULL");
    return FMGP_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  // about 30 ms per launch on a GB300 (FP32 ~75 TFLOP/s, FP64 ~1.2 TFLOP/s)
  return pipe == 0 ? run_probe<float>(400000, flops_per_s, s)
                   : run_probe<double>(8000, flops_per_s, s);
}
