// fmgp_loocv_objective_noalloc: the LOOCV objective without any device
// allocation.  Some callers cannot allocate device memory once they are
// running: a host application that hands this library a fixed device-memory
// budget up front, or a plugin living inside a framework that owns the
// device allocator and forbids its guests from calling cudaMalloc.  For them
// this entry point keeps its scratch (the per-point residuals, the objective
// and a failure counter) in one file-scope device array instead of the
// stream-ordered workspace the other entry points use.
#include <mutex>
#include "block.cuh"
#include "knn.cuh"

namespace fmgp {
namespace {

// Largest batch this entry point accepts.
constexpr int64_t kNoAllocMaxBatch = 65536;

struct NoAllocScratch {
  double resid[kNoAllocMaxBatch];  // per-point squared residuals
  double q;                        // the objective
  unsigned long long queue;        // work counter of the persistent block kernel
  int fails;                       // blocks whose Cholesky failed
};

// About 512 KB; every device that loads the library holds it until exit.
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

// Device address of g_noalloc_scratch per device.  In host code the symbol
// itself is only a host-side stand-in, so the address is looked up once per
// device (with that device current) and reused.
std::mutex g_noalloc_mu;
NoAllocScratch* g_noalloc_addr[64];

int noalloc_scratch(NoAllocScratch** out) {
  int dev = 0;
  FMGP_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    set_error("device ordinal %d out of range", dev);
    return FMGP_EUNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_noalloc_addr[dev] = (NoAllocScratch*)p;
  }
  *out = g_noalloc_addr[dev];
  return FMGP_OK;
}

// Fixed-shape, deterministic sum of the residuals (same order as the
// allocating entry point): thread t adds entries t, t+1024, ..., then a tree.
__global__ void __launch_bounds__(1024) noalloc_reduce(const double* resid, int64_t b,
                                                       double* out) {
  __shared__ double part[1024];
  double s = 0.0;
  for (int64_t q = threadIdx.x; q < b; q += 1024) s += resid[q];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int w = 512; w > 0; w >>= 1) {
    if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = part[0] / (double)b;
}

bool noalloc_kernel_ok(const fmgp_kernel* k) {
  if (!k) return false;
  if (k->kind != FMGP_KERNEL_MATERN && k->kind != FMGP_KERNEL_RBF) return false;
  if (k->kind == FMGP_KERNEL_MATERN && !(k->nu == 0.5 || k->nu == 1.5 || k->nu == 2.5))
    return false;
  return k->length_scale > 0.0 && isfinite(k->length_scale) && k->variance > 0.0 &&
         isfinite(k->variance) && k->nugget >= 0.0 && isfinite(k->nugget);
}

}  // namespace
}  // namespace fmgp

using namespace fmgp;

extern "C" int fmgp_loocv_objective_noalloc(const void* X, fmgp_dtype dtype, const double* Y,
                                            int64_t n, int32_t d, int32_t r,
                                            const int32_t* nbr, int32_t nbr_ld, int32_t k,
                                            const int64_t* batch, int64_t b,
                                            const fmgp_kernel* kernel, fmgp_precision precision,
                                            double* Q_out, double* resid_out, void* stream) {
  clear_error();
  if (dtype != FMGP_F32 && dtype != FMGP_F64) {
    set_error("dtype %d unknown", (int)dtype);
    return FMGP_EINVAL;
  }
  if (!noalloc_kernel_ok(kernel)) {
    set_error("kernel hyperparameters invalid (nu in {0.5,1.5,2.5}, rho>0, sigma^2>0, tau^2>=0)");
    return FMGP_EINVAL;
  }
  if (!X || !Y || !nbr || !batch || !Q_out) {
    set_error("X, Y, nbr, batch and Q_out must be non-NULL");
    return FMGP_EINVAL;
  }
  if (n < 2 || n >= INT32_MAX || d < 1 || r < 1 || k < 1 || k > n - 1 || k > kMaxK ||
      nbr_ld < k) {
    set_error("shape invalid: n=%lld d=%d r=%d k=%d nbr_ld=%d", (long long)n, d, r, k, nbr_ld);
    return FMGP_EINVAL;
  }
  if (b < 1 || b > kNoAllocMaxBatch) {
    set_error("batch size b = %lld outside [1, %lld], the fixed scratch limit of "
              "fmgp_loocv_objective_noalloc", (long long)b, (long long)kNoAllocMaxBatch);
    return FMGP_EINVAL;
  }
  if (precision != FMGP_PREC_FP64) {
    set_error("fmgp_loocv_objective_noalloc computes in FP64 only");
    return FMGP_EUNSUPPORTED;
  }
  NoAllocScratch* sc = nullptr;
  int rc = noalloc_scratch(&sc);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  FMGP_CUDA_TRY(cudaMemsetAsync(&sc->fails, 0, sizeof(int), s));
  BlockArgs a{};
  a.Y = Y;
  a.nbr = nbr;
  a.batch = batch;
  a.resid = resid_out ? resid_out : sc->resid;
  a.fail_count = &sc->fails;
  a.queue = block_persistent_for((int)FMGP_PREC_FP64, k, d, r, (int)dtype) ? &sc->queue : nullptr;
  a.n = n;
  a.count = b;
  a.d = d;
  a.r = r;
  a.ld = nbr_ld;
  a.k = k;
  a.kp = make_kparams(*kernel);
  a.layout = block_layout(k, d, r, dtype == FMGP_F64 ? 8 : 4, false);
  if (a.layout.bytes_per_warp > 200 * 1024) {
    set_error("neighbourhood k=%d d=%d r=%d needs %zu bytes of shared memory per warp", k, d, r,
              a.layout.bytes_per_warp);
    return FMGP_EUNSUPPORTED;
  }
  // the launch shape of fmgp_loocv_objective: the user's or the autotuner's
  // warps per CTA, else (0) the occupancy-best one (the search allocates nothing)
  int warps = tune_params().block_warps;
  if (warps == 0) warps = tuned_block_warps((int)FMGP_PREC_FP64, k, d, r, (int)dtype);
  rc = launch_block_f64(a, X, dtype, kModeLoocv, warps, s);
  if (rc) return rc;
  FMGP_LAUNCH(noalloc_reduce<<<1, 1024, 0, s>>>(a.resid, b, &sc->q));
  FMGP_CUDA_TRY(cudaGetLastError());
  int h = 0;
  FMGP_CUDA_TRY(cudaMemcpyAsync(Q_out, &sc->q, sizeof(double), cudaMemcpyDeviceToHost, s));
  FMGP_CUDA_TRY(cudaMemcpyAsync(&h, &sc->fails, sizeof(int), cudaMemcpyDeviceToHost, s));
  FMGP_CUDA_TRY(cudaStreamSynchronize(s));
  if (h) {
    set_error("%d LOOCV blocks were not positive definite", h);
    return FMGP_ENOTSPD;
  }
  return FMGP_OK;
}
