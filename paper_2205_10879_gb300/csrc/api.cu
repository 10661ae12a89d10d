// C-ABI entry points of libfmgp: argument validation on the host, workspace,
// and the launch sequence of each step.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>
#include <math.h>
#include <atomic>
#include <initializer_list>
#include <map>
#include <tuple>
#include <string>
#include <mutex>
#include "block.cuh"
#include "knn.cuh"
#include "predict.cuh"

namespace fmgp {

static thread_local char g_err[512] = "";
static std::atomic<unsigned long long> g_launches{0};

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

void clear_error() { g_err[0] = 0; }

int cuda_fail(cudaError_t e, const char* what) {
  set_error("CUDA error %d (%s) in %s", (int)e, cudaGetErrorString(e), what);
  return FMGP_ECUDA;
}

cudaError_t ensure_smem(const void* func, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  size_t& cur = cache[{dev, func}];
  if (cur >= bytes) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}

int active_ctas(const void* func, int threads, size_t smem) {
  static std::mutex mu;
  static std::map<std::tuple<int, const void*, int, size_t>, int> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find({dev, func, threads, smem});
    if (it != cache.end()) return it->second;
  }
  int nb = 0;
  if (smem > 227 * 1024 || ensure_smem(func, smem) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, func, threads, smem) != cudaSuccess) {
    cudaGetLastError();
    nb = 0;
  }
  std::lock_guard<std::mutex> lk(mu);
  cache[{dev, func, threads, smem}] = nb;
  return nb;
}

int num_sms() {
  static int cached[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (!cached[dev]) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cached[dev] = v > 0 ? v : 1;
  }
  return cached[dev];
}

static void keep_pool_memory() {
  static std::once_flag once[64];
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return;
  std::call_once(once[dev], [dev]() {
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t thr = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
  });
}

}  // namespace fmgp

// A workspace context: a private stream-ordered memory pool of fixed maximum
// size on one device, with that size reserved at creation.
struct fmgp_context {
  int device = 0;
  cudaMemPool_t pool = nullptr;
  int64_t bytes = 0;
  std::atomic<int64_t> in_use{0};  // bytes the library's buffers hold from it
};

namespace fmgp {

static thread_local fmgp_context* t_ctx = nullptr;  // bound by fmgp_context_bind
// Host-side failure injection (tuning key "fail_alloc_after"): the number of
// workspace allocations still allowed before every further one fails; < 0 = off.
static std::atomic<long long> g_alloc_budget{-1};

void* Workspace::alloc(size_t bytes) {
  if (count_ >= 32) {
    set_error("workspace: too many allocations");
    return nullptr;
  }
  if (g_alloc_budget.load() >= 0 && g_alloc_budget.fetch_sub(1) <= 0) {
    g_alloc_budget.store(0);
    set_error("workspace: allocation refused (injected failure)");
    return nullptr;
  }
  void* p = nullptr;
  cudaError_t e;
  int dev = 0;
  cudaGetDevice(&dev);
  if (t_ctx && t_ctx->device == dev) {
    // the context's size is a hard limit on what the library holds from it
    const int64_t need = (int64_t)((bytes + 255) & ~(size_t)255);
    if (t_ctx->in_use.fetch_add(need) + need > t_ctx->bytes) {
      t_ctx->in_use.fetch_sub(need);
      set_error("workspace: %zu bytes do not fit the bound context (%lld of %lld bytes in use)",
                bytes, (long long)t_ctx->in_use.load(), (long long)t_ctx->bytes);
      return nullptr;
    }
    e = cudaMallocFromPoolAsync(&p, bytes > 0 ? bytes : 16, t_ctx->pool, stream_);
    if (e != cudaSuccess) t_ctx->in_use.fetch_sub(need);
    else {
      ctx_ = t_ctx;
      ctx_bytes_ += need;
    }
  } else {
    keep_pool_memory();
    e = cudaMallocAsync(&p, bytes > 0 ? bytes : 16, stream_);
  }
  if (e != cudaSuccess) {
    set_error("workspace: allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    cudaGetLastError();
    return nullptr;
  }
  ptrs_[count_++] = p;
  bytes_ += bytes;
  return p;
}

Workspace::~Workspace() {
  for (int i = 0; i < count_; ++i) cudaFreeAsync(ptrs_[i], stream_);
  if (ctx_) context_release(ctx_, ctx_bytes_);
}

void context_release(fmgp_context* ctx, int64_t bytes) {
  if (ctx && bytes) ctx->in_use.fetch_sub(bytes);
}

// ------------------------------------------------------------ validation --
static bool kernel_ok(const fmgp_kernel* k) {
  if (!k) { set_error("kernel is NULL"); return false; }
  if (k->kind != FMGP_KERNEL_MATERN && k->kind != FMGP_KERNEL_RBF) {
    set_error("kernel kind %d unknown", k->kind);
    return false;
  }
  if (k->kind == FMGP_KERNEL_MATERN && !(k->nu == 0.5 || k->nu == 1.5 || k->nu == 2.5)) {
    set_error("Matern nu = %g unsupported (0.5, 1.5 or 2.5)", k->nu);
    return false;
  }
  if (!(k->length_scale > 0.0) || !isfinite(k->length_scale)) {
    set_error("length_scale must be positive and finite");
    return false;
  }
  if (!(k->variance > 0.0) || !isfinite(k->variance)) {
    set_error("variance must be positive and finite");
    return false;
  }
  if (!(k->nugget >= 0.0) || !isfinite(k->nugget)) {
    set_error("nugget must be non-negative and finite");
    return false;
  }
  return true;
}

static bool dtype_ok(fmgp_dtype t) {
  if (t != FMGP_F32 && t != FMGP_F64) { set_error("dtype %d unknown", (int)t); return false; }
  return true;
}

static bool prec_ok(fmgp_precision p) {
  if (p != FMGP_PREC_FP64 && p != FMGP_PREC_MIXED) {
    set_error("precision %d unknown", (int)p);
    return false;
  }
  return true;
}

#define FMGP_REQUIRE(cond, ...)       \
  do {                                \
    if (!(cond)) {                    \
      ::fmgp::set_error(__VA_ARGS__); \
      return FMGP_EINVAL;             \
    }                                 \
  } while (0)

TuneParams& tune_params() {
  static TuneParams tp;
  return tp;
}

static std::atomic<long long> g_tc_calls{0};
static int* g_tc_fallbacks_host = nullptr;  // pinned

void diag_record_tc(const int* fb_count_dev, cudaStream_t s) {
  static std::once_flag once;
  std::call_once(once, []() {
    if (cudaHostAlloc((void**)&g_tc_fallbacks_host, sizeof(int), cudaHostAllocDefault) !=
        cudaSuccess) {
      cudaGetLastError();
      g_tc_fallbacks_host = nullptr;
    }
  });
  g_tc_calls.fetch_add(1);
  if (g_tc_fallbacks_host)
    cudaMemcpyAsync(g_tc_fallbacks_host, fb_count_dev, sizeof(int), cudaMemcpyDeviceToHost, s);
}

static unsigned long long* g_visits_dev = nullptr;
static unsigned long long* g_visits_host = nullptr;  // pinned: examined, keys
static std::atomic<long long> g_visits_queries{0};

unsigned long long* diag_visits_begin(int64_t queries, cudaStream_t s) {
  static std::once_flag once;
  std::call_once(once, []() {
    if (cudaMalloc((void**)&g_visits_dev, 2 * sizeof(unsigned long long)) != cudaSuccess ||
        cudaHostAlloc((void**)&g_visits_host, 2 * sizeof(unsigned long long),
                      cudaHostAllocDefault) != cudaSuccess) {
      cudaGetLastError();
      g_visits_dev = nullptr;
      g_visits_host = nullptr;
    }
  });
  if (!g_visits_dev || !g_visits_host) return nullptr;
  if (cudaMemsetAsync(g_visits_dev, 0, 2 * sizeof(unsigned long long), s) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  g_visits_queries.store(queries);
  return g_visits_dev;
}

void diag_visits_end(cudaStream_t s) {
  if (g_visits_dev && g_visits_host)
    cudaMemcpyAsync(g_visits_host, g_visits_dev, 2 * sizeof(unsigned long long),
                    cudaMemcpyDeviceToHost, s);
}

// Precompute / LOOCV blocks in the requested precision.
static int run_blocks(BlockArgs& a, const void* X, fmgp_dtype dtype, int mode,
                      const fmgp_kernel& kern, fmgp_precision precision, Workspace& ws,
                      cudaStream_t s) {
  const int xb = dtype == FMGP_F64 ? 8 : 4;
  a.layout = block_layout(a.k, a.d, a.r, xb, false);
  const size_t bytes = precision == FMGP_PREC_FP64 ? a.layout.bytes_per_warp
                                                   : mixed_bytes_per_warp(a.k, a.d, a.r, xb);
  if (bytes > 200 * 1024 || a.layout.bytes_per_warp > 200 * 1024) {
    set_error("neighbourhood k=%d d=%d r=%d needs %zu bytes of shared memory per warp", a.k, a.d,
              a.r, std::max(bytes, a.layout.bytes_per_warp));
    return FMGP_EUNSUPPORTED;
  }
  // persistent launch (one wave of CTAs claiming neighbourhoods from a
  // counter) unless the tuning key or the autotuner chose eight waves
  a.queue = nullptr;
  if (block_persistent_for((int)precision, a.k, a.d, a.r, (int)dtype)) {
    a.queue = ws.get<unsigned long long>(1);
    if (!a.queue) return FMGP_ENOMEM;
  }
  // warps per CTA: the user's or the autotuner's choice, else (0) the
  // launchers pick the one with the most resident warps per SM
  int req = tune_params().block_warps;
  if (req == 0) req = tuned_block_warps((int)precision, a.k, a.d, a.r, (int)dtype);
  if (precision == FMGP_PREC_FP64) return launch_block_f64(a, X, dtype, mode, req, s);
  int panel = tune_params().block_panel;
  if (panel == 0) panel = tuned_block_panel((int)precision, a.k, a.d, a.r, (int)dtype);
  return run_block_mixed(a, X, dtype, mode, req, panel, kern, ws, s);
}

// flag = 1 if some value of the array is NaN or +-Inf.
template <typename T>
__global__ void nonfinite_kernel(const T* a, int64_t count, int* flag) {
  bool bad = false;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    bad |= !isfinite(a[i]);
  if (__any_sync(kFull, bad) && (threadIdx.x & 31) == 0) *flag = 1;
}

// With the tuning key "check_finite" set: scan the floating-point inputs on
// the device (stream-ordered), read the result back (synchronising `s`) and
// return FMGP_EINVAL naming the first array holding a NaN or an infinity.
// Does nothing while `s` is being captured into a CUDA graph.
int check_finite(std::initializer_list<FloatArray> arrays, cudaStream_t s) {
  if (!tune_params().check_finite) return FMGP_OK;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  FMGP_CUDA_TRY(cudaStreamIsCapturing(s, &cap));
  if (cap != cudaStreamCaptureStatusNone) return FMGP_OK;
  Workspace ws(s);
  int* flags = ws.get<int>(arrays.size());
  if (!flags) return FMGP_ENOMEM;
  FMGP_CUDA_TRY(cudaMemsetAsync(flags, 0, sizeof(int) * arrays.size(), s));
  int i = 0;
  for (const FloatArray& a : arrays) {
    if (a.p && a.count > 0) {
      const int blocks = (int)std::max<int64_t>(
          1, std::min<int64_t>(ceil_div(a.count, 256), (int64_t)num_sms() * 4));
      if (a.f64)
        FMGP_LAUNCH(nonfinite_kernel<double><<<blocks, 256, 0, s>>>((const double*)a.p, a.count, flags + i));
      else
        FMGP_LAUNCH(nonfinite_kernel<float><<<blocks, 256, 0, s>>>((const float*)a.p, a.count, flags + i));
    }
    ++i;
  }
  FMGP_CUDA_TRY(cudaGetLastError());
  int h[8] = {0};
  const size_t nb = sizeof(int) * std::min<size_t>(arrays.size(), 8);
  FMGP_CUDA_TRY(cudaMemcpyAsync(h, flags, nb, cudaMemcpyDeviceToHost, s));
  FMGP_CUDA_TRY(cudaStreamSynchronize(s));
  i = 0;
  for (const FloatArray& a : arrays) {
    if (i < 8 && h[i]) {
      set_error("%s holds a NaN or an infinity", a.name);
      return FMGP_EINVAL;
    }
    ++i;
  }
  return FMGP_OK;
}

// Deterministic single-CTA sum of the LOOCV residuals: thread t adds
// entries t, t+1024, ... in order, then a fixed tree.
__global__ void __launch_bounds__(1024) loocv_reduce(const double* resid, int64_t b, double* out) {
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

}  // namespace fmgp

using namespace fmgp;

// ------------------------------------------------ subsampled precompute --
namespace {

// flag = 1 if some rows[p] lies outside [0, n).
__global__ void check_rows_kernel(const int32_t* rows, int64_t s, int64_t n, int* flag) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < s;
       p += (int64_t)gridDim.x * blockDim.x)
    if (rows[p] < 0 || rows[p] >= n) *flag = 1;
}

// Xc[p] = X[rows[p]] (rows checked beforehand).
template <typename T>
__global__ void gather_rows_kernel(const T* X, int d, const int32_t* rows, int64_t s, T* Xc) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < s * d;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = e / d;
    Xc[e] = X[(int64_t)rows[p] * d + (e - p * d)];
  }
}

// nearest[t] = rows[pos[t]]: the training index of the chosen centre.
__global__ void centre_index_kernel(const int32_t* rows, const int32_t* pos, int64_t m,
                                    int32_t* nearest) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m;
       t += (int64_t)gridDim.x * blockDim.x)
    nearest[t] = rows[pos[t]];
}

int grid_for(int64_t count) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(count, 256), (int64_t)num_sms() * 8));
}

}  // namespace

extern "C" {

const char* fmgp_last_error(void) { return g_err; }

int fmgp_context_create(int64_t bytes, fmgp_context** out) {
  clear_error();
  if (!out || bytes < 1) {
    set_error("out must be non-NULL and bytes >= 1");
    return FMGP_EINVAL;
  }
  *out = nullptr;
  int dev = 0;
  FMGP_CUDA_TRY(cudaGetDevice(&dev));
  cudaMemPoolProps props;
  memset(&props, 0, sizeof(props));
  props.allocType = cudaMemAllocationTypePinned;
  props.handleTypes = cudaMemHandleTypeNone;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  // whole 2 MiB chunks: the pool reserves device memory in units of its
  // allocation granularity
  bytes = (bytes + (2 << 20) - 1) / (2 << 20) * (2 << 20);
  props.maxSize = (size_t)bytes;
  cudaMemPool_t pool;
  FMGP_CUDA_TRY(cudaMemPoolCreate(&pool, &props));
  // keep what the pool holds between calls, and take the whole size now so
  // that later calls are served from memory already reserved
  uint64_t thr = UINT64_MAX;
  cudaError_t e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  void* p = nullptr;
  if (e == cudaSuccess) e = cudaMallocFromPoolAsync(&p, (size_t)bytes, pool, 0);
  if (e == cudaSuccess) e = cudaFreeAsync(p, 0);
  if (e == cudaSuccess) e = cudaStreamSynchronize(0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    cudaMemPoolDestroy(pool);
    set_error("context: cannot reserve %lld device bytes: %s", (long long)bytes,
              cudaGetErrorString(e));
    return FMGP_ENOMEM;
  }
  fmgp_context* c = new fmgp_context();
  c->device = dev;
  c->pool = pool;
  c->bytes = bytes;
  *out = c;
  return FMGP_OK;
}

int fmgp_context_bind(fmgp_context* ctx) {
  clear_error();
  t_ctx = ctx;
  return FMGP_OK;
}

int64_t fmgp_context_bytes_in_use(const fmgp_context* ctx) {
  return ctx ? ctx->in_use.load() : -1;
}

int fmgp_context_destroy(fmgp_context* ctx) {
  clear_error();
  if (!ctx) {
    set_error("context is NULL");
    return FMGP_EINVAL;
  }
  if (t_ctx == ctx) t_ctx = nullptr;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();  // stream-ordered frees into the pool have completed
  const cudaError_t e = cudaMemPoolDestroy(ctx->pool);
  cudaSetDevice(prev);
  delete ctx;
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemPoolDestroy");
  return FMGP_OK;
}
const char* fmgp_version(void) { return "0.1.0"; }
uint64_t fmgp_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

int64_t fmgp_diag_counter(int32_t which) {
  if (which == 0) return (int64_t)g_launches.load();
  if (which == 1) return (int64_t)g_tc_calls.load();
  if (which == 2) return g_tc_fallbacks_host ? (int64_t)*(volatile int*)g_tc_fallbacks_host : -1;
  if (which == 3 || which == 4)
    return g_visits_host ? (int64_t)((volatile unsigned long long*)g_visits_host)[which - 3] : -1;
  if (which == 5) return g_visits_host ? (int64_t)g_visits_queries.load() : -1;
  return -1;
}

int fmgp_tune_set(const char* key, double value) {
  if (!key) { set_error("key is NULL"); return FMGP_EINVAL; }
  TuneParams& tp = tune_params();
  const std::string k(key);
  if (k == "grid_target") {
    if (!(value >= 1.0 && value <= 4096.0)) { set_error("grid_target out of range"); return FMGP_EINVAL; }
    tp.grid_target = value;
  } else if (k == "block_warps") {
    if (!(value >= 0 && value <= 8)) { set_error("block_warps out of range"); return FMGP_EINVAL; }
    tp.block_warps = (int)value;
  } else if (k == "block_panel") {
    if (!(value == 0 || value == 4 || value == 8)) { set_error("block_panel must be 0, 4 or 8"); return FMGP_EINVAL; }
    tp.block_panel = (int)value;
  } else if (k == "block_persistent") {
    if (!(value == -1 || value == 0 || value == 1)) { set_error("block_persistent must be -1, 0 or 1"); return FMGP_EINVAL; }
    tp.block_persistent = (int)value;
  } else if (k == "tensor_cores") {
    tp.use_tensor_cores = value != 0.0;
  } else if (k == "tc_fused_select") {
    tp.tc_fused_select = value != 0.0;
  } else if (k == "tc_fused_r") {
    if (!(value == 0 || value == 8 || value == 16 || value == 32)) { set_error("tc_fused_r must be 0, 8, 16 or 32"); return FMGP_EINVAL; }
    tp.tc_fused_r = (int)value;
  } else if (k == "count_visits") {
    tp.count_visits = value != 0.0;
  } else if (k == "tc_oversample") {
    if (!(value >= 2 && value <= 4)) { set_error("tc_oversample out of range [2, 4]"); return FMGP_EINVAL; }
    tp.tc_oversample = (int)value;
  } else if (k == "tc_wait_ns") {
    if (!(value >= 0 && value <= 2e9)) { set_error("tc_wait_ns out of range [0, 2e9]"); return FMGP_EINVAL; }
    tp.tc_wait_ns = (int64_t)value;
  } else if (k == "check_finite") {
    tp.check_finite = value != 0.0;
  } else if (k == "fail_alloc_after") {
    if (!(value >= -1 && value <= 1e9)) { set_error("fail_alloc_after out of range"); return FMGP_EINVAL; }
    g_alloc_budget.store((long long)value);
  } else if (k == "tc_chunk_queries") {
    if (!(value >= 0 && value <= 2147483647.0)) { set_error("tc_chunk_queries out of range"); return FMGP_EINVAL; }
    tp.tc_chunk_queries = (int64_t)value;
  } else {
    set_error("unknown tuning key '%s'", key);
    return FMGP_EINVAL;
  }
  return FMGP_OK;
}

double fmgp_tune_get(const char* key) {
  if (!key) return -1.0;
  const TuneParams& tp = tune_params();
  const std::string k(key);
  if (k == "grid_target") return tp.grid_target;
  if (k == "block_warps") return tp.block_warps;
  if (k == "block_panel") return tp.block_panel;
  if (k == "block_persistent") return tp.block_persistent;
  if (k == "tensor_cores") return tp.use_tensor_cores ? 1.0 : 0.0;
  if (k == "tc_fused_select") return tp.tc_fused_select ? 1.0 : 0.0;
  if (k == "tc_oversample") return tp.tc_oversample;
  if (k == "count_visits") return tp.count_visits ? 1.0 : 0.0;
  if (k == "tc_fused_r") return tp.tc_fused_r;
  if (k == "tc_chunk_queries") return (double)tp.tc_chunk_queries;
  if (k == "fail_alloc_after") return (double)g_alloc_budget.load();
  if (k == "check_finite") return tp.check_finite ? 1.0 : 0.0;
  if (k == "tc_wait_ns") return (double)tp.tc_wait_ns;
  return -1.0;
}

int fmgp_build_knn(const void* X, fmgp_dtype dtype, int64_t n, int32_t d, int32_t kq,
                   int32_t* nbr_out, double* dist_out, int32_t flags, void* stream) {
  clear_error();
  if (!dtype_ok(dtype)) return FMGP_EINVAL;
  FMGP_REQUIRE(X && nbr_out, "X and nbr_out must be non-NULL");
  FMGP_REQUIRE(n >= 2 && n < INT32_MAX, "n = %lld out of range [2, 2^31)", (long long)n);
  FMGP_REQUIRE(d >= 1, "d = %d must be >= 1", d);
  FMGP_REQUIRE(kq >= 1 && kq <= n - 1 && kq <= kMaxK, "kq = %d must be in [1, min(n-1, %d)]",
               kq, kMaxK);
  FMGP_REQUIRE(flags == 0, "flags must be 0");
  cudaStream_t s = (cudaStream_t)stream;
  if (int fc = check_finite({{X, dtype == FMGP_F64, n * (int64_t)d, "X"}}, s)) return fc;
  Workspace ws(s);
  TuneParams tp = tune_params();
  tp.grid_target = grid_target_for(d, kq);
  return knn_self(X, dtype, n, d, kq, nbr_out, dist_out, tp, ws, s);
}

static int validate_block_args(const void* X, fmgp_dtype dtype, const double* Y, int64_t n,
                               int32_t d, int32_t r, const int32_t* nbr, int32_t nbr_ld,
                               const fmgp_kernel* kernel, fmgp_precision precision) {
  if (!dtype_ok(dtype) || !kernel_ok(kernel) || !prec_ok(precision)) return FMGP_EINVAL;
  FMGP_REQUIRE(X && Y && nbr, "X, Y and nbr must be non-NULL");
  FMGP_REQUIRE(n >= 1 && n < INT32_MAX, "n = %lld out of range [1, 2^31)", (long long)n);
  FMGP_REQUIRE(d >= 1, "d = %d must be >= 1", d);
  FMGP_REQUIRE(r >= 1, "r = %d must be >= 1", r);
  (void)nbr_ld;
  return FMGP_OK;
}

int fmgp_precompute(const void* X, fmgp_dtype dtype, const double* Y, int64_t n, int32_t d,
                    int32_t r, const int32_t* nbr, int32_t nbr_ld, int32_t k,
                    const fmgp_kernel* kernel, fmgp_precision precision, void* C_out,
                    int8_t* status_out, void* stream) {
  clear_error();
  int rc = validate_block_args(X, dtype, Y, n, d, r, k > 1 ? nbr : (const int32_t*)X, nbr_ld,
                               kernel, precision);
  if (rc) return rc;
  FMGP_REQUIRE(C_out, "C_out must be non-NULL");
  FMGP_REQUIRE(k >= 1 && k <= n && k <= kMaxK, "k = %d must be in [1, min(n, %d)]", k, kMaxK);
  FMGP_REQUIRE(nbr_ld >= k - 1 && nbr_ld >= 0, "nbr_ld = %d must be >= k-1 = %d", nbr_ld, k - 1);
  cudaStream_t s = (cudaStream_t)stream;
  if (int fc = check_finite({{X, dtype == FMGP_F64, n * (int64_t)d, "X"}, {Y, true, n * (int64_t)r, "Y"}}, s)) return fc;
  Workspace ws(s);
  int* fails = ws.get<int>(1);
  if (!fails) return FMGP_ENOMEM;
  FMGP_CUDA_TRY(cudaMemsetAsync(fails, 0, sizeof(int), s));
  BlockArgs a{};
  a.Y = Y;
  a.nbr = nbr;
  a.C = C_out;
  a.status = status_out;
  a.fail_count = fails;
  a.n = n;
  a.count = n;
  a.d = d;
  a.r = r;
  a.ld = nbr_ld;
  a.k = k;
  a.kp = make_kparams(*kernel);
  rc = run_blocks(a, X, dtype, kModePrecompute, *kernel, precision, ws, s);
  if (rc) return rc;
  if (!status_out) {
    int h = 0;
    FMGP_CUDA_TRY(cudaMemcpyAsync(&h, fails, sizeof(int), cudaMemcpyDeviceToHost, s));
    FMGP_CUDA_TRY(cudaStreamSynchronize(s));
    if (h) {
      set_error("%d neighbourhood blocks were not positive definite", h);
      return FMGP_ENOTSPD;
    }
  }
  return FMGP_OK;
}

int fmgp_predict(const void* X, fmgp_dtype dtype, int64_t n, int32_t d, const int32_t* nbr,
                 int32_t nbr_ld, const void* C, int32_t k, int32_t r, const fmgp_kernel* kernel,
                 fmgp_precision precision, const void* Z, int64_t m, double* Yhat_out,
                 int32_t* nearest_out, void* stream) {
  clear_error();
  if (!dtype_ok(dtype) || !kernel_ok(kernel) || !prec_ok(precision)) return FMGP_EINVAL;
  FMGP_REQUIRE(m >= 0, "m = %lld must be >= 0", (long long)m);
  FMGP_REQUIRE(X && C, "X and C must be non-NULL");
  FMGP_REQUIRE(n >= 1 && n < INT32_MAX, "n = %lld out of range [1, 2^31)", (long long)n);
  FMGP_REQUIRE(d >= 1 && r >= 1, "d and r must be >= 1");
  FMGP_REQUIRE(k >= 1 && k <= n && k <= kMaxK, "k = %d must be in [1, min(n, %d)]", k, kMaxK);
  FMGP_REQUIRE(k == 1 || nbr, "nbr must be non-NULL when k > 1");
  FMGP_REQUIRE(nbr_ld >= k - 1, "nbr_ld = %d must be >= k-1", nbr_ld);
  if (m == 0) return FMGP_OK;
  FMGP_REQUIRE(Z && Yhat_out, "Z and Yhat_out must be non-NULL");
  cudaStream_t s = (cudaStream_t)stream;
  if (int fc = check_finite({{X, dtype == FMGP_F64, n * (int64_t)d, "X"}, {Z, dtype == FMGP_F64, m * (int64_t)d, "Z"}}, s)) return fc;
  Workspace ws(s);
  int32_t* near = nearest_out;
  if (!near) {
    near = ws.get<int32_t>(m);
    if (!near) return FMGP_ENOMEM;
  }
  int rc = nearest_train(X, dtype, n, d, Z, m, near, tune_params(), ws, s);
  if (rc) return rc;
  return gather_dot(X, dtype, n, d, nbr, nbr_ld, C, k, r, make_kparams(*kernel), *kernel,
                    precision, Z, m, near, Yhat_out, ws, s);
}

// Enqueue the LOOCV objective: residuals, then Q (the mean over the batch,
// in a fixed order) into the device double qd and the number of failed blocks
// into the device int fails (both written on `s`).
static int loocv_enqueue(const void* X, fmgp_dtype dtype, const double* Y, int64_t n, int32_t d,
                         int32_t r, const int32_t* nbr, int32_t nbr_ld, int32_t k,
                         const int64_t* batch, int64_t b, const fmgp_kernel* kernel,
                         fmgp_precision precision, double* qd, int* fails, double* resid_out,
                         Workspace& ws, cudaStream_t s) {
  double* resid = resid_out ? resid_out : ws.get<double>(b);
  if (!resid) return FMGP_ENOMEM;
  FMGP_CUDA_TRY(cudaMemsetAsync(fails, 0, sizeof(int), s));
  BlockArgs a{};
  a.Y = Y;
  a.nbr = nbr;
  a.batch = batch;
  a.resid = resid;
  a.fail_count = fails;
  a.n = n;
  a.count = b;
  a.d = d;
  a.r = r;
  a.ld = nbr_ld;
  a.k = k;
  a.kp = make_kparams(*kernel);
  int rc = run_blocks(a, X, dtype, kModeLoocv, *kernel, precision, ws, s);
  if (rc) return rc;
  FMGP_LAUNCH(loocv_reduce<<<1, 1024, 0, s>>>(resid, b, qd));
  FMGP_CUDA_TRY(cudaGetLastError());
  return FMGP_OK;
}

static int loocv_validate(const void* X, fmgp_dtype dtype, const double* Y, int64_t n, int32_t d,
                          int32_t r, const int32_t* nbr, int32_t nbr_ld, int32_t k,
                          const int64_t* batch, int64_t b, const fmgp_kernel* kernel,
                          fmgp_precision precision, const double* Q_out) {
  int rc = validate_block_args(X, dtype, Y, n, d, r, nbr, nbr_ld, kernel, precision);
  if (rc) return rc;
  FMGP_REQUIRE(Q_out && batch, "Q_out and batch must be non-NULL");
  FMGP_REQUIRE(n >= 2, "LOOCV needs n >= 2");
  FMGP_REQUIRE(k >= 1 && k <= n - 1 && k <= kMaxK, "k = %d must be in [1, min(n-1, %d)]", k,
               kMaxK);
  FMGP_REQUIRE(nbr_ld >= k, "nbr_ld = %d must be >= k = %d", nbr_ld, k);
  FMGP_REQUIRE(b >= 1, "batch size b = %lld must be >= 1", (long long)b);
  return FMGP_OK;
}

int fmgp_loocv_objective(const void* X, fmgp_dtype dtype, const double* Y, int64_t n,
                         int32_t d, int32_t r, const int32_t* nbr, int32_t nbr_ld, int32_t k,
                         const int64_t* batch, int64_t b, const fmgp_kernel* kernel,
                         fmgp_precision precision, double* Q_out, double* resid_out,
                         void* stream) {
  clear_error();
  int rc = loocv_validate(X, dtype, Y, n, d, r, nbr, nbr_ld, k, batch, b, kernel, precision, Q_out);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if (int fc = check_finite({{X, dtype == FMGP_F64, n * (int64_t)d, "X"}, {Y, true, n * (int64_t)r, "Y"}}, s)) return fc;
  Workspace ws(s);
  int* fails = ws.get<int>(1);
  double* qd = ws.get<double>(1);
  if (!fails || !qd) return FMGP_ENOMEM;
  rc = loocv_enqueue(X, dtype, Y, n, d, r, nbr, nbr_ld, k, batch, b, kernel, precision, qd, fails,
                     resid_out, ws, s);
  if (rc) return rc;
  int h = 0;
  FMGP_CUDA_TRY(cudaMemcpyAsync(Q_out, qd, sizeof(double), cudaMemcpyDeviceToHost, s));
  FMGP_CUDA_TRY(cudaMemcpyAsync(&h, fails, sizeof(int), cudaMemcpyDeviceToHost, s));
  FMGP_CUDA_TRY(cudaStreamSynchronize(s));
  if (h) {
    set_error("%d LOOCV blocks were not positive definite", h);
    return FMGP_ENOTSPD;
  }
  return FMGP_OK;
}

int fmgp_loocv_objective_device(const void* X, fmgp_dtype dtype, const double* Y, int64_t n,
                                int32_t d, int32_t r, const int32_t* nbr, int32_t nbr_ld,
                                int32_t k, const int64_t* batch, int64_t b,
                                const fmgp_kernel* kernel, fmgp_precision precision,
                                double* Q_dev, int32_t* fails_dev, double* resid_out,
                                void* stream) {
  clear_error();
  int rc = loocv_validate(X, dtype, Y, n, d, r, nbr, nbr_ld, k, batch, b, kernel, precision, Q_dev);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if (int fc = check_finite({{X, dtype == FMGP_F64, n * (int64_t)d, "X"}, {Y, true, n * (int64_t)r, "Y"}}, s)) return fc;
  Workspace ws(s);
  int* fails = fails_dev ? (int*)fails_dev : ws.get<int>(1);
  if (!fails) return FMGP_ENOMEM;
  return loocv_enqueue(X, dtype, Y, n, d, r, nbr, nbr_ld, k, batch, b, kernel, precision, Q_dev,
                       fails, resid_out, ws, s);
}

int fmgp_muygps_predict(const void* X, fmgp_dtype dtype, const double* Y, int64_t n, int32_t d,
                        int32_t r, const void* Z, int64_t m, int32_t k, const fmgp_kernel* kernel,
                        fmgp_precision precision, double* Yhat_out, int32_t* nbr_out,
                        void* stream) {
  clear_error();
  if (!dtype_ok(dtype) || !kernel_ok(kernel) || !prec_ok(precision)) return FMGP_EINVAL;
  FMGP_REQUIRE(X && Y, "X and Y must be non-NULL");
  FMGP_REQUIRE(n >= 1 && n < INT32_MAX, "n = %lld out of range [1, 2^31)", (long long)n);
  FMGP_REQUIRE(d >= 1 && r >= 1, "d and r must be >= 1");
  FMGP_REQUIRE(k >= 1 && k <= n && k <= kMaxK, "k = %d must be in [1, min(n, %d)]", k, kMaxK);
  FMGP_REQUIRE(m >= 0, "m = %lld must be >= 0", (long long)m);
  if (m == 0) return FMGP_OK;
  FMGP_REQUIRE(Z && Yhat_out, "Z and Yhat_out must be non-NULL");
  cudaStream_t s = (cudaStream_t)stream;
  if (int fc = check_finite({{X, dtype == FMGP_F64, n * (int64_t)d, "X"}, {Y, true, n * (int64_t)r, "Y"}, {Z, dtype == FMGP_F64, m * (int64_t)d, "Z"}}, s)) return fc;
  Workspace ws(s);
  int32_t* nbr = nbr_out ? nbr_out : ws.get<int32_t>((size_t)m * k);
  int* fails = ws.get<int>(1);
  if (!nbr || !fails) return FMGP_ENOMEM;
  TuneParams tp = tune_params();
  tp.grid_target = grid_target_for(d, k);
  int rc = knn_query(X, dtype, n, d, Z, m, k, nbr, nullptr, tp, ws, s);
  if (rc) return rc;
  FMGP_CUDA_TRY(cudaMemsetAsync(fails, 0, sizeof(int), s));
  BlockArgs a{};
  a.Y = Y;
  a.nbr = nbr;
  a.fail_count = fails;
  a.Zq = Z;
  a.yhat = Yhat_out;
  a.n = n;
  a.count = m;
  a.d = d;
  a.r = r;
  a.ld = k;
  a.k = k;
  a.kp = make_kparams(*kernel);
  if (precision == FMGP_PREC_MIXED) {
    float2* Zdf = ws.get<float2>((size_t)m * d);
    if (!Zdf) return FMGP_ENOMEM;
    rc = to_df(Z, dtype == FMGP_F64, m * d, Zdf, s);
    if (rc) return rc;
    a.Zdf = Zdf;
  }
  return run_blocks(a, X, dtype, kModeMuygps, *kernel, precision, ws, s);
}

int fmgp_precompute_rows(const void* X, fmgp_dtype dtype, const double* Y, int64_t n, int32_t d,
                         int32_t r, const int32_t* nbr, int32_t nbr_ld, int32_t k,
                         const int32_t* rows, int64_t s_rows, const fmgp_kernel* kernel,
                         fmgp_precision precision, void* C_out, int8_t* status_out,
                         void* stream) {
  clear_error();
  int rc = validate_block_args(X, dtype, Y, n, d, r, k > 1 ? nbr : (const int32_t*)X, nbr_ld,
                               kernel, precision);
  if (rc) return rc;
  FMGP_REQUIRE(s_rows >= 0 && s_rows < INT32_MAX, "s = %lld out of range [0, 2^31)",
               (long long)s_rows);
  if (s_rows == 0) return FMGP_OK;
  FMGP_REQUIRE(rows && C_out, "rows and C_out must be non-NULL");
  FMGP_REQUIRE(k >= 1 && k <= n && k <= kMaxK, "k = %d must be in [1, min(n, %d)]", k, kMaxK);
  FMGP_REQUIRE(nbr_ld >= k - 1 && nbr_ld >= 0, "nbr_ld = %d must be >= k-1 = %d", nbr_ld, k - 1);
  cudaStream_t s = (cudaStream_t)stream;
  if (int fc = check_finite({{X, dtype == FMGP_F64, n * (int64_t)d, "X"}, {Y, true, n * (int64_t)r, "Y"}}, s)) return fc;
  Workspace ws(s);
  int* fails = ws.get<int>(1);
  if (!fails) return FMGP_ENOMEM;
  FMGP_CUDA_TRY(cudaMemsetAsync(fails, 0, sizeof(int), s));
  BlockArgs a{};
  a.Y = Y;
  a.nbr = nbr;
  a.C = C_out;
  a.status = status_out;
  a.fail_count = fails;
  a.rows = rows;
  a.n = n;
  a.count = s_rows;
  a.d = d;
  a.r = r;
  a.ld = nbr_ld;
  a.k = k;
  a.kp = make_kparams(*kernel);
  rc = run_blocks(a, X, dtype, kModePrecompute, *kernel, precision, ws, s);
  if (rc) return rc;
  if (!status_out) {
    int h = 0;
    FMGP_CUDA_TRY(cudaMemcpyAsync(&h, fails, sizeof(int), cudaMemcpyDeviceToHost, s));
    FMGP_CUDA_TRY(cudaStreamSynchronize(s));
    if (h) {
      set_error("%d neighbourhood blocks were not positive definite or had a bad index", h);
      return FMGP_ENOTSPD;
    }
  }
  return FMGP_OK;
}

int fmgp_predict_rows(const void* X, fmgp_dtype dtype, int64_t n, int32_t d, const int32_t* nbr,
                      int32_t nbr_ld, const int32_t* rows, int64_t s_rows, const void* C,
                      int32_t k, int32_t r, const fmgp_kernel* kernel, fmgp_precision precision,
                      const void* Z, int64_t m, double* Yhat_out, int32_t* nearest_out,
                      void* stream) {
  clear_error();
  if (!dtype_ok(dtype) || !kernel_ok(kernel) || !prec_ok(precision)) return FMGP_EINVAL;
  FMGP_REQUIRE(m >= 0, "m = %lld must be >= 0", (long long)m);
  FMGP_REQUIRE(X && C && rows, "X, C and rows must be non-NULL");
  FMGP_REQUIRE(n >= 1 && n < INT32_MAX, "n = %lld out of range [1, 2^31)", (long long)n);
  FMGP_REQUIRE(s_rows >= 1 && s_rows <= n, "s = %lld must be in [1, n]", (long long)s_rows);
  FMGP_REQUIRE(d >= 1 && r >= 1, "d and r must be >= 1");
  FMGP_REQUIRE(k >= 1 && k <= n && k <= kMaxK, "k = %d must be in [1, min(n, %d)]", k, kMaxK);
  FMGP_REQUIRE(k == 1 || nbr, "nbr must be non-NULL when k > 1");
  FMGP_REQUIRE(nbr_ld >= k - 1, "nbr_ld = %d must be >= k-1", nbr_ld);
  if (m == 0) return FMGP_OK;
  FMGP_REQUIRE(Z && Yhat_out, "Z and Yhat_out must be non-NULL");
  cudaStream_t s = (cudaStream_t)stream;
  if (int fc = check_finite({{X, dtype == FMGP_F64, n * (int64_t)d, "X"}, {Z, dtype == FMGP_F64, m * (int64_t)d, "Z"}}, s)) return fc;
  Workspace ws(s);
  int* flag = ws.get<int>(1);
  const size_t xb = dtype == FMGP_F64 ? 8 : 4;
  void* Xc = ws.alloc((size_t)s_rows * d * xb);
  int32_t* pos = ws.get<int32_t>(m);
  int32_t* near = nearest_out ? nearest_out : ws.get<int32_t>(m);
  if (!flag || !Xc || !pos || !near) return FMGP_ENOMEM;
  FMGP_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(int), s));
  FMGP_LAUNCH(check_rows_kernel<<<grid_for(s_rows), 256, 0, s>>>(rows, s_rows, n, flag));
  int h = 0;
  FMGP_CUDA_TRY(cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  FMGP_CUDA_TRY(cudaStreamSynchronize(s));
  FMGP_REQUIRE(h == 0, "rows holds an index outside [0, n)");
  if (dtype == FMGP_F64)
    FMGP_LAUNCH(gather_rows_kernel<double><<<grid_for(s_rows * d), 256, 0, s>>>(
        (const double*)X, d, rows, s_rows, (double*)Xc));
  else
    FMGP_LAUNCH(gather_rows_kernel<float><<<grid_for(s_rows * d), 256, 0, s>>>(
        (const float*)X, d, rows, s_rows, (float*)Xc));
  int rc = nearest_train(Xc, dtype, s_rows, d, Z, m, pos, tune_params(), ws, s);
  if (rc) return rc;
  FMGP_LAUNCH(centre_index_kernel<<<grid_for(m), 256, 0, s>>>(rows, pos, m, near));
  return gather_dot(X, dtype, n, d, nbr, nbr_ld, C, k, r, make_kparams(*kernel), *kernel,
                    precision, Z, m, near, Yhat_out, ws, s, pos);
}

}  // extern "C"
