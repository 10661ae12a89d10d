// Shared device/host helpers of libfmgp (CUDA path only).
#pragma once
#include <initializer_list>
#include <cuda_runtime.h>
#include <stdint.h>
#include <limits.h>
#include <string>
#include "fmgp.h"

namespace fmgp {

constexpr int kWarp = 32;
constexpr unsigned kFull = 0xffffffffu;
constexpr int kMaxK = 160;  // largest neighbourhood a block kernel handles (5 slots of 32)

// Kernel hyperparameters as the device sees them.  phi(D) is the correlation
// at squared distance D (Eq. 3; RBF as its nu -> infinity limit).
struct KParams {
  int kind;          // FMGP_KERNEL_MATERN / FMGP_KERNEL_RBF
  int nu2;           // 2*nu for Matern: 1, 3 or 5
  double inv_rho;    // 1 / rho
  double half_inv_rho2;  // 1 / (2 rho^2)
  double var;        // sigma^2
  double diag;       // sigma^2 (1 + tau^2)
  float inv_rho_f, half_inv_rho2_f, var_f, diag_f;
};

inline KParams make_kparams(const fmgp_kernel& k) {
  KParams p;
  p.kind = k.kind;
  p.nu2 = (int)(2.0 * k.nu + 0.5);
  p.inv_rho = 1.0 / k.length_scale;
  p.half_inv_rho2 = 0.5 / (k.length_scale * k.length_scale);
  p.var = k.variance;
  p.diag = k.variance * (1.0 + k.nugget);
  p.inv_rho_f = (float)p.inv_rho;
  p.half_inv_rho2_f = (float)p.half_inv_rho2;
  p.var_f = (float)p.var;
  p.diag_f = (float)p.diag;
  return p;
}

// Matern closed forms at half-integer nu (Eq. 3 with K_nu for nu = 1/2, 3/2,
// 5/2) and the RBF limit, in FP64 with CUDA's exp/sqrt.
__device__ __forceinline__ double phi64(const KParams& p, double D) {
  if (p.kind == FMGP_KERNEL_RBF) return exp(-D * p.half_inv_rho2);
  double u = sqrt(D) * p.inv_rho;
  if (p.nu2 == 1) return exp(-u);
  if (p.nu2 == 3) {
    const double s3 = 1.7320508075688772;
    double a = s3 * u;
    return (1.0 + a) * exp(-a);
  }
  const double s5 = 2.23606797749979;
  double a = s5 * u;
  return (1.0 + a + a * a * (1.0 / 3.0)) * exp(-a);
}

__device__ __forceinline__ float phi32(const KParams& p, float D) {
  if (p.kind == FMGP_KERNEL_RBF) return __expf(-D * p.half_inv_rho2_f);
  float u = sqrtf(D) * p.inv_rho_f;
  if (p.nu2 == 1) return __expf(-u);
  if (p.nu2 == 3) {
    float a = 1.7320508f * u;
    return (1.0f + a) * __expf(-a);
  }
  float a = 2.2360680f * u;
  return (1.0f + a + a * a * (1.0f / 3.0f)) * __expf(-a);
}

template <typename T> __device__ __forceinline__ double ld64(const T* p) { return (double)(*p); }

// Canonical ranking key (library-wide convention): FP64, left to right, each
// operation rounded on its own; the first term is t0*t0 (0 + t0*t0 is exact).
template <typename T>
__device__ __forceinline__ double canon_key(const double* q, const T* x, int d) {
  double t = __dsub_rn(q[0], (double)x[0]);
  double s = __dmul_rn(t, t);
  for (int j = 1; j < d; ++j) {
    t = __dsub_rn(q[j], (double)x[j]);
    s = __dadd_rn(s, __dmul_rn(t, t));
  }
  return s;
}

// (key, index) lexicographic order on the IEEE bit patterns of non-negative
// doubles (which order like unsigned integers), avoiding FP64 compares.
__device__ __forceinline__ bool key_less(unsigned long long ka, int ia, unsigned long long kb,
                                         int ib) {
  return ka < kb || (ka == kb && ia < ib);
}

// Round a non-negative double given by its bits up to a float (>= value),
// using integer operations only.  Used to compare FP32 lower bounds with FP64
// keys without FP64 instructions.
__device__ __forceinline__ float key_bits_to_float_up(unsigned long long b) {
  if (b >= 0x7ff0000000000000ull) return __int_as_float(0x7f800000);  // inf / nan -> inf
  int e = (int)(b >> 52);
  unsigned long long mant = b & 0xfffffffffffffull;
  int fe = e - 1023 + 127;
  if (fe >= 255) return __int_as_float(0x7f800000);
  if (fe <= 0) return 1.1754944e-38f;  // below FLT_MIN: FLT_MIN is an upper bound
  unsigned int fm = (unsigned int)(mant >> 29);
  unsigned int bits = ((unsigned int)fe << 23) | fm;
  return __uint_as_float(bits + 1u);  // next float up (truncation was downward)
}

__device__ __forceinline__ unsigned long long dbits(double x) {
  return (unsigned long long)__double_as_longlong(x);
}

// ------------------------------------------------------------------ host --
// Every kernel launch of the library goes through FMGP_LAUNCH so that
// fmgp_kernel_launches() can report how many kernels were enqueued.
void note_launch();
#define FMGP_LAUNCH(...)   \
  do {                     \
    __VA_ARGS__;           \
    ::fmgp::note_launch(); \
  } while (0)

void set_error(const char* fmt, ...);
// Empty this thread's error message (every entry point starts with it).
void clear_error();
int cuda_fail(cudaError_t e, const char* what);

// Raise a kernel's dynamic shared-memory limit to at least `bytes`, calling
// cudaFuncSetAttribute only when the cached limit (per device and function)
// is too low, so that steady-state launches (and stream capture into CUDA
// graphs after a warm-up call) make no attribute calls.
cudaError_t ensure_smem(const void* func, size_t bytes);

// CTAs of `func` (threads per CTA, dynamic shared memory bytes) resident per
// SM, from the CUDA occupancy calculator (raises the function's dynamic
// shared-memory limit first; cached per device).  0 if it cannot run.
int active_ctas(const void* func, int threads, size_t smem);

#define FMGP_CUDA_TRY(call)                                  \
  do {                                                       \
    cudaError_t _e = (call);                                 \
    if (_e != cudaSuccess) return ::fmgp::cuda_fail(_e, #call); \
  } while (0)

// Stream-ordered workspace: every allocation is returned on the same stream
// when the object goes out of scope.
class Workspace {
 public:
  explicit Workspace(cudaStream_t s) : stream_(s) {}
  ~Workspace();
  // Returns nullptr (and records the error) on failure.
  void* alloc(size_t bytes);
  template <typename T> T* get(size_t count) { return (T*)alloc(count * sizeof(T)); }
  // Hand every allocation so far to the caller (who then frees them, and
  // returns `*ctx_bytes` to `*ctx` with context_release when ctx is set);
  // returns the count.
  int detach(void** out, int max, fmgp_context** ctx, int64_t* ctx_bytes) {
    int c = count_ < max ? count_ : max;
    for (int i = 0; i < c; ++i) out[i] = ptrs_[i];
    *ctx = ctx_;
    *ctx_bytes = ctx_bytes_;
    count_ = 0;
    ctx_bytes_ = 0;
    return c;
  }
  size_t bytes() const { return bytes_; }

 private:
  size_t bytes_ = 0;
  cudaStream_t stream_;
  void* ptrs_[32];
  int count_ = 0;
  fmgp_context* ctx_ = nullptr;  // the context the allocations came from, if any
  int64_t ctx_bytes_ = 0;        // bytes charged to it
};

// Give bytes charged to a workspace context back to it (a resident model's
// buffers when the model is destroyed).
void context_release(fmgp_context* ctx, int64_t bytes);

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// A floating-point input array for check_finite (FP64 or FP32, `count` values).
struct FloatArray {
  const void* p;
  bool f64;
  int64_t count;
  const char* name;
};
// With the tuning key "check_finite" set: scan the arrays on the device,
// synchronise `s`, and return FMGP_EINVAL naming the first one holding a NaN
// or an infinity; otherwise (and while `s` is being captured) FMGP_OK.
int check_finite(std::initializer_list<FloatArray> arrays, cudaStream_t s);

// Diagnostics: count a tensor-core kNN call and copy its number of queries
// that needed the exact fallback (device int) to a host slot read by
// fmgp_diag_counter after the stream has completed.
void diag_record_tc(const int* fb_count_dev, cudaStream_t s);
// Grid kNN visit counters: zeroed device counters for a call over `queries`
// queries (null if they cannot be had), and their copy to the host slots read
// by fmgp_diag_counter once the stream has completed.
unsigned long long* diag_visits_begin(int64_t queries, cudaStream_t s);
void diag_visits_end(cudaStream_t s);
int num_sms();

}  // namespace fmgp
