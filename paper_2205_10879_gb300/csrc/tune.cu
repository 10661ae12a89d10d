// Autotuner: times candidate launch shapes on the caller's own data and
// caches the fastest per problem key.  Only speed depends on the choice:
// every shape computes identical results.
//   block kernels (precompute / LOOCV): warps per CTA, Cholesky panel width
//     (mixed, k <= 64) and persistent or multi-wave grid, key (precision, k, d, r, dtype)
//   grid kNN (d <= 3): mean points per cell, key (d, kq)
#include <map>
#include <mutex>
#include <tuple>
#include <vector>
#include "block.cuh"
#include "knn.cuh"

namespace fmgp {
namespace {

std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int>, int> g_warps;
std::map<std::tuple<int, int, int, int, int>, int> g_panel;
std::map<std::tuple<int, int, int, int, int>, int> g_persist;
std::map<std::tuple<int, int>, double> g_grid;

}  // namespace

int tuned_block_warps(int prec, int k, int d, int r, int dtype) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_warps.find({prec, k, d, r, dtype});
  return it == g_warps.end() ? 0 : it->second;
}

int tuned_block_panel(int prec, int k, int d, int r, int dtype) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_panel.find({prec, k, d, r, dtype});
  return it == g_panel.end() ? 0 : it->second;
}

bool block_persistent_for(int prec, int k, int d, int r, int dtype) {
  const int p = tune_params().block_persistent;
  if (p >= 0) return p != 0;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_persist.find({prec, k, d, r, dtype});
  return it == g_persist.end() ? true : it->second != 0;
}

double grid_target_for(int d, int kq) {
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_grid.find({d, kq});
    if (it != g_grid.end()) return it->second;
  }
  return tune_params().grid_target;
}

}  // namespace fmgp

using namespace fmgp;

namespace {

// Mean of `reps` timed calls of f() on stream s (after one untimed call).
template <typename F>
int time_ms(cudaStream_t s, int reps, F&& f, float* out) {
  int rc = f();
  if (rc) return rc;
  cudaEvent_t e0, e1;
  FMGP_CUDA_TRY(cudaEventCreate(&e0));
  FMGP_CUDA_TRY(cudaEventCreate(&e1));
  FMGP_CUDA_TRY(cudaEventRecord(e0, s));
  for (int i = 0; i < reps && !rc; ++i) rc = f();
  FMGP_CUDA_TRY(cudaEventRecord(e1, s));
  FMGP_CUDA_TRY(cudaEventSynchronize(e1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *out = ms / reps;
  return rc;
}

}  // namespace

extern "C" int fmgp_autotune_precompute(const void* X, fmgp_dtype dtype, const double* Y,
                                        int64_t n, int32_t d, int32_t r, const int32_t* nbr,
                                        int32_t nbr_ld, int32_t k, const fmgp_kernel* kernel,
                                        fmgp_precision precision, int64_t sample_rows,
                                        int32_t* warps_out, void* stream) {
  if (!X || !Y || !nbr || !kernel || !warps_out) {
    set_error("X, Y, nbr, kernel and warps_out are required");
    return FMGP_EINVAL;
  }
  if (n < 1 || d < 1 || r < 1 || k < 1 || k > n || k > kMaxK || nbr_ld < k - 1 ||
      sample_rows < 1 || (precision != FMGP_PREC_FP64 && precision != FMGP_PREC_MIXED) ||
      (dtype != FMGP_F32 && dtype != FMGP_F64)) {
    set_error("autotune: arguments out of range");
    return FMGP_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  Workspace ws(s);
  const int64_t cnt = sample_rows < n ? sample_rows : n;
  void* Ctmp = ws.alloc((size_t)cnt * k * r * 8);
  int* fails = ws.get<int>(1);
  unsigned long long* queue = ws.get<unsigned long long>(1);
  if (!Ctmp || !fails || !queue) return FMGP_ENOMEM;
  BlockArgs a{};
  a.Y = Y;
  a.nbr = nbr;
  a.C = Ctmp;
  a.fail_count = fails;
  a.n = n;
  a.count = cnt;
  a.d = d;
  a.r = r;
  a.ld = nbr_ld;
  a.k = k;
  a.kp = make_kparams(*kernel);
  a.layout = block_layout(k, d, r, dtype == FMGP_F64 ? 8 : 4, false);
  const size_t bytes = precision == FMGP_PREC_FP64 ? a.layout.bytes_per_warp
                                                   : mixed_bytes_per_warp(k, d, r, dtype == FMGP_F64 ? 8 : 4);
  int best = 0, best_panel = 0, best_persist = 1;
  float best_ms = 1e30f;
  // the mixed kernel's Cholesky panel width: both instantiated widths for k <= 64
  const bool panels = precision == FMGP_PREC_MIXED && k <= 64;
  // persistent (one wave claiming items from a counter) or eight waves of
  // grid-stride CTAs, unless the tuning key fixes it
  const int fixed = tune_params().block_persistent;
  for (int persist : {1, 0}) {
    if (fixed >= 0 && persist != (fixed != 0)) continue;
    a.queue = persist ? queue : nullptr;
    for (int panel : {0, 4, 8}) {
      if (panel && !panels) continue;
      if (!panel && panels) continue;
      for (int w : {1, 2, 4, 6, 8}) {
        if ((size_t)w * bytes > 200 * 1024) continue;
        float ms = 0.f;
        int rc = time_ms(s, 2, [&]() {
          Workspace inner(s);
          return precision == FMGP_PREC_FP64
                     ? launch_block_f64(a, X, dtype, kModePrecompute, w, s)
                     : run_block_mixed(a, X, dtype, kModePrecompute, w, panel, *kernel, inner, s);
        }, &ms);
        if (rc) return rc;
        if (ms < best_ms) { best_ms = ms; best = w; best_panel = panel; best_persist = persist; }
      }
    }
  }
  if (!best) {
    set_error("autotune: no feasible warps-per-CTA for k=%d d=%d r=%d", k, d, r);
    return FMGP_EUNSUPPORTED;
  }
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_warps[{(int)precision, k, d, r, (int)dtype}] = best;
    g_panel[{(int)precision, k, d, r, (int)dtype}] = best_panel;
    g_persist[{(int)precision, k, d, r, (int)dtype}] = best_persist;
  }
  *warps_out = best;
  return FMGP_OK;
}

extern "C" int fmgp_autotune_choice(fmgp_precision precision, int32_t k, int32_t d, int32_t r,
                                    fmgp_dtype dtype, int32_t* warps, int32_t* panel,
                                    int32_t* persistent) {
  if (!warps || !panel || !persistent) {
    set_error("warps, panel and persistent must be non-NULL");
    return FMGP_EINVAL;
  }
  *warps = tuned_block_warps((int)precision, k, d, r, (int)dtype);
  *panel = tuned_block_panel((int)precision, k, d, r, (int)dtype);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_persist.find({(int)precision, k, d, r, (int)dtype});
  *persistent = it == g_persist.end() ? -1 : it->second;
  return FMGP_OK;
}

extern "C" int fmgp_autotune_knn(const void* X, fmgp_dtype dtype, int64_t n, int32_t d, int32_t kq,
                                 double* grid_target_out, void* stream) {
  if (!X || !grid_target_out || n < 2 || d < 1 || kq < 1 || kq > n - 1 || kq > kMaxK ||
      (dtype != FMGP_F32 && dtype != FMGP_F64)) {
    set_error("autotune: arguments out of range");
    return FMGP_EINVAL;
  }
  if (d > kGridMaxD) {
    *grid_target_out = 0.0;  // nothing to tune: exhaustive / tensor-core search
    return FMGP_OK;
  }
  cudaStream_t s = (cudaStream_t)stream;
  Workspace ws(s);
  int32_t* nbr = ws.get<int32_t>((size_t)n * kq);
  if (!nbr) return FMGP_ENOMEM;
  double best = 0.0;
  float best_ms = 1e30f;
  for (double t : {4.0, 6.0, 8.0, 12.0, 16.0, 24.0, 32.0}) {
    TuneParams tp = tune_params();
    tp.grid_target = t;
    float ms = 0.f;
    int rc = time_ms(s, 2, [&]() {
      Workspace inner(s);
      return knn_self(X, dtype, n, d, kq, nbr, nullptr, tp, inner, s);
    }, &ms);
    if (rc) return rc;
    if (ms < best_ms) { best_ms = ms; best = t; }
  }
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_grid[{(int)d, (int)kq}] = best;
  }
  *grid_target_out = best;
  return FMGP_OK;
}

extern "C" int fmgp_autotune_reset(void) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_warps.clear();
  g_panel.clear();
  g_persist.clear();
  g_grid.clear();
  return FMGP_OK;
}
