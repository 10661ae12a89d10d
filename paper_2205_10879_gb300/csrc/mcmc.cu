// Metropolis calibration of one model input against one observation (Sec. 4.2,
// the borehole inverse problem), with a resident model's posterior mean
// (Eq. 7) as the emulator.  All chains advance together: every step is one
// pass over the chains (accept the previous proposal, draw the next), the
// nearest-training-point lookup of all proposals, and the gather-dot.  The
// random draws are inputs; a move is decided by delta + expo > 0 in FP64
// with every operation rounded as written, so the decisions are reproducible
// and need no transcendental function.
#include <math.h>

#include "model.cuh"
#include "predict.cuh"

namespace fmgp {
namespace {

struct ChainState {
  double* x;           // chains: current state
  double* e;           // chains: f_obs - yhat(current) of response column col
  double* xp;          // chains: pending proposal
  int8_t* ok;          // chains: pending proposal inside [lo, hi]
  int64_t* acc;        // chains: accepted moves
  const double* yhat;  // chains x r: emulator at the pending proposals
  const double* z0;    // d: base input
  const double* noise; // steps x chains, N(0, 1)
  const double* expo;  // steps x chains, Exp(1)
  double* samples;     // steps x chains or null
  int64_t chains;
  int d, dim, r, col;
  double lo, hi, f_obs, step, two_s2;
};

// Writes the model input of each chain: z0 with coordinate dim = v[c].
template <typename T>
__device__ __forceinline__ void write_row(const ChainState& s, T* Zp, int64_t c, double v) {
  T* row = Zp + c * s.d;
  for (int j = 0; j < s.d; ++j) row[j] = (T)(j == s.dim ? v : s.z0[j]);
}

template <typename T>
__global__ void chain_start_kernel(ChainState s, const double* x0, T* Zp) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= s.chains) return;
  s.x[c] = x0[c];
  s.acc[c] = 0;
  write_row(s, Zp, c, x0[c]);
}

__global__ void chain_error_kernel(ChainState s) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= s.chains) return;
  s.e[c] = __dsub_rn(s.f_obs, s.yhat[c * s.r + s.col]);
}

// t > 0: decide proposal t-1 (emulated in yhat) and record the state;
// t < steps: draw proposal t and write its model input.
template <typename T>
__global__ void chain_step_kernel(ChainState s, int64_t t, int64_t steps, T* Zp) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= s.chains) return;
  double x = s.x[c];
  if (t > 0) {
    const int64_t at = (t - 1) * s.chains + c;
    if (s.ok[c]) {
      const double e = s.e[c];
      const double ep = __dsub_rn(s.f_obs, s.yhat[c * s.r + s.col]);
      const double delta = __ddiv_rn(__dsub_rn(__dmul_rn(e, e), __dmul_rn(ep, ep)), s.two_s2);
      if (__dadd_rn(delta, s.expo[at]) > 0.0) {
        x = s.xp[c];
        s.x[c] = x;
        s.e[c] = ep;
        s.acc[c] += 1;
      }
    }
    if (s.samples) s.samples[at] = x;
  }
  if (t < steps) {
    const double xp = __dadd_rn(x, __dmul_rn(s.step, s.noise[t * s.chains + c]));
    const bool ok = xp >= s.lo && xp <= s.hi;
    s.xp[c] = xp;
    s.ok[c] = ok ? 1 : 0;
    write_row(s, Zp, c, ok ? xp : x);  // a rejected-by-prior proposal is emulated harmlessly
  }
}

// Posterior mean at the rows of Zp (m = chains) into yhat.
int emulate(const Model& md, const void* Zp, int64_t m, const unsigned int* mx, int32_t* near,
            double* yhat, cudaStream_t s) {
  Workspace ws(s);
  int rc;
  if (md.has_grid)
    rc = nearest_on_grid(md.grid, Zp, md.dtype, m, near, s);
  else if (md.d <= kNn1ScanMaxD)
    rc = nearest_scan(md.X, md.dtype, md.n, md.d, Zp, m, mx, near, ws, s, md.Xf32);
  else if (tune_params().use_tensor_cores && tc_knn_eligible(md.n, md.d, m, 1))
    rc = knn_query_brute(md.X, md.dtype, md.n, md.d, Zp, m, 1, near, nullptr, ws, s);
  else
    rc = knn_query_brute_mx(md.X, md.dtype, md.n, md.d, Zp, m, 1, mx, near, nullptr, ws, s);
  if (rc) return rc;
  const KParams kp = make_kparams(md.kern);
  if (md.prec == FMGP_PREC_MIXED)
    return gather_dot_mixed(md.X, md.dtype, md.n, md.d, md.nbr, md.ld, md.C, md.k, md.r, kp,
                            md.kern, Zp, m, near, yhat, ws, s, md.Xdf);
  return gather_dot(md.X, md.dtype, md.n, md.d, md.nbr, md.ld, md.C, md.k, md.r, kp, md.kern,
                    md.prec, Zp, m, near, yhat, ws, s);
}

template <typename T>
int run_chains(const Model& md, ChainState st, const double* x0_host, int64_t steps,
               const double* z0_host, double* x_out, cudaStream_t s) {
  const int64_t C = st.chains;
  Workspace ws(s);
  st.x = ws.get<double>(C);
  st.e = ws.get<double>(C);
  st.xp = ws.get<double>(C);
  st.ok = ws.get<int8_t>(C);
  int64_t* acc_own = st.acc ? nullptr : ws.get<int64_t>(C);
  if (!st.acc) st.acc = acc_own;
  double* yhat = ws.get<double>((size_t)C * md.r);
  int32_t* near = ws.get<int32_t>(C);
  T* Zp = ws.get<T>((size_t)C * md.d);
  double* z0 = ws.get<double>(md.d);
  double* zb = ws.get<double>(md.d);
  double* x0 = ws.get<double>(C);
  unsigned int* mx = ws.get<unsigned int>(1);
  if (!st.x || !st.e || !st.xp || !st.ok || !st.acc || !yhat || !near || !Zp || !z0 || !zb ||
      !x0 || !mx)
    return FMGP_ENOMEM;
  st.yhat = yhat;
  st.z0 = z0;
  // magnitude bound of every proposal input: z0 off the calibrated
  // coordinate, max(|lo|, |hi|) on it
  double* zb_host = (double*)malloc(sizeof(double) * md.d);
  if (!zb_host) return FMGP_ENOMEM;
  for (int j = 0; j < md.d; ++j) zb_host[j] = z0_host[j];
  zb_host[st.dim] = fmax(fabs(st.lo), fabs(st.hi));
  cudaError_t e1 = cudaMemcpyAsync(z0, z0_host, sizeof(double) * md.d, cudaMemcpyHostToDevice, s);
  cudaError_t e2 = cudaMemcpyAsync(zb, zb_host, sizeof(double) * md.d, cudaMemcpyHostToDevice, s);
  cudaError_t e3 = cudaMemcpyAsync(x0, x0_host, sizeof(double) * C, cudaMemcpyHostToDevice, s);
  // pageable sources are staged before the copies return
  free(zb_host);
  FMGP_CUDA_TRY(e1);
  FMGP_CUDA_TRY(e2);
  FMGP_CUDA_TRY(e3);
  FMGP_CUDA_TRY(cudaMemsetAsync(mx, 0, sizeof(unsigned int), s));
  int rc = maxabs_into(md.X, md.dtype == FMGP_F64, md.n * md.d, mx, s);
  if (!rc) rc = maxabs_into(zb, true, md.d, mx, s);
  if (rc) return rc;
  const int threads = 256;
  const int blocks = ceil_div(C, threads);
  FMGP_LAUNCH(chain_start_kernel<T><<<blocks, threads, 0, s>>>(st, x0, Zp));
  rc = emulate(md, Zp, C, mx, near, yhat, s);
  if (rc) return rc;
  FMGP_LAUNCH(chain_error_kernel<<<blocks, threads, 0, s>>>(st));
  for (int64_t t = 0; t <= steps; ++t) {
    FMGP_LAUNCH(chain_step_kernel<T><<<blocks, threads, 0, s>>>(st, t, steps, Zp));
    if (t == steps) break;
    rc = emulate(md, Zp, C, mx, near, yhat, s);
    if (rc) return rc;
  }
  if (x_out)
    FMGP_CUDA_TRY(cudaMemcpyAsync(x_out, st.x, sizeof(double) * C, cudaMemcpyDeviceToDevice, s));
  FMGP_CUDA_TRY(cudaGetLastError());
  return FMGP_OK;
}

}  // namespace
}  // namespace fmgp

using namespace fmgp;

extern "C" int fmgp_model_mcmc(fmgp_model* model, const double* z0, int32_t dim, double lo,
                               double hi, double f_obs, int32_t col, double sigma, double step,
                               int64_t chains, int64_t steps, const double* x0,
                               const double* noise, const double* expo, double* samples_out,
                               int64_t* accepted_out, double* x_out, void* stream) {
  Model* md = reinterpret_cast<Model*>(model);
  if (!md) { set_error("model is NULL"); return FMGP_EINVAL; }
  if (!z0) { set_error("z0 must be non-NULL"); return FMGP_EINVAL; }
  if (dim < 0 || dim >= md->d) { set_error("dim = %d outside [0, %d)", dim, md->d); return FMGP_EINVAL; }
  if (col < 0 || col >= md->r) { set_error("col = %d outside [0, %d)", col, md->r); return FMGP_EINVAL; }
  if (!isfinite(lo) || !isfinite(hi) || !(lo <= hi)) {
    set_error("prior bounds must be finite with lo <= hi");
    return FMGP_EINVAL;
  }
  if (!(sigma > 0) || !isfinite(sigma) || !isfinite(step) || !isfinite(f_obs)) {
    set_error("sigma must be positive and finite; step and f_obs finite");
    return FMGP_EINVAL;
  }
  if (chains < 0 || steps < 0 || chains >= INT32_MAX) {
    set_error("chains = %lld and steps = %lld must be >= 0 (chains < 2^31)", (long long)chains,
              (long long)steps);
    return FMGP_EINVAL;
  }
  if (chains == 0) return FMGP_OK;
  if (!x0 || (steps > 0 && (!noise || !expo))) {
    set_error("x0 (and noise, expo when steps > 0) must be non-NULL");
    return FMGP_EINVAL;
  }
  for (int64_t c = 0; c < chains; ++c)
    if (!(x0[c] >= lo && x0[c] <= hi)) {
      set_error("x0[%lld] = %g outside the prior [%g, %g]", (long long)c, x0[c], lo, hi);
      return FMGP_EINVAL;
    }
  for (int j = 0; j < md->d; ++j)
    if (!isfinite(z0[j])) { set_error("z0[%d] is not finite", j); return FMGP_EINVAL; }
  ChainState st{};
  st.acc = accepted_out;
  st.noise = noise;
  st.expo = expo;
  st.samples = samples_out;
  st.chains = chains;
  st.d = md->d;
  st.dim = dim;
  st.r = md->r;
  st.col = col;
  st.lo = lo;
  st.hi = hi;
  st.f_obs = f_obs;
  st.step = step;
  st.two_s2 = 2.0 * sigma * sigma;
  cudaStream_t s = (cudaStream_t)stream;
  if (md->dtype == FMGP_F64) return run_chains<double>(*md, st, x0, steps, z0, x_out, s);
  return run_chains<float>(*md, st, x0, steps, z0, x_out, s);
}
