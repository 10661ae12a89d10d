// Resident fitted models: a model borrows the caller's X, neighbour table and
// coefficients (or keeps copies of its own) and owns what prediction would
// otherwise rebuild per call (the
// search grid over X for d <= 3, an FP32 copy of an FP64 X for the
// nearest-point scan at 4 <= d <= 15, the packed training side of the
// tensor-core search at d >= 16, the double-float copy of X for the mixed
// form), so repeated prediction batches (the serving loop) only run the
// nearest-point lookup and the gather-dot.
#include "model.cuh"
#include "predict.cuh"

namespace fmgp {

Model::~Model() {
  for (int i = 0; i < nbufs; ++i) cudaFree(bufs[i]);
  context_release(ctx, ctx_bytes);
}

}  // namespace fmgp

using namespace fmgp;

namespace fmgp {

// Validate a model's arguments and build what its predictions reuse; the
// buffers in owned[0..nowned) (X, nbr, C of a loaded model) become the
// model's and are freed with it, also when this fails.
int model_create(const void* X, fmgp_dtype dtype, int64_t n, int32_t d, const int32_t* nbr,
                 int32_t nbr_ld, const void* C, int32_t k, int32_t r, const fmgp_kernel* kernel,
                 fmgp_precision precision, fmgp_model** out, cudaStream_t s, void* const* owned,
                 int nowned, bool copy) {
  auto release = [&]() {
    for (int i = 0; i < nowned; ++i) cudaFree(owned[i]);
  };
  if (!out) { release(); set_error("out must be non-NULL"); return FMGP_EINVAL; }
  *out = nullptr;
  if (!X || !C || (k > 1 && !nbr) || !kernel) {
    set_error("X, C, kernel (and nbr when k > 1) must be non-NULL");
    return release(), FMGP_EINVAL;
  }
  if (dtype != FMGP_F32 && dtype != FMGP_F64) { set_error("dtype unknown"); return release(), FMGP_EINVAL; }
  if (precision != FMGP_PREC_FP64 && precision != FMGP_PREC_MIXED) {
    set_error("precision unknown");
    return release(), FMGP_EINVAL;
  }
  if (n < 1 || n >= INT32_MAX || d < 1 || r < 1 || k < 1 || k > n || k > kMaxK ||
      nbr_ld < k - 1) {
    set_error("shape invalid: n=%lld d=%d r=%d k=%d nbr_ld=%d", (long long)n, d, r, k, nbr_ld);
    return release(), FMGP_EINVAL;
  }
  if (kernel->kind == FMGP_KERNEL_MATERN &&
      !(kernel->nu == 0.5 || kernel->nu == 1.5 || kernel->nu == 2.5)) {
    set_error("Matern nu = %g unsupported", kernel->nu);
    return release(), FMGP_EINVAL;
  }
  if (!(kernel->length_scale > 0) || !(kernel->variance > 0) || !(kernel->nugget >= 0)) {
    set_error("kernel hyperparameters invalid");
    return release(), FMGP_EINVAL;
  }
  if (int fc = check_finite({{X, dtype == FMGP_F64, n * (int64_t)d, "X"}}, s))
    return release(), fc;
  Model* m = new Model();
  for (int i = 0; i < nowned && i < Model::kMaxBufs; ++i) m->bufs[m->nbufs++] = owned[i];
  m->X = X; m->dtype = dtype; m->n = n; m->d = d; m->nbr = nbr; m->ld = nbr_ld; m->C = C;
  m->k = k; m->r = r; m->kern = *kernel; m->prec = precision;
  Workspace ws(s);
  int rc = FMGP_OK;
  if (copy) {
    // the model's own copies of X, the neighbour table and C
    const size_t xb = (size_t)n * d * (dtype == FMGP_F64 ? 8 : 4);
    const size_t nb = k > 1 ? (size_t)n * nbr_ld * 4 : 0;
    const size_t cb = (size_t)n * k * r * 8;
    void* Xc = ws.alloc(xb);
    void* Cc = ws.alloc(cb);
    void* Nc = nb ? ws.alloc(nb) : nullptr;
    if (!Xc || !Cc || (nb && !Nc)) {
      rc = FMGP_ENOMEM;
    } else {
      cudaError_t e = cudaMemcpyAsync(Xc, X, xb, cudaMemcpyDeviceToDevice, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(Cc, C, cb, cudaMemcpyDeviceToDevice, s);
      if (e == cudaSuccess && nb) e = cudaMemcpyAsync(Nc, nbr, nb, cudaMemcpyDeviceToDevice, s);
      if (e != cudaSuccess) rc = cuda_fail(e, "cudaMemcpyAsync (model copy)");
      m->X = X = Xc;
      m->C = Cc;
      if (nb) m->nbr = (const int32_t*)Nc;
    }
  }
  if (!rc && d <= kGridMaxD) {
    rc = build_grid(X, dtype, n, d, tune_params().grid_target, ws, s, &m->grid);
    m->has_grid = (rc == FMGP_OK);
  }
  if (!rc && d > kGridMaxD && d <= kNn1ScanMaxD && dtype == FMGP_F64) {
    m->Xf32 = ws.get<float>((size_t)n * d);
    if (!m->Xf32) rc = FMGP_ENOMEM;
    else rc = to_f32((const double*)X, n * d, m->Xf32, s);
  }
  if (!rc && d > kNn1ScanMaxD && tc_knn_eligible(n, d, 1 << 20, 1)) {
    rc = tc_pack_train(X, dtype, n, d, ws, s, &m->tc);
    m->has_tc = (rc == FMGP_OK);
  }
  if (!rc && precision == FMGP_PREC_MIXED) {
    m->Xdf = ws.get<float2>((size_t)n * d);
    if (!m->Xdf) rc = FMGP_ENOMEM;
    else rc = to_df(X, dtype == FMGP_F64, n * d, m->Xdf, s);
  }
  if (!rc) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = cuda_fail(e, "cudaStreamSynchronize");
  }
  m->bytes = ws.bytes();
  m->nbufs += ws.detach(m->bufs + m->nbufs, Model::kMaxBufs - m->nbufs, &m->ctx, &m->ctx_bytes);
  if (rc) {
    delete m;
    return rc;
  }
  *out = reinterpret_cast<fmgp_model*>(m);
  return FMGP_OK;
}

}  // namespace fmgp

extern "C" int fmgp_model_create(const void* X, fmgp_dtype dtype, int64_t n, int32_t d,
                                 const int32_t* nbr, int32_t nbr_ld, const void* C, int32_t k,
                                 int32_t r, const fmgp_kernel* kernel, fmgp_precision precision,
                                 int32_t flags, fmgp_model** out, void* stream) {
  clear_error();
  if (flags != FMGP_MODEL_BORROW && flags != FMGP_MODEL_COPY) {
    if (out) *out = nullptr;
    set_error("flags = %d: FMGP_MODEL_BORROW (0) or FMGP_MODEL_COPY (1)", flags);
    return FMGP_EINVAL;
  }
  return model_create(X, dtype, n, d, nbr, nbr_ld, C, k, r, kernel, precision, out,
                      (cudaStream_t)stream, nullptr, 0, flags == FMGP_MODEL_COPY);
}

extern "C" int fmgp_model_predict(fmgp_model* model, const void* Z, int64_t m, double* Yhat_out,
                                  int32_t* nearest_out, void* stream) {
  clear_error();
  Model* md = reinterpret_cast<Model*>(model);
  if (!md) { set_error("model is NULL"); return FMGP_EINVAL; }
  if (m < 0) { set_error("m = %lld must be >= 0", (long long)m); return FMGP_EINVAL; }
  if (m == 0) return FMGP_OK;
  if (!Z || !Yhat_out) { set_error("Z and Yhat_out must be non-NULL"); return FMGP_EINVAL; }
  if (int fc = check_finite({{Z, md->dtype == FMGP_F64, m * (int64_t)md->d, "Z"}},
                            (cudaStream_t)stream))
    return fc;
  return model_predict(*md, Z, m, Yhat_out, nearest_out, (cudaStream_t)stream);
}

extern "C" int fmgp_model_destroy(fmgp_model* model) {
  Model* md = reinterpret_cast<Model*>(model);
  if (!md) return FMGP_EINVAL;
  cudaDeviceSynchronize();  // in-flight work may still read the model's buffers
  delete md;
  return FMGP_OK;
}

extern "C" int64_t fmgp_model_device_bytes(const fmgp_model* model) {
  const Model* md = reinterpret_cast<const Model*>(model);
  return md ? (int64_t)md->bytes : -1;
}

namespace fmgp {

int model_predict(const Model& md, const void* Z, int64_t m, double* Yhat, int32_t* nearest,
                  cudaStream_t s) {
  Workspace ws(s);
  int32_t* near = nearest;
  if (!near) {
    near = ws.get<int32_t>(m);
    if (!near) return FMGP_ENOMEM;
  }
  int rc = md.has_grid ? nearest_on_grid(md.grid, Z, md.dtype, m, near, s)
           : md.d <= kNn1ScanMaxD
               ? nearest_scan(md.X, md.dtype, md.n, md.d, Z, m, nullptr, near, ws, s, md.Xf32)
           : md.has_tc && tc_knn_eligible(md.n, md.d, m, 1)
               ? tc_knn_query_packed(md.tc, md.X, md.dtype, md.n, md.d, Z, m, 1, near, nullptr,
                                     ws, s)
               : nearest_train(md.X, md.dtype, md.n, md.d, Z, m, near, tune_params(), ws, s);
  if (rc) return rc;
  const KParams kp = make_kparams(md.kern);
  if (md.prec == FMGP_PREC_MIXED)
    return gather_dot_mixed(md.X, md.dtype, md.n, md.d, md.nbr, md.ld, md.C, md.k, md.r, kp,
                            md.kern, Z, m, near, Yhat, ws, s, md.Xdf);
  return gather_dot(md.X, md.dtype, md.n, md.d, md.nbr, md.ld, md.C, md.k, md.r, kp, md.kern,
                    md.prec, Z, m, near, Yhat, ws, s);
}

}  // namespace fmgp
