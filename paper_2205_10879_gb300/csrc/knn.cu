// A1 (self kNN table) and the nearest-training-point search of A4.
//   d <= 3 : uniform grid, one warp per query, rings of cells in order of
//            Chebyshev distance with box pruning and an exact stop test.
//   d >= 4 : tiled scan of all training points; a CTA of 8 warps (8 queries)
//            stages 256 candidate rows at a time in shared memory as FP32.
//   nearest point only, 4 <= d <= 15: one thread per query over slices of
//            the training points, then a minimum over the slices.
// Both rank on the canonical FP64 key; FP32 is used only for lower bounds.
#include <algorithm>
#include "knn.cuh"
#include "topk.cuh"

namespace fmgp {
namespace {

constexpr float kU = 5.9604645e-8f;  // 2^-24

// ---------------------------------------------------------------- grid ----
// Initial distance threshold from the local density: the number of points in
// the 3^D block of cells around the query, over the block's volume, gives the
// radius expected to hold ~1.4 kq points.  It only prunes: if the search ends
// with fewer than kq points inside it, or with a k-th key above it, the query
// is searched again without it, so the result never depends on the guess.
template <int D>
__device__ __forceinline__ float density_threshold(const GridView& gv, const GridGeom& g,
                                                   const int* cq, int kq) {
  int cnt = 0;
  float vol = 1.f;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    const int lo = max(cq[j] - 1, 0), hi = min(cq[j] + 1, g.G - 1);
    vol *= (float)(hi - lo + 1) * g.w[j];
  }
  const int lo0 = max(cq[0] - 1, 0), hi0 = min(cq[0] + 1, g.G - 1);
  const int lo1 = D > 1 ? max(cq[D > 1 ? 1 : 0] - 1, 0) : 0;
  const int hi1 = D > 1 ? min(cq[D > 1 ? 1 : 0] + 1, g.G - 1) : 0;
  const int lo2 = D > 2 ? max(cq[D > 2 ? 2 : 0] - 1, 0) : 0;
  const int hi2 = D > 2 ? min(cq[D > 2 ? 2 : 0] + 1, g.G - 1) : 0;
  for (int c2 = lo2; c2 <= hi2; ++c2)
    for (int c1 = lo1; c1 <= hi1; ++c1)
      cnt += gv.cell_start[cell_linear(hi0, c1, c2, g.G, D) + 1] -
             gv.cell_start[cell_linear(lo0, c1, c2, g.G, D)];
  if (cnt < 2 || !(vol > 0.f)) return __int_as_float(0x7f800000);
  const float unit = D == 1 ? 2.f : (D == 2 ? 3.14159265f : 4.18879020f);
  const float rD = 1.4f * (float)kq * vol / ((float)cnt * unit);  // r^D
  const float r = D == 1 ? rD : (D == 2 ? sqrtf(rD) : cbrtf(rD));
  return r * r;
}

// Exact kq-nearest search of one query (q64/qf, excluding training index
// `excl`, -1 for none) on the grid; the result is left in `top`.
template <int D, int L>
__device__ __forceinline__ void grid_knn_search(const GridView& gv, const GridGeom& g,
                                                const double* q64, const float* qf, int excl,
                                                int kq, int lane, WarpTopK<L>& top) {
  const float qs = query_slack<D>(qf);
  const float margin = g.margin + qs;
  const float cerr = g.conv_err + (g.conv_err > 0.f ? qs : 0.f);
  int cq[3] = {0, 0, 0};
  cell_of<D>(g, qf, cq);
  float pre = density_threshold<D>(gv, g, cq, kq);
  unsigned int n_exam = 0, n_key = 0;  // per lane, for the optional counters
  for (int attempt = 0; attempt < 2; ++attempt) {
    top.init(kq);
    bool fresh = true;  // the first batch goes into the empty list by one sort
    for (int r = 0;; ++r) {
      for_ring_segments<D>(r, cq, g.G, [&](int c0a, int c0b, int c1, int c2) {
        const float lim = fminf(top.t_up, pre);
        if (lim < __int_as_float(0x7f800000) && box_lower<D>(g, qf, margin, c0a, c0b, c1, c2) > lim)
          return;
        const int s0 = gv.cell_start[cell_linear(c0a, c1, c2, g.G, D)];
        const int e0 = gv.cell_start[cell_linear(c0b, c1, c2, g.G, D) + 1];
        for (int base = s0; base < e0; base += 32) {
          const int j = base + lane;
          unsigned long long ck = ~0ull;
          int ci = INT_MAX;
          if (j < e0) {
            const int id = gv.ids[j];
            if (id != excl) {
              float xf[D];
#pragma unroll
              for (int t = 0; t < D; ++t) xf[t] = gv.xs32[(int64_t)j * D + t];
              ++n_exam;
              if (dist_lower_f32<D>(qf, xf, cerr) <= fminf(top.t_up, pre)) {
                ck = dbits(canon_key<double>(q64, gv.xs64 + (int64_t)j * D, D));
                ci = id;
                ++n_key;
              }
            }
          }
          if (fresh) {
            top.fill_sorted(ck, ci, lane);
            fresh = false;
          } else {
            top.offer(ck, ci, lane);
          }
        }
      });
      const float out = outside_lower<D>(g, qf, margin, cq, r);
      if (top.full() && out > top.t_up) break;
      if (out > pre) break;  // nothing outside can pass the threshold
      if (r >= g.G) break;
    }
    // exact iff the kq-th key does not exceed the threshold (every skipped
    // candidate has key > pre); otherwise search again without it
    if (top.full() && top.t_up <= pre) break;
    if (pre == __int_as_float(0x7f800000)) break;
    pre = __int_as_float(0x7f800000);
  }
  if (gv.visits) {
    n_exam = __reduce_add_sync(kFull, n_exam);
    n_key = __reduce_add_sync(kFull, n_key);
    if (lane == 0) {
      atomicAdd(&gv.visits[0], (unsigned long long)n_exam);
      atomicAdd(&gv.visits[1], (unsigned long long)n_key);
    }
  }
}

// A1: queries are the training points themselves, in cell order (warp w takes
// sorted point w), each excluded from its own list.  At D = 3 the launch
// bound keeps four 256-thread CTAs per SM (64 registers, a 4-byte spill)
// where the compiler would otherwise take 80 registers and three CTAs (the
// 10^7-point table: 99 -> 87 ms); at D <= 2 its own choice is kept.
template <int D, int L>
__global__ void __launch_bounds__(256, D == 3 ? 4 : 0) knn_grid_self_kernel(GridView gv, int kq,
                                                            int32_t* nbr_out, double* dist_out) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= gv.n) return;
  const GridGeom g = *gv.geom;
  double q64[D];
  float qf[D];
#pragma unroll
  for (int j = 0; j < D; ++j) {
    q64[j] = gv.xs64[w * D + j];
    qf[j] = gv.xs32[w * D + j];
  }
  const int qi = gv.ids[w];
  WarpTopK<L> top;
  grid_knn_search<D, L>(gv, g, q64, qf, qi, kq, lane, top);
  top.store(kq, lane, nbr_out + (int64_t)qi * kq, dist_out ? dist_out + (int64_t)qi * kq : nullptr);
}

// kq nearest training points of external query points (MuyGPs prediction).
template <int D, int L, typename T>
__global__ void __launch_bounds__(256, D == 3 ? 4 : 0) knn_grid_query_kernel(GridView gv, const T* Q, int64_t m,
                                                             int kq, int32_t* idx_out,
                                                             double* key_out) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= m) return;
  const GridGeom g = *gv.geom;
  double q64[D];
  float qf[D];
#pragma unroll
  for (int j = 0; j < D; ++j) {
    q64[j] = (double)Q[w * D + j];
    qf[j] = (float)Q[w * D + j];
  }
  WarpTopK<L> top;
  grid_knn_search<D, L>(gv, g, q64, qf, -1, kq, lane, top);
  top.store(kq, lane, idx_out + w * kq, key_out ? key_out + w * kq : nullptr);
}

// ---------------------------------------------------------- brute force ----
constexpr int kBfWarps = 8;
constexpr int kBfTile = 256;   // candidate rows staged per pass (8 per lane)
constexpr int kBfSub = kBfTile / 32;
constexpr int kBfChunk = 64;   // feature columns staged per pass

// gate: optional device count; nothing to do (and no bound needed) when it is 0.
__global__ void maxabs_kernel(const void* X, int f64, int64_t count, unsigned int* out_bits,
                              const int* gate) {
  if (gate && *gate == 0) return;
  float m = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    float v = f64 ? fabsf((float)((const double*)X)[i]) : fabsf(((const float*)X)[i]);
    m = fmaxf(m, v);
  }
  for (int off = 16; off; off >>= 1) m = fmaxf(m, __shfl_xor_sync(kFull, m, off));
  if ((threadIdx.x & 31) == 0) atomicMax(out_bits, __float_as_uint(m));
}

// Each warp owns one query; the CTA stages kBfTile candidate rows at a time
// (FP32 copy of X, kBfChunk feature columns per pass) and lane l bounds rows
// l, l + 32, ... of the tile.  The FP32 partial distances give a lower bound
// (relative rounding of d non-negative terms plus the FP64->FP32 conversion
// slack).  Each lane marks its rows whose bound does not exceed the current
// k-th key; then, round by round, every lane takes its next marked row,
// checks it against the k-th key as it stands, and the warp forms the
// canonical FP64 keys of those rows together and offers them to the list.
// So the FP64 key path runs once per round (not once for every row that any
// lane passes), and the result is the exact top kq by (key, index).
//
// Split form (part_idx != null): the launch covers list positions
// [pos0, pos_end) and blockIdx.y picks the candidate rows
// [y * range_rows, (y + 1) * range_rows); each warp writes the exact top kq of
// its range (INT_MAX past the end) to part_idx/part_key at
// ((p - pos0) * gridDim.y + y) * kq, for merge_parts_kernel.  Otherwise the
// positions [pos0, count) scan all rows into idx_out/key_out.
template <typename T, int L>
__global__ void __launch_bounds__(kBfWarps * 32) knn_brute_kernel(
    const T* X, const float* Xf, int64_t n, int d, const T* Q, int64_t m, int kq,
    int exclude_self, const unsigned int* maxabs_bits, int32_t* idx_out, double* key_out,
    const int* qlist, const int* qcount, int64_t pos0, int64_t pos_end, int64_t range_rows,
    int32_t* part_idx, double* part_key) {
  extern __shared__ float sm[];
  const int ld = d | 1;                      // query rows
  const int tld = min(d, kBfChunk) | 1;      // tile rows: odd stride, conflict-free
  float* tile = sm;                          // kBfTile x tld (chunk of columns)
  float* qs = sm + kBfTile * tld;            // kBfWarps x ld
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // query of this warp: position p of the (optional) list
  const int64_t count = min(qlist ? (int64_t)*qcount : m, pos_end);
  if (pos0 + (int64_t)blockIdx.x * kBfWarps >= count) return;  // whole CTA idle
  const int64_t pos = pos0 + (int64_t)blockIdx.x * kBfWarps + wid;
  const bool qvalid = pos < count;
  const int64_t r0 = part_idx ? (int64_t)blockIdx.y * range_rows : 0;
  const int64_t r1 = part_idx ? min(n, r0 + range_rows) : n;
  const int64_t q = qvalid ? (qlist ? (int64_t)qlist[pos] : pos) : 0;
  const float M = __uint_as_float(*maxabs_bits);
  const float cerr = (sizeof(T) == 8) ? 2.5f * kU * M : 0.f;
  const float rel = 1.0f - (2.0f * d + 8.0f) * kU;
  // stage this CTA's queries (FP32)
  for (int e = threadIdx.x; e < kBfWarps * d; e += blockDim.x) {
    const int w = e / d, j = e % d;
    const int64_t pp = pos0 + (int64_t)blockIdx.x * kBfWarps + w;
    const int64_t qq = pp < count ? (qlist ? (int64_t)qlist[pp] : pp) : -1;
    qs[w * ld + j] = qq >= 0 ? (float)Q[qq * d + j] : 0.f;
  }
  WarpTopK<L> top;
  top.init(kq);
  const float* myq = qs + wid * ld;
  const T* qr = Q + q * d;
  for (int64_t base = r0; base < r1; base += kBfTile) {
    float acc[kBfSub];
#pragma unroll
    for (int u = 0; u < kBfSub; ++u) acc[u] = 0.f;
    for (int c0 = 0; c0 < d; c0 += kBfChunk) {
      const int cw = min(kBfChunk, d - c0);
      __syncthreads();
      for (int e = threadIdx.x; e < kBfTile * cw; e += blockDim.x) {
        const int rr = e / cw, j = e - rr * cw;
        const int64_t row = base + rr;
        tile[rr * tld + j] = row < r1 ? Xf[row * d + c0 + j] : 0.f;
      }
      __syncthreads();
      for (int j = 0; j < cw; ++j) {
        const float qj = myq[c0 + j];
#pragma unroll
        for (int u = 0; u < kBfSub; ++u) {
          float t = fabsf(qj - tile[(u * 32 + lane) * tld + j]) * (1.0f - 2.0f * kU) - cerr;
          t = fmaxf(t, 0.f);
          acc[u] = fmaf(t, t, acc[u]);
        }
      }
    }
    if (!qvalid) continue;
    unsigned pm = 0;  // rows of this lane still to consider
#pragma unroll
    for (int u = 0; u < kBfSub; ++u) {
      const int64_t cand = base + u * 32 + lane;
      if (cand < r1 && !(exclude_self && cand == q)) pm |= 1u << u;
    }
    while (true) {
      // next marked row of each lane whose bound passes the current k-th key
      int ci = INT_MAX;
      while (pm) {
        const int u = __ffs(pm) - 1;
        pm &= pm - 1;
        float a = acc[0];
#pragma unroll
        for (int v = 1; v < kBfSub; ++v)
          if (v == u) a = acc[v];
        if (a * rel <= top.t_up) {
          ci = (int)(base + u * 32 + lane);
          break;
        }
      }
      if (!__any_sync(kFull, ci != INT_MAX)) break;
      unsigned long long ck = ~0ull;
      if (ci != INT_MAX) {
        const T* xr = X + (int64_t)ci * d;
        double t = __dsub_rn((double)qr[0], (double)xr[0]);
        double sum = __dmul_rn(t, t);
        for (int j = 1; j < d; ++j) {
          t = __dsub_rn((double)qr[j], (double)xr[j]);
          sum = __dadd_rn(sum, __dmul_rn(t, t));
        }
        ck = dbits(sum);
      }
      top.offer(ck, ci, lane);
    }
  }
  if (!qvalid) return;
  if (part_idx) {
    const int64_t slot = ((pos - pos0) * gridDim.y + blockIdx.y) * kq;
    top.store(kq, lane, part_idx + slot, part_key + slot);
  } else {
    top.store(kq, lane, idx_out + q * kq, key_out ? key_out + q * kq : nullptr);
  }
}

// One warp per list position p in [pos0, min(count, pos_end)): the kq best by
// (key, index) of the ny partial lists the split scan wrote for it.
template <int L>
__global__ void __launch_bounds__(256) merge_parts_kernel(
    const int32_t* __restrict__ part_idx, const double* __restrict__ part_key, int ny, int kq,
    const int* qlist, const int* qcount, int64_t pos0, int64_t pos_end, int32_t* idx_out,
    double* key_out) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t pos = pos0 + w;
  if (pos >= (qlist ? min((int64_t)*qcount, pos_end) : pos_end)) return;
  const int64_t q = qlist ? (int64_t)qlist[pos] : pos;
  const int tot = ny * kq;
  const int32_t* pi = part_idx + w * tot;
  const unsigned long long* pk = reinterpret_cast<const unsigned long long*>(part_key) + w * tot;
  WarpTopK<L> top;
  top.init(kq);
  for (int base = 0; base < tot; base += 32) {
    const int e = base + lane;
    const int j = e < tot ? pi[e] : INT_MAX;
    top.offer(j != INT_MAX ? pk[e] : ~0ull, j, lane);
  }
  top.store(kq, lane, idx_out + q * kq, key_out ? key_out + q * kq : nullptr);
}

template <int D>
int launch_grid_self(const GridView& gv, int kq, int32_t* nbr, double* dist, cudaStream_t s) {
  const int blocks = ceil_div(gv.n * 32, 256);
  if (kq <= 32) FMGP_LAUNCH(knn_grid_self_kernel<D, 1><<<blocks, 256, 0, s>>>(gv, kq, nbr, dist));
  else if (kq <= 64) FMGP_LAUNCH(knn_grid_self_kernel<D, 2><<<blocks, 256, 0, s>>>(gv, kq, nbr, dist));
  else if (kq <= 96) FMGP_LAUNCH(knn_grid_self_kernel<D, 3><<<blocks, 256, 0, s>>>(gv, kq, nbr, dist));
  else if (kq <= 128) FMGP_LAUNCH(knn_grid_self_kernel<D, 4><<<blocks, 256, 0, s>>>(gv, kq, nbr, dist));
  else FMGP_LAUNCH(knn_grid_self_kernel<D, 5><<<blocks, 256, 0, s>>>(gv, kq, nbr, dist));
  FMGP_CUDA_TRY(cudaGetLastError());
  return FMGP_OK;
}

template <int D, typename T>
int launch_grid_query(const GridView& gv, const T* Q, int64_t m, int kq, int32_t* idx,
                      double* key, cudaStream_t s) {
  const int blocks = ceil_div(m * 32, 256);
  if (kq <= 32) FMGP_LAUNCH((knn_grid_query_kernel<D, 1, T><<<blocks, 256, 0, s>>>(gv, Q, m, kq, idx, key)));
  else if (kq <= 64) FMGP_LAUNCH((knn_grid_query_kernel<D, 2, T><<<blocks, 256, 0, s>>>(gv, Q, m, kq, idx, key)));
  else if (kq <= 96) FMGP_LAUNCH((knn_grid_query_kernel<D, 3, T><<<blocks, 256, 0, s>>>(gv, Q, m, kq, idx, key)));
  else if (kq <= 128) FMGP_LAUNCH((knn_grid_query_kernel<D, 4, T><<<blocks, 256, 0, s>>>(gv, Q, m, kq, idx, key)));
  else FMGP_LAUNCH((knn_grid_query_kernel<D, 5, T><<<blocks, 256, 0, s>>>(gv, Q, m, kq, idx, key)));
  FMGP_CUDA_TRY(cudaGetLastError());
  return FMGP_OK;
}

// List positions (the exact fallback of the tensor-core search) below
// kSplitPos are spread over up to kSplitRanges candidate ranges, so that a
// short list keeps many SMs busy; the partial lists are merged per position.
// Positions beyond scan all rows, kBfWarps queries per CTA.
constexpr int kSplitPos = 64;
constexpr int kSplitRanges = 64;

template <typename T, int L>
int launch_brute_t(const T* X, const float* Xf, int64_t n, int d, const T* Q, int64_t m, int kq,
                   int excl, const unsigned int* mx, int32_t* idx, double* key, cudaStream_t s,
                   const int* qlist = nullptr, const int* qcount = nullptr,
                   Workspace* ws = nullptr) {
  const int ld = d | 1;
  const int tld = std::min(d, kBfChunk) | 1;
  const size_t smem = sizeof(float) * ((size_t)kBfTile * tld + (size_t)kBfWarps * ld);
  if (smem > 200 * 1024) {
    set_error("brute-force kNN: d = %d needs %zu bytes of shared memory", d, smem);
    return FMGP_EUNSUPPORTED;
  }
  auto kern = knn_brute_kernel<T, L>;
  FMGP_CUDA_TRY(ensure_smem((const void*)kern, smem));
  if (!qlist) {
    // few queries: split the candidate rows over CTAs so that about four
    // waves of CTAs scan them, then merge each query's partial lists
    const int64_t qblocks = ceil_div(m, kBfWarps);
    const int64_t tiles = ceil_div(n, kBfTile);
    const int64_t want = 4ll * num_sms();
    if (ws && qblocks * 2 <= want && tiles >= 4) {
      const int64_t ny0 = std::min<int64_t>({tiles, 1024, std::max<int64_t>(2, want / qblocks)});
      const int64_t range_rows = (int64_t)ceil_div(ceil_div(n, ny0), kBfTile) * kBfTile;
      const int ny = ceil_div(n, range_rows);
      int32_t* pidx = ws->get<int32_t>((size_t)m * ny * kq);
      double* pkey = ws->get<double>((size_t)m * ny * kq);
      if (!pidx || !pkey) return FMGP_ENOMEM;
      FMGP_LAUNCH(kern<<<dim3((unsigned)qblocks, (unsigned)ny), kBfWarps * 32, smem, s>>>(
          X, Xf, n, d, Q, m, kq, excl, mx, idx, key, nullptr, nullptr, 0, m, range_rows, pidx, pkey));
      FMGP_LAUNCH(merge_parts_kernel<L><<<ceil_div(m * 32, 256), 256, 0, s>>>(
          pidx, pkey, ny, kq, nullptr, nullptr, 0, m, idx, key));
      FMGP_CUDA_TRY(cudaGetLastError());
      return FMGP_OK;
    }
    FMGP_LAUNCH(kern<<<ceil_div(m, kBfWarps), kBfWarps * 32, smem, s>>>(
        X, Xf, n, d, Q, m, kq, excl, mx, idx, key, nullptr, nullptr, 0, m, 0, nullptr, nullptr));
    FMGP_CUDA_TRY(cudaGetLastError());
    return FMGP_OK;
  }
  if (!ws) {
    set_error("exhaustive kNN over a list needs a workspace");
    return FMGP_EINVAL;
  }
  const int64_t P = std::min<int64_t>(m, kSplitPos);
  const int64_t range_rows =
      (int64_t)ceil_div(ceil_div(n, std::min<int64_t>(kSplitRanges, ceil_div(n, kBfTile))),
                        kBfTile) * kBfTile;
  const int ny = ceil_div(n, range_rows);
  int32_t* pidx = ws->get<int32_t>((size_t)P * ny * kq);
  double* pkey = ws->get<double>((size_t)P * ny * kq);
  if (!pidx || !pkey) return FMGP_ENOMEM;
  FMGP_LAUNCH(kern<<<dim3((unsigned)ceil_div(P, kBfWarps), (unsigned)ny), kBfWarps * 32, smem, s>>>(
      X, Xf, n, d, Q, m, kq, excl, mx, idx, key, qlist, qcount, 0, P, range_rows, pidx, pkey));
  FMGP_LAUNCH(merge_parts_kernel<L><<<ceil_div(P * 32, 256), 256, 0, s>>>(
      pidx, pkey, ny, kq, qlist, qcount, 0, P, idx, key));
  if (m > P)
    FMGP_LAUNCH(kern<<<ceil_div(m - P, kBfWarps), kBfWarps * 32, smem, s>>>(
        X, Xf, n, d, Q, m, kq, excl, mx, idx, key, qlist, qcount, P, m, 0, nullptr, nullptr));
  FMGP_CUDA_TRY(cudaGetLastError());
  return FMGP_OK;
}

template <typename T>
int launch_brute_mx(const T* X, const float* Xf, int64_t n, int d, const T* Q, int64_t m, int kq,
                    int excl, const unsigned int* mx, int32_t* idx, double* key, cudaStream_t s,
                    const int* qlist = nullptr, const int* qcount = nullptr,
                    Workspace* ws = nullptr) {
  if (kq <= 32) return launch_brute_t<T, 1>(X, Xf, n, d, Q, m, kq, excl, mx, idx, key, s, qlist, qcount, ws);
  if (kq <= 64) return launch_brute_t<T, 2>(X, Xf, n, d, Q, m, kq, excl, mx, idx, key, s, qlist, qcount, ws);
  if (kq <= 96) return launch_brute_t<T, 3>(X, Xf, n, d, Q, m, kq, excl, mx, idx, key, s, qlist, qcount, ws);
  if (kq <= 128) return launch_brute_t<T, 4>(X, Xf, n, d, Q, m, kq, excl, mx, idx, key, s, qlist, qcount, ws);
  return launch_brute_t<T, 5>(X, Xf, n, d, Q, m, kq, excl, mx, idx, key, s, qlist, qcount, ws);
}

// FP32 rows the exhaustive scan stages: X itself, or a copy of an FP64 X.
template <typename T>
const float* brute_rows(const T* X, int64_t n, int d, Workspace& ws, cudaStream_t s, int* rc) {
  *rc = FMGP_OK;
  if (sizeof(T) == 4) return (const float*)X;
  float* f = ws.get<float>((size_t)n * d);
  if (!f) { *rc = FMGP_ENOMEM; return nullptr; }
  *rc = to_f32((const double*)X, n * d, f, s);
  return f;
}

// Xf_in: an FP32 copy of X the caller already holds (or null).  With a query
// list the magnitude bound is only computed when the list is not empty.
template <typename T>
int launch_brute(const T* X, int64_t n, int d, const T* Q, int64_t m, int kq, int excl,
                 Workspace& ws, int32_t* idx, double* key, cudaStream_t s,
                 const int* qlist = nullptr, const int* qcount = nullptr,
                 const float* Xf_in = nullptr) {
  unsigned int* mx = ws.get<unsigned int>(1);
  if (!mx) return FMGP_ENOMEM;
  FMGP_CUDA_TRY(cudaMemsetAsync(mx, 0, sizeof(unsigned int), s));
  int rc = maxabs_into(X, sizeof(T) == 8, n * d, mx, s, qcount);
  if (!rc && Q != X) rc = maxabs_into(Q, sizeof(T) == 8, m * d, mx, s, qcount);
  if (rc) return rc;
  const float* Xf = Xf_in ? Xf_in : brute_rows(X, n, d, ws, s, &rc);
  if (rc) return rc;
  return launch_brute_mx<T>(X, Xf, n, d, Q, m, kq, excl, mx, idx, key, s, qlist, qcount, &ws);
}

// ------------------------------------------- nearest point, 4 <= d < 16 --
// One thread per query keeps the query in registers; CTA (x, y) scans slice
// y of the training points, staged kNnTile rows at a time in shared memory as
// FP32 and read by all threads at the same address.  A candidate whose plain
// FP32 squared distance is within a rounding-safe threshold of the current
// best (nn1_threshold) gets its canonical FP64 key.  Lanes pass that test at
// different rows, and a warp would run the FP64 key path once for every such
// row; so the threshold is first seeded with the key of each lane's nearest
// candidate (by FP32 distance) in the first tile, one round for all lanes, and
// then passing candidates are queued per lane and keyed together at the end
// of each tile.  Every passing candidate is keyed and compared by (key,
// index), so the result is the exact minimum.  Each slice's minimum goes to
// part; nn1_merge_kernel takes the minimum over slices.
constexpr int kNnThreads = 128;
constexpr int kNnTile = 256;
constexpr int kNnQueue = 4;

// Pass threshold on the plain FP32 squared distance a = sum_j (qf_j - xf_j)^2
// (FP32 copies of the query and the candidate).  With e = qf - xf and
// delta = (q - x) - e the FP64->FP32 conversion error (|delta_j| <= cerr, so
// ||delta|| <= cvec = cerr sqrt(D)), ||q - x|| >= ||e|| - cvec, and the FMA
// chain gives ||e||^2 >= a * rel.  A candidate can reach the current best
// (whose key is at most bup) only if sqrt(a * rel) <= sqrt(bup) + cvec, i.e.
// a <= (sqrt(bup) + cvec)^2 / rel; the factors below round that bound up.
__device__ __forceinline__ float nn1_threshold(float bup, float cvec, float rel) {
  if (!(bup < __int_as_float(0x7f800000))) return __int_as_float(0x7f800000);
  const float s = sqrtf(bup) * (1.0f + 16.0f * kU) + cvec;
  return s * s * (1.0f + 16.0f * kU) / rel;
}

template <typename T, int D>
__device__ __forceinline__ void nn1_key(const T* __restrict__ X, const T* __restrict__ qg,
                                        int cand, unsigned long long& best, int& bi, float& thr,
                                        float cvec, float rel) {
  const T* xg = X + (int64_t)cand * D;
  double t = __dsub_rn((double)qg[0], (double)xg[0]);
  double sum = __dmul_rn(t, t);
#pragma unroll
  for (int j = 1; j < D; ++j) {
    t = __dsub_rn((double)qg[j], (double)xg[j]);
    sum = __dadd_rn(sum, __dmul_rn(t, t));
  }
  const unsigned long long ck = dbits(sum);
  if (key_less(ck, cand, best, bi)) {
    best = ck;
    bi = cand;
    thr = nn1_threshold(key_bits_to_float_up(best), cvec, rel);
  }
}

template <int D>
__device__ __forceinline__ float nn1_approx(const float* qf, const float* xr) {
  float acc = 0.f;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    const float t = qf[j] - xr[j];
    acc = fmaf(t, t, acc);
  }
  return acc;
}

template <typename T, int D>
__global__ void __launch_bounds__(kNnThreads, 8) nn1_scan_kernel(
    const T* __restrict__ X, const float* __restrict__ Xf, int64_t n, const T* __restrict__ Q,
    int64_t m, const unsigned int* maxabs_bits, int64_t slice, unsigned long long* part_key,
    int* part_idx) {
  __shared__ __align__(16) float tile[kNnTile * D];
  const int64_t q = blockIdx.x * (int64_t)kNnThreads + threadIdx.x;
  const bool qv = q < m;
  const int64_t c0 = (int64_t)blockIdx.y * slice;
  const int64_t c1 = min(n, c0 + slice);
  const float M = __uint_as_float(*maxabs_bits);
  const float cerr = (sizeof(T) == 8) ? 2.5f * kU * M : 0.f;
  const float cvec = cerr * (sqrtf((float)D) * (1.0f + 16.0f * kU));
  const float rel = 1.0f - (2.0f * D + 8.0f) * kU;
  const T* qg = Q + (qv ? q : 0) * D;
  float qf[D];
#pragma unroll
  for (int j = 0; j < D; ++j) qf[j] = qv ? (float)qg[j] : 0.f;
  unsigned long long best = ~0ull;
  int bi = INT_MAX;
  float thr = __int_as_float(0x7f800000);
  int qi[kNnQueue];
  int qn = 0;
  for (int64_t base = c0; base < c1; base += kNnTile) {
    const int rows = (int)min((int64_t)kNnTile, c1 - base);
    __syncthreads();
    for (int e = threadIdx.x; e < rows * D; e += kNnThreads) tile[e] = Xf[base * D + e];
    __syncthreads();
    if (!qv) continue;
    if (base == c0) {
      // seed the threshold: key the first tile's nearest candidate by the
      // FP32 distance (one round for all lanes)
      float amin = __int_as_float(0x7f800000);
      int rmin = 0;
      for (int rr = 0; rr < rows; ++rr) {
        const float a = nn1_approx<D>(qf, tile + rr * D);
        if (a < amin) {
          amin = a;
          rmin = rr;
        }
      }
      nn1_key<T, D>(X, qg, (int)(base + rmin), best, bi, thr, cvec, rel);
    }
    for (int rr = 0; rr < rows; ++rr) {
      if (nn1_approx<D>(qf, tile + rr * D) <= thr) {
        const int cand = (int)(base + rr);
        if (qn < kNnQueue) {
#pragma unroll
          for (int s = 0; s < kNnQueue; ++s)
            if (s == qn) qi[s] = cand;
          ++qn;
        } else {  // this lane's queue is full: drain it alone (rare)
#pragma unroll
          for (int s = 0; s < kNnQueue; ++s)
            nn1_key<T, D>(X, qg, qi[s], best, bi, thr, cvec, rel);
          qi[0] = cand;
          qn = 1;
        }
      }
    }
    // key the queued candidates of all lanes together
#pragma unroll
    for (int s = 0; s < kNnQueue; ++s)
      if (s < qn) nn1_key<T, D>(X, qg, qi[s], best, bi, thr, cvec, rel);
    qn = 0;
  }
  if (qv) {
    part_key[q * gridDim.y + blockIdx.y] = best;
    part_idx[q * gridDim.y + blockIdx.y] = bi;
  }
}

__global__ void nn1_merge_kernel(const unsigned long long* part_key, const int* part_idx,
                                 int64_t m, int slices, int32_t* nearest) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= m) return;
  unsigned long long bk = part_key[q * slices];
  int bi = part_idx[q * slices];
  for (int y = 1; y < slices; ++y) {
    const unsigned long long k = part_key[q * slices + y];
    const int i = part_idx[q * slices + y];
    if (key_less(k, i, bk, bi)) { bk = k; bi = i; }
  }
  nearest[q] = bi;
}

template <typename T, int D>
int launch_nn1_scan(const T* X, const float* Xf, int64_t n, const T* Q, int64_t m,
                    const unsigned int* mx, int32_t* nearest, Workspace& ws, cudaStream_t s) {
  const int qblocks = ceil_div(m, kNnThreads);
  // about eight CTAs per SM in total, slices of at least 2048 rows
  int slices = (int)std::max<int64_t>(1, ((int64_t)num_sms() * 8 + qblocks - 1) / qblocks);
  slices = (int)std::min<int64_t>(slices, std::max<int64_t>(1, n / 2048));
  const int64_t slice = (n + slices - 1) / slices;
  unsigned long long* pk = ws.get<unsigned long long>((size_t)m * slices);
  int* pi = ws.get<int>((size_t)m * slices);
  if (!pk || !pi) return FMGP_ENOMEM;
  FMGP_LAUNCH((nn1_scan_kernel<T, D><<<dim3((unsigned)qblocks, (unsigned)slices), kNnThreads, 0, s>>>(
      X, Xf, n, Q, m, mx, slice, pk, pi)));
  FMGP_LAUNCH(nn1_merge_kernel<<<ceil_div(m, 256), 256, 0, s>>>(pk, pi, m, slices, nearest));
  FMGP_CUDA_TRY(cudaGetLastError());
  return FMGP_OK;
}

template <typename T>
int nn1_scan_t(const T* X, const float* Xf, int64_t n, int d, const T* Q, int64_t m,
               const unsigned int* mx, int32_t* nearest, Workspace& ws, cudaStream_t s) {
  switch (d) {
    case 4: return launch_nn1_scan<T, 4>(X, Xf, n, Q, m, mx, nearest, ws, s);
    case 5: return launch_nn1_scan<T, 5>(X, Xf, n, Q, m, mx, nearest, ws, s);
    case 6: return launch_nn1_scan<T, 6>(X, Xf, n, Q, m, mx, nearest, ws, s);
    case 7: return launch_nn1_scan<T, 7>(X, Xf, n, Q, m, mx, nearest, ws, s);
    case 8: return launch_nn1_scan<T, 8>(X, Xf, n, Q, m, mx, nearest, ws, s);
    case 9: return launch_nn1_scan<T, 9>(X, Xf, n, Q, m, mx, nearest, ws, s);
    case 10: return launch_nn1_scan<T, 10>(X, Xf, n, Q, m, mx, nearest, ws, s);
    case 11: return launch_nn1_scan<T, 11>(X, Xf, n, Q, m, mx, nearest, ws, s);
    case 12: return launch_nn1_scan<T, 12>(X, Xf, n, Q, m, mx, nearest, ws, s);
    case 13: return launch_nn1_scan<T, 13>(X, Xf, n, Q, m, mx, nearest, ws, s);
    case 14: return launch_nn1_scan<T, 14>(X, Xf, n, Q, m, mx, nearest, ws, s);
    case 15: return launch_nn1_scan<T, 15>(X, Xf, n, Q, m, mx, nearest, ws, s);
    default:
      set_error("nearest-point scan: d = %d outside [4, %d]", d, kNn1ScanMaxD);
      return FMGP_EUNSUPPORTED;
  }
}

}  // namespace

int knn_brute_list(const void* X, fmgp_dtype dtype, int64_t n, int d, const void* Q, int64_t m,
                   int kq, bool self, const int* qlist, const int* qcount, int32_t* idx,
                   double* key, Workspace& ws, cudaStream_t stream, const float* Xf) {
  if (dtype == FMGP_F64)
    return launch_brute<double>((const double*)X, n, d, (const double*)Q, m, kq, self ? 1 : 0, ws,
                                idx, key, stream, qlist, qcount, Xf);
  return launch_brute<float>((const float*)X, n, d, (const float*)Q, m, kq, self ? 1 : 0, ws, idx,
                             key, stream, qlist, qcount, Xf);
}

int knn_self(const void* X, fmgp_dtype dtype, int64_t n, int d, int kq, int32_t* nbr,
             double* dist, const TuneParams& tp, Workspace& ws, cudaStream_t stream) {
  if (d <= kGridMaxD) {
    GridView gv;
    int rc = build_grid(X, dtype, n, d, tp.grid_target, ws, stream, &gv);
    if (rc) return rc;
    if (tp.count_visits) gv.visits = diag_visits_begin(n, stream);
    rc = d == 1   ? launch_grid_self<1>(gv, kq, nbr, dist, stream)
         : d == 2 ? launch_grid_self<2>(gv, kq, nbr, dist, stream)
                  : launch_grid_self<3>(gv, kq, nbr, dist, stream);
    if (!rc && gv.visits) diag_visits_end(stream);
    return rc;
  }
  if (tc_knn_eligible(n, d, n, kq))
    return tc_knn(X, dtype, n, d, X, n, kq, true, nbr, dist, ws, stream);
  if (dtype == FMGP_F64)
    return launch_brute<double>((const double*)X, n, d, (const double*)X, n, kq, 1, ws, nbr, dist,
                                stream);
  return launch_brute<float>((const float*)X, n, d, (const float*)X, n, kq, 1, ws, nbr, dist,
                             stream);
}

int knn_query(const void* X, fmgp_dtype dtype, int64_t n, int d, const void* Q, int64_t m, int kq,
              int32_t* idx, double* key, const TuneParams& tp, Workspace& ws, cudaStream_t stream) {
  if (m == 0) return FMGP_OK;
  if (d <= kGridMaxD) {
    GridView gv;
    int rc = build_grid(X, dtype, n, d, tp.grid_target, ws, stream, &gv);
    if (rc) return rc;
    if (tp.count_visits) gv.visits = diag_visits_begin(m, stream);
    if (dtype == FMGP_F64) {
      const double* q = (const double*)Q;
      rc = d == 1   ? launch_grid_query<1>(gv, q, m, kq, idx, key, stream)
           : d == 2 ? launch_grid_query<2>(gv, q, m, kq, idx, key, stream)
                    : launch_grid_query<3>(gv, q, m, kq, idx, key, stream);
    } else {
      const float* q = (const float*)Q;
      rc = d == 1   ? launch_grid_query<1>(gv, q, m, kq, idx, key, stream)
           : d == 2 ? launch_grid_query<2>(gv, q, m, kq, idx, key, stream)
                    : launch_grid_query<3>(gv, q, m, kq, idx, key, stream);
    }
    if (!rc && gv.visits) diag_visits_end(stream);
    return rc;
  }
  return knn_query_brute(X, dtype, n, d, Q, m, kq, idx, key, ws, stream);
}

int maxabs_into(const void* X, bool f64, int64_t count, unsigned int* mx, cudaStream_t s,
                const int* gate) {
  if (count <= 0) return FMGP_OK;
  const int blocks = (int)std::min<int64_t>(ceil_div(count, 256), (int64_t)num_sms() * 8);
  FMGP_LAUNCH(maxabs_kernel<<<blocks, 256, 0, s>>>(X, f64, count, mx, gate));
  FMGP_CUDA_TRY(cudaGetLastError());
  return FMGP_OK;
}

int knn_query_brute_mx(const void* X, fmgp_dtype dtype, int64_t n, int d, const void* Q,
                       int64_t m, int kq, const unsigned int* mx, int32_t* idx, double* key,
                       Workspace& ws, cudaStream_t stream) {
  if (m == 0) return FMGP_OK;
  int rc;
  if (dtype == FMGP_F64) {
    const float* Xf = brute_rows((const double*)X, n, d, ws, stream, &rc);
    if (rc) return rc;
    return launch_brute_mx<double>((const double*)X, Xf, n, d, (const double*)Q, m, kq, 0, mx,
                                   idx, key, stream);
  }
  return launch_brute_mx<float>((const float*)X, (const float*)X, n, d, (const float*)Q, m, kq,
                                0, mx, idx, key, stream);
}

__global__ void to_f32_kernel(const double* in, int64_t count, float* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}

int to_f32(const double* in, int64_t count, float* out, cudaStream_t s) {
  if (count <= 0) return FMGP_OK;
  const int blocks = (int)std::min<int64_t>(ceil_div(count, 256), (int64_t)num_sms() * 8);
  FMGP_LAUNCH(to_f32_kernel<<<blocks, 256, 0, s>>>(in, count, out));
  FMGP_CUDA_TRY(cudaGetLastError());
  return FMGP_OK;
}

int nearest_scan(const void* X, fmgp_dtype dtype, int64_t n, int d, const void* Q, int64_t m,
                 const unsigned int* mx, int32_t* nearest, Workspace& ws, cudaStream_t stream,
                 const float* Xf32) {
  if (m == 0) return FMGP_OK;
  if (!mx) {
    unsigned int* own = ws.get<unsigned int>(1);
    if (!own) return FMGP_ENOMEM;
    FMGP_CUDA_TRY(cudaMemsetAsync(own, 0, sizeof(unsigned int), stream));
    int rc = maxabs_into(X, dtype == FMGP_F64, n * d, own, stream);
    if (!rc) rc = maxabs_into(Q, dtype == FMGP_F64, m * d, own, stream);
    if (rc) return rc;
    mx = own;
  }
  if (dtype == FMGP_F64) {
    // the candidate tiles are staged from an FP32 copy (converted once here
    // unless the caller keeps one): converting per tile would load the FP64 pipe
    if (!Xf32) {
      float* own = ws.get<float>((size_t)n * d);
      if (!own) return FMGP_ENOMEM;
      const int rc = to_f32((const double*)X, n * d, own, stream);
      if (rc) return rc;
      Xf32 = own;
    }
    return nn1_scan_t<double>((const double*)X, Xf32, n, d, (const double*)Q, m, mx, nearest,
                              ws, stream);
  }
  return nn1_scan_t<float>((const float*)X, (const float*)X, n, d, (const float*)Q, m, mx,
                           nearest, ws, stream);
}

int knn_query_brute(const void* X, fmgp_dtype dtype, int64_t n, int d, const void* Q, int64_t m,
                    int kq, int32_t* idx, double* key, Workspace& ws, cudaStream_t stream) {
  if (m == 0) return FMGP_OK;
  if (tc_knn_eligible(n, d, m, kq))
    return tc_knn(X, dtype, n, d, Q, m, kq, false, idx, key, ws, stream);
  if (dtype == FMGP_F64)
    return launch_brute<double>((const double*)X, n, d, (const double*)Q, m, kq, 0, ws, idx, key,
                                stream);
  return launch_brute<float>((const float*)X, n, d, (const float*)Q, m, kq, 0, ws, idx, key,
                             stream);
}

}  // namespace fmgp
