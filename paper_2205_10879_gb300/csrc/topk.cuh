// Warp-distributed sorted list of the best (key, index) pairs, used by the
// exact k-nearest-neighbour searches.  Lane l holds list positions
// l*L .. l*L+L-1 (ascending); empty positions hold (~0, INT_MAX).
#pragma once
#include "common.cuh"

namespace fmgp {

template <int L>
struct WarpTopK {
  unsigned long long k[L];
  int i[L];
  unsigned long long tk;  // key of position kq-1 (the current k-th best), ~0 while not full
  int ti;
  float t_up;             // FP32 upper bound of tk
  int tl, ts;             // lane and slot of position kq-1

  __device__ __forceinline__ void init(int kq) {
#pragma unroll
    for (int s = 0; s < L; ++s) { k[s] = ~0ull; i[s] = INT_MAX; }
    tk = ~0ull;
    ti = INT_MAX;
    t_up = __int_as_float(0x7f800000);
    tl = (kq - 1) / L;
    ts = (kq - 1) % L;
  }

  __device__ __forceinline__ bool full() const { return tk != ~0ull; }

  __device__ __forceinline__ bool admits(unsigned long long ck, int ci) const {
    return key_less(ck, ci, tk, ti);
  }

  // Insert (bk, bi) (warp-uniform arguments); it must not already be present.
  __device__ __forceinline__ void insert(unsigned long long bk, int bi, int lane) {
    int cnt = 0;
#pragma unroll
    for (int s = 0; s < L; ++s) cnt += key_less(k[s], i[s], bk, bi) ? 1 : 0;
    const int pos = __reduce_add_sync(kFull, cnt);
    const unsigned long long pk = __shfl_up_sync(kFull, k[L - 1], 1);
    const int pi = __shfl_up_sync(kFull, i[L - 1], 1);
#pragma unroll
    for (int s = L - 1; s >= 0; --s) {
      const int g = lane * L + s;
      if (g > pos) {
        if (s > 0) { k[s] = k[s - 1]; i[s] = i[s - 1]; }
        else { k[s] = pk; i[s] = pi; }
      } else if (g == pos) {
        k[s] = bk;
        i[s] = bi;
      }
    }
    unsigned long long mk = k[0];
    int mi = i[0];
#pragma unroll
    for (int s = 1; s < L; ++s)
      if (s == ts) { mk = k[s]; mi = i[s]; }
    tk = __shfl_sync(kFull, mk, tl);
    ti = __shfl_sync(kFull, mi, tl);
    // t_up is refreshed by the caller (offer) once its inserts are done
  }

  // Into an empty list (just after init), put the one candidate per lane
  // (ck = ~0 for none) in order: a bitonic sort across the warp by (key,
  // index), then lane l takes sorted positions l*L .. l*L+L-1.  The same list
  // as offering them one by one, for the cost of one sorting network.
  __device__ __forceinline__ void fill_sorted(unsigned long long ck, int ci, int lane) {
#pragma unroll
    for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        const unsigned long long ok = __shfl_xor_sync(kFull, ck, stride);
        const int oi = __shfl_xor_sync(kFull, ci, stride);
        const bool asc = (lane & size) == 0;
        const bool low = (lane & stride) == 0;
        // the lower lane of a pair keeps the smaller in an ascending run
        const bool take = (low == asc) ? key_less(ok, oi, ck, ci) : key_less(ck, ci, ok, oi);
        if (take) { ck = ok; ci = oi; }
      }
    }
#pragma unroll
    for (int s = 0; s < L; ++s) {
      const int src = lane * L + s;
      const unsigned long long vk = __shfl_sync(kFull, ck, src & 31);
      const int vi = __shfl_sync(kFull, ci, src & 31);
      k[s] = src < 32 ? vk : ~0ull;
      i[s] = src < 32 ? vi : INT_MAX;
    }
    unsigned long long mk = k[0];
    int mi = i[0];
#pragma unroll
    for (int s = 1; s < L; ++s)
      if (s == ts) { mk = k[s]; mi = i[s]; }
    tk = __shfl_sync(kFull, mk, tl);
    ti = __shfl_sync(kFull, mi, tl);
    t_up = key_bits_to_float_up(tk);
  }

  // Offer one candidate per lane (ck = ~0 for none); inserts every candidate
  // that belongs in the list, lowest lane first.  The inserts keep (tk, ti)
  // current for the admission test; the FP32 bound t_up, which only the
  // search's pruning reads, is formed once afterwards.
  __device__ __forceinline__ void offer(unsigned long long ck, int ci, int lane) {
    unsigned hits = __ballot_sync(kFull, admits(ck, ci));
    if (!hits) return;
    while (hits) {
      const int src = __ffs(hits) - 1;
      const unsigned long long bk = __shfl_sync(kFull, ck, src);
      const int bi = __shfl_sync(kFull, ci, src);
      insert(bk, bi, lane);
      hits &= ~(1u << src);
      hits &= __ballot_sync(kFull, admits(ck, ci));
    }
    t_up = key_bits_to_float_up(tk);
  }

  __device__ __forceinline__ void store(int kq, int lane, int32_t* idx_row, double* key_row) const {
#pragma unroll
    for (int s = 0; s < L; ++s) {
      const int g = lane * L + s;
      if (g < kq) {
        idx_row[g] = i[s];
        if (key_row) key_row[g] = __longlong_as_double((long long)k[s]);
      }
    }
  }
};

// The same list with 32-bit keys (the bits of non-negative FP32 values, whose
// order as unsigned integers is their numeric order): half the compare and
// shuffle work of the 64-bit list, for searches that rank FP32 distances.
template <int L>
struct WarpTopK32 {
  unsigned int k[L];
  int i[L];
  unsigned int tk;  // key of position kq-1, ~0 while not full
  int ti;
  int tl, ts;

  __device__ __forceinline__ static bool less(unsigned int ka, int ia, unsigned int kb, int ib) {
    return ka < kb || (ka == kb && ia < ib);
  }

  __device__ __forceinline__ void init(int kq) {
#pragma unroll
    for (int s = 0; s < L; ++s) { k[s] = ~0u; i[s] = INT_MAX; }
    tk = ~0u;
    ti = INT_MAX;
    tl = (kq - 1) / L;
    ts = (kq - 1) % L;
  }

  __device__ __forceinline__ bool full() const { return tk != ~0u; }

  __device__ __forceinline__ void refresh_threshold() {
    unsigned int mk = k[0];
    int mi = i[0];
#pragma unroll
    for (int s = 1; s < L; ++s)
      if (s == ts) { mk = k[s]; mi = i[s]; }
    tk = __shfl_sync(kFull, mk, tl);
    ti = __shfl_sync(kFull, mi, tl);
  }

  __device__ __forceinline__ void insert(unsigned int bk, int bi, int lane) {
    int cnt = 0;
#pragma unroll
    for (int s = 0; s < L; ++s) cnt += less(k[s], i[s], bk, bi) ? 1 : 0;
    const int pos = __reduce_add_sync(kFull, cnt);
    const unsigned int pk = __shfl_up_sync(kFull, k[L - 1], 1);
    const int pi = __shfl_up_sync(kFull, i[L - 1], 1);
#pragma unroll
    for (int s = L - 1; s >= 0; --s) {
      const int g = lane * L + s;
      if (g > pos) {
        if (s > 0) { k[s] = k[s - 1]; i[s] = i[s - 1]; }
        else { k[s] = pk; i[s] = pi; }
      } else if (g == pos) {
        k[s] = bk;
        i[s] = bi;
      }
    }
    refresh_threshold();
  }

  // Offer one candidate per lane (ck = ~0 for none).
  __device__ __forceinline__ void offer(unsigned int ck, int ci, int lane) {
    unsigned hits = __ballot_sync(kFull, less(ck, ci, tk, ti));
    while (hits) {
      const int src = __ffs(hits) - 1;
      const unsigned int bk = __shfl_sync(kFull, ck, src);
      const int bi = __shfl_sync(kFull, ci, src);
      insert(bk, bi, lane);
      hits &= ~(1u << src);
      hits &= __ballot_sync(kFull, less(ck, ci, tk, ti));
    }
  }
};

// Warp argmin of (key, index) pairs.
__device__ __forceinline__ void warp_argmin(unsigned long long& bk, int& bi) {
#pragma unroll
  for (int off = 16; off; off >>= 1) {
    unsigned long long ok = __shfl_xor_sync(kFull, bk, off);
    int oi = __shfl_xor_sync(kFull, bi, off);
    if (key_less(ok, oi, bk, bi)) { bk = ok; bi = oi; }
  }
}

}  // namespace fmgp
