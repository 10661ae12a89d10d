#include "scan.cuh"

namespace fmgp {
namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanPer = 4;
constexpr int kScanChunk = kScanThreads * kScanPer;  // 4096

// Block-wide exclusive scan of kScanChunk ints starting at in + blockIdx.x*chunk.
__global__ void __launch_bounds__(kScanThreads) scan_chunks(const int* in, int* out, int count,
                                                            int* block_sums) {
  __shared__ int warp_tot[kScanThreads / kWarp];
  const int base = blockIdx.x * kScanChunk + threadIdx.x * kScanPer;
  int v[kScanPer];
  int local = 0;
#pragma unroll
  for (int t = 0; t < kScanPer; ++t) {
    v[t] = (base + t < count) ? in[base + t] : 0;
    local += v[t];
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int incl = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_tot[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    int w = warp_tot[lane];
    int wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(kFull, wi, o);
      if (lane >= o) wi += y;
    }
    warp_tot[lane] = wi - w;  // exclusive
  }
  __syncthreads();
  int run = warp_tot[wid] + incl - local;
#pragma unroll
  for (int t = 0; t < kScanPer; ++t) {
    if (base + t < count) out[base + t] = run;
    run += v[t];
  }
  if (threadIdx.x == kScanThreads - 1) block_sums[blockIdx.x] = run;
}

__global__ void add_block_offsets(int* out, int count, const int* block_offsets) {
  const int b = blockIdx.x;
  const int add = block_offsets[b];
  const int base = b * kScanChunk;
  for (int t = threadIdx.x; t < kScanChunk; t += blockDim.x)
    if (base + t < count) out[base + t] += add;
}

__global__ void write_total(int* out, int count, const int* block_offsets, int nblocks) {
  out[count] = block_offsets[nblocks];
}

}  // namespace

int exclusive_scan_int(const int* in, int* out, int count, Workspace& ws, cudaStream_t stream) {
  if (count <= 0) {
    FMGP_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(int), stream));
    return FMGP_OK;
  }
  const int nblocks = ceil_div(count, kScanChunk);
  if (nblocks > kScanChunk) {
    set_error("prefix sum over %d cells exceeds %d", count, kScanChunk * kScanChunk);
    return FMGP_EUNSUPPORTED;
  }
  int* sums = ws.get<int>(nblocks);
  int* offs = ws.get<int>(nblocks + 1);
  if (!sums || !offs) return FMGP_ENOMEM;
  FMGP_LAUNCH(scan_chunks<<<nblocks, kScanThreads, 0, stream>>>(in, out, count, sums));
  FMGP_LAUNCH(scan_chunks<<<1, kScanThreads, 0, stream>>>(sums, offs, nblocks, offs + nblocks));
  FMGP_LAUNCH(add_block_offsets<<<nblocks, 256, 0, stream>>>(out, count, offs));
  FMGP_LAUNCH(write_total<<<1, 1, 0, stream>>>(out, count, offs, nblocks));
  FMGP_CUDA_TRY(cudaGetLastError());
  return FMGP_OK;
}

}  // namespace fmgp
