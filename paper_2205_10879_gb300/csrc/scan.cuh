// Exclusive prefix sum of int counts (device), used to turn per-cell counts
// into the cell start offsets of the sorted point array.
#pragma once
#include "common.cuh"

namespace fmgp {
// out[0..count] = exclusive scan of in[0..count), out[count] = total.
// count <= 4096 * 4096.  Returns FMGP_OK or an error code.
int exclusive_scan_int(const int* in, int* out, int count, Workspace& ws, cudaStream_t stream);
}  // namespace fmgp
