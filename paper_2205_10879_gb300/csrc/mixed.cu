// Mixed-precision block and prediction kernels (placeholder until written).
#include "block.cuh"
#include "predict.cuh"

namespace fmgp {

size_t block_mixed_extra_bytes(int, int, int) { return 0; }

int launch_block_mixed(const BlockArgs&, const void*, fmgp_dtype, bool, int, cudaStream_t) {
  set_error("mixed precision not built yet");
  return FMGP_EUNSUPPORTED;
}

int gather_dot_mixed(const void*, fmgp_dtype, int64_t, int, const int32_t*, int, const void*, int,
                     int, const KParams&, const void*, int64_t, const int32_t*, double*,
                     cudaStream_t) {
  set_error("mixed precision not built yet");
  return FMGP_EUNSUPPORTED;
}

}  // namespace fmgp
