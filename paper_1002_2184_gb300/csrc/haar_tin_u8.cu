// Launchers for uint8 input storage: analysis only (coefficients are never
// stored as uint8).
#include "haar_launch.cuh"

namespace fh {

cudaError_t launch_dwt2d_u8(int tout, Pass p, int cfg, bool vec, int cap, cudaStream_t s) {
  FH_TOUT_SWITCH_FLOATS((dwt2d_t<uint8_t, float>(p, cfg, vec, cap, s)),
                        (dwt2d_t<uint8_t, __nv_bfloat16>(p, cfg, vec, cap, s)),
                        (dwt2d_t<uint8_t, __half>(p, cfg, vec, cap, s)))
}

cudaError_t launch_idwt2d_u8(int, Pass, int, bool, int, cudaStream_t) {
  return cudaErrorInvalidValue;
}

cudaError_t launch_dwt1d_u8(int tout, Pass p, int cfg, bool vec, cudaStream_t s) {
  FH_TOUT_SWITCH_FLOATS((dwt1d_t<uint8_t, float>(p, cfg, vec, s)),
                        (dwt1d_t<uint8_t, __nv_bfloat16>(p, cfg, vec, s)),
                        (dwt1d_t<uint8_t, __half>(p, cfg, vec, s)))
}

cudaError_t launch_idwt1d_u8(int, Pass, int, bool, cudaStream_t) {
  return cudaErrorInvalidValue;
}

cudaError_t launch_ragged_u8(int tout, bool fwd, const RaggedArgs& a, int unit, unsigned grid,
                            cudaStream_t s) {
  if (!fwd) return cudaErrorInvalidValue;
  FH_TOUT_SWITCH_FLOATS((ragged_t<uint8_t, float>(true, a, unit, grid, s)),
                        (ragged_t<uint8_t, __nv_bfloat16>(true, a, unit, grid, s)),
                        (ragged_t<uint8_t, __half>(true, a, unit, grid, s)))
}

}  // namespace fh
