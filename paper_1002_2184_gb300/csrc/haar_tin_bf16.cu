// Launchers for __nv_bfloat16 input storage (all fp output types).
#include "haar_launch.cuh"

namespace fh {

cudaError_t launch_dwt2d_bf16(int tout, Pass p, int cfg, bool vec, int cap, cudaStream_t s) {
  FH_TOUT_SWITCH_FLOATS((dwt2d_t<__nv_bfloat16, float>(p, cfg, vec, cap, s)),
                        (dwt2d_t<__nv_bfloat16, __nv_bfloat16>(p, cfg, vec, cap, s)),
                        (dwt2d_t<__nv_bfloat16, __half>(p, cfg, vec, cap, s)))
}

cudaError_t launch_idwt2d_bf16(int tout, Pass p, int cfg, bool vec, int cap, cudaStream_t s) {
  FH_TOUT_SWITCH_FLOATS((idwt2d_t<__nv_bfloat16, float>(p, cfg, vec, cap, s)),
                        (idwt2d_t<__nv_bfloat16, __nv_bfloat16>(p, cfg, vec, cap, s)),
                        (idwt2d_t<__nv_bfloat16, __half>(p, cfg, vec, cap, s)))
}

cudaError_t launch_dwt1d_bf16(int tout, Pass p, int cfg, bool vec, cudaStream_t s) {
  FH_TOUT_SWITCH_FLOATS((dwt1d_t<__nv_bfloat16, float>(p, cfg, vec, s)),
                        (dwt1d_t<__nv_bfloat16, __nv_bfloat16>(p, cfg, vec, s)),
                        (dwt1d_t<__nv_bfloat16, __half>(p, cfg, vec, s)))
}

cudaError_t launch_idwt1d_bf16(int tout, Pass p, int cfg, bool vec, cudaStream_t s) {
  FH_TOUT_SWITCH_FLOATS((idwt1d_t<__nv_bfloat16, float>(p, cfg, vec, s)),
                        (idwt1d_t<__nv_bfloat16, __nv_bfloat16>(p, cfg, vec, s)),
                        (idwt1d_t<__nv_bfloat16, __half>(p, cfg, vec, s)))
}

cudaError_t launch_ragged_bf16(int tout, bool fwd, const RaggedArgs& a, int unit, unsigned grid,
                             cudaStream_t s) {
  FH_TOUT_SWITCH_FLOATS((ragged_t<__nv_bfloat16, float>(fwd, a, unit, grid, s)),
                        (ragged_t<__nv_bfloat16, __nv_bfloat16>(fwd, a, unit, grid, s)),
                        (ragged_t<__nv_bfloat16, __half>(fwd, a, unit, grid, s)))
}

}  // namespace fh
