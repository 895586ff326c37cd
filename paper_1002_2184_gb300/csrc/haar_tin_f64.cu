// Launchers for fp64 storage and arithmetic (gradient checks only).
#include "haar_launch.cuh"

namespace fh {

cudaError_t launch_dwt2d_f64(int tout, Pass p, int cfg, bool vec, int cap, cudaStream_t s) {
  if (tout != kF64) return cudaErrorInvalidValue;
  return dwt2d_t<double, double>(p, cfg, vec, cap, s);
}

cudaError_t launch_idwt2d_f64(int tout, Pass p, int cfg, bool vec, int cap, cudaStream_t s) {
  if (tout != kF64) return cudaErrorInvalidValue;
  return idwt2d_t<double, double>(p, cfg, vec, cap, s);
}

cudaError_t launch_dwt1d_f64(int tout, Pass p, int cfg, bool vec, cudaStream_t s) {
  if (tout != kF64) return cudaErrorInvalidValue;
  return dwt1d_t<double, double>(p, cfg, vec, s);
}

cudaError_t launch_idwt1d_f64(int tout, Pass p, int cfg, bool vec, cudaStream_t s) {
  if (tout != kF64) return cudaErrorInvalidValue;
  return idwt1d_t<double, double>(p, cfg, vec, s);
}

cudaError_t launch_ragged_f64(int tout, bool fwd, const RaggedArgs& a, int unit, unsigned grid,
                             cudaStream_t s) {
  if (tout != kF64) return cudaErrorInvalidValue;
  return ragged_t<double, double>(fwd, a, unit, grid, s);
}

}  // namespace fh
