// haar_launch.cuh -- __global__ wrappers around the tile functions and the
// launcher templates instantiated once per storage type.
#pragma once

#include <type_traits>

#include "haar_internal.h"
#include "haar_fast1d.cuh"
#include "haar_fast2d.cuh"
#include "haar_fast2d_wide.cuh"
#include "haar_ragged.cuh"
#include "haar_kernels.cuh"

namespace fh {

constexpr int kNT2 = 256;  // threads per 2D block

template <typename T, typename A>
__device__ __forceinline__ void* ll_ptr(void* base, int ll_acc, int64_t off) {
  return ll_acc ? (void*)(static_cast<A*>(base) + off) : (void*)(static_cast<T*>(base) + off);
}

template <typename Tin, typename Tout>
__device__ __forceinline__ Tile2 make_tile2_fwd(const Pass& p, int64_t tile, int TH, int TW) {
  using A = typename AccT<Tin>::type;
  const int64_t per = p.tiles_x * p.tiles_y;
  const int64_t b = tile / per, r = tile - b * per;
  const int64_t ty = r / p.tiles_x, tx = r - ty * p.tiles_x;
  Tile2 t;
  t.src = static_cast<const Tin*>(p.src) + b * p.s_bs;
  t.s_rs = p.s_rs;
  t.dst = static_cast<Tout*>(p.dst) + b * p.d_bs;
  t.d_rs = p.d_rs;
  t.ll = ll_ptr<Tout, A>(p.ll, p.ll_acc, b * p.l_bs);
  t.l_rs = p.l_rs;
  t.ll_acc = p.ll_acc;
  t.levels = p.levels;
  t.h = p.h;
  t.w = p.w;
  t.y0 = ty * TH;
  t.x0 = tx * TW;
  return t;
}

template <typename Tin, typename Tout>
__device__ __forceinline__ Tile2 make_tile2_inv(const Pass& p, int64_t tile, int TH, int TW) {
  using A = typename AccT<Tin>::type;
  const int64_t per = p.tiles_x * p.tiles_y;
  const int64_t b = tile / per, r = tile - b * per;
  const int64_t ty = r / p.tiles_x, tx = r - ty * p.tiles_x;
  Tile2 t;
  t.src = static_cast<const Tin*>(p.src) + b * p.s_bs;
  t.s_rs = p.s_rs;
  t.dst = static_cast<Tout*>(p.dst) + b * p.d_bs;
  t.d_rs = p.d_rs;
  t.ll = ll_ptr<Tin, A>(p.ll, p.ll_acc, b * p.l_bs);
  t.l_rs = p.l_rs;
  t.ll_acc = p.ll_acc;
  t.levels = p.levels;
  t.h = p.h;
  t.w = p.w;
  t.y0 = ty * TH;
  t.x0 = tx * TW;
  return t;
}

template <typename Tin, typename Tout, int TH, int TW, bool VEC>
__global__ void __launch_bounds__(kNT2) k_dwt2d(const Pass p) {
  pdl_wait();
  pdl_trigger();
  using A = typename AccT<Tin>::type;
  __shared__ __align__(16) A S[TH / 2][TW / 2 + kPad];
  for (int64_t tile = blockIdx.x; tile < p.ntiles; tile += gridDim.x) {
    const Tile2 t = make_tile2_fwd<Tin, Tout>(p, tile, TH, TW);
    dwt2d_tile<Tin, Tout, TH, TW, kNT2, VEC>(t, S);
    __syncthreads();
  }
}

template <typename Tin, typename Tout, int TH, int TW, bool VEC>
__global__ void __launch_bounds__(kNT2) k_idwt2d(const Pass p) {
  pdl_wait();
  pdl_trigger();
  using A = typename AccT<Tin>::type;
  __shared__ __align__(16) A S[TH / 2][TW / 2 + kPad];
  for (int64_t tile = blockIdx.x; tile < p.ntiles; tile += gridDim.x) {
    const Tile2 t = make_tile2_inv<Tin, Tout>(p, tile, TH, TW);
    idwt2d_tile<Tin, Tout, TH, TW, kNT2, VEC>(t, S);
    __syncthreads();
  }
}

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

inline unsigned grid_for(int64_t ntiles, int grid_cap) {
  int64_t g = ntiles;
  if (grid_cap > 0 && g > grid_cap) g = grid_cap;
  if (g > 0x7fffffffLL) g = 0x7fffffffLL;
  return (unsigned)g;
}

// The wide-lane analysis of 1- and 2-byte images (haar_fast2d_wide.cuh):
// 2-warp blocks (a block row is one or two 128-byte lines), 32 resident warps
// per SM (64 registers), L2 warm-up in the first wave.
template <typename Tin, typename Tout>
cudaError_t dwt2d_t(Pass p, int cfg, bool vec, int grid_cap, cudaStream_t s) {
  if constexpr (sizeof(Tin) <= 2) {
    if (cfg == kFast && wide_ok<Tin, Tout>(p)) return dwt2d_w_cfg<Tin, Tout, 2, 32, 2>(p, s);
  }
  if (cfg == kFast) return dwt2d_fast_t<Tin, Tout>(p, s);
  const int TH = vec ? tile_h(cfg) : 64, TW = vec ? tile_w(cfg) : 64;
  p.tiles_x = ceil_div(p.w, TW);
  p.tiles_y = ceil_div(p.h, TH);
  p.ntiles = p.batch * p.tiles_x * p.tiles_y;
  if (p.ntiles == 0) return cudaSuccess;
  const unsigned g = grid_for(p.ntiles, grid_cap);
  cudaError_t e = cudaSuccess;
  if (!vec)
    e = launch_pdl(k_dwt2d<Tin, Tout, 64, 64, false>, g, kNT2, s, p);
  else if (cfg == kT32x128)
    e = launch_pdl(k_dwt2d<Tin, Tout, 32, 128, true>, g, kNT2, s, p);
  else if (cfg == kT64x128)
    e = launch_pdl(k_dwt2d<Tin, Tout, 64, 128, true>, g, kNT2, s, p);
  else
    e = launch_pdl(k_dwt2d<Tin, Tout, 64, 64, true>, g, kNT2, s, p);
  return e;
}

template <typename Tin, typename Tout>
cudaError_t idwt2d_t(Pass p, int cfg, bool vec, int grid_cap, cudaStream_t s) {
  if (cfg == kFast) return idwt2d_fast_t<Tin, Tout>(p, s);
  const int TH = vec ? tile_h(cfg) : 64, TW = vec ? tile_w(cfg) : 64;
  p.tiles_x = ceil_div(p.w, TW);
  p.tiles_y = ceil_div(p.h, TH);
  p.ntiles = p.batch * p.tiles_x * p.tiles_y;
  if (p.ntiles == 0) return cudaSuccess;
  const unsigned g = grid_for(p.ntiles, grid_cap);
  cudaError_t e = cudaSuccess;
  if (!vec)
    e = launch_pdl(k_idwt2d<Tin, Tout, 64, 64, false>, g, kNT2, s, p);
  else if (cfg == kT32x128)
    e = launch_pdl(k_idwt2d<Tin, Tout, 32, 128, true>, g, kNT2, s, p);
  else if (cfg == kT64x128)
    e = launch_pdl(k_idwt2d<Tin, Tout, 64, 128, true>, g, kNT2, s, p);
  else
    e = launch_pdl(k_idwt2d<Tin, Tout, 64, 64, true>, g, kNT2, s, p);
  return e;
}

// ---------------------------------------------------------------------------
// 1D: every row of every batch item is a signal of length w; tiles are
// (signal, chunk) pairs.
// ---------------------------------------------------------------------------
template <typename Tin, typename Tout, int CH, int NT, bool VEC>
__global__ void __launch_bounds__(NT) k_dwt1d(const Pass p) {
  pdl_wait();
  pdl_trigger();
  using A = typename AccT<Tin>::type;
  __shared__ __align__(16) A S[CH / 2];
  for (int64_t tile = blockIdx.x; tile < p.ntiles; tile += gridDim.x) {
    const int64_t sig = tile / p.tiles_x, ch = tile - sig * p.tiles_x;
    const int64_t b = sig / p.h, y = sig - b * p.h;
    Tile1 t;
    t.src = static_cast<const Tin*>(p.src) + b * p.s_bs + y * p.s_rs;
    t.dst = static_cast<Tout*>(p.dst) + b * p.d_bs + y * p.d_rs;
    t.ll = ll_ptr<Tout, A>(p.ll, p.ll_acc, b * p.l_bs + y * p.l_rs);
    t.ll_acc = p.ll_acc;
    t.levels = p.levels;
    t.n = p.w;
    t.x0 = ch * CH;
    dwt1d_chunk<Tin, Tout, CH, NT, VEC>(t, S);
    __syncthreads();
  }
}

template <typename Tin, typename Tout, int CH, int NT, bool VEC>
__global__ void __launch_bounds__(NT) k_idwt1d(const Pass p) {
  pdl_wait();
  pdl_trigger();
  using A = typename AccT<Tin>::type;
  __shared__ __align__(16) A S[CH / 2];
  for (int64_t tile = blockIdx.x; tile < p.ntiles; tile += gridDim.x) {
    const int64_t sig = tile / p.tiles_x, ch = tile - sig * p.tiles_x;
    const int64_t b = sig / p.h, y = sig - b * p.h;
    Tile1 t;
    t.src = static_cast<const Tin*>(p.src) + b * p.s_bs + y * p.s_rs;
    t.dst = static_cast<Tout*>(p.dst) + b * p.d_bs + y * p.d_rs;
    t.ll = ll_ptr<Tin, A>(p.ll, p.ll_acc, b * p.l_bs + y * p.l_rs);
    t.ll_acc = p.ll_acc;
    t.levels = p.levels;
    t.n = p.w;
    t.x0 = ch * CH;
    idwt1d_chunk<Tin, Tout, CH, NT, VEC>(t, S);
    __syncthreads();
  }
}

template <typename Tin, typename Tout>
cudaError_t dwt1d_t(Pass p, int cfg, bool vec, cudaStream_t s) {
  if (cfg == kFast1) return dwt1d_fast_t<Tin, Tout>(p, true, s);
  const int CH = cfg == kC1024 ? 1024 : 4096;
  p.tiles_x = ceil_div(p.w, CH);
  p.tiles_y = 1;
  p.ntiles = p.batch * p.h * p.tiles_x;
  if (p.ntiles == 0) return cudaSuccess;
  const unsigned g = grid_for(p.ntiles, 0);
  cudaError_t e = cudaSuccess;
  if (cfg == kC1024) {
    if (vec)
      e = launch_pdl(k_dwt1d<Tin, Tout, 1024, 128, true>, g, 128, s, p);
    else
      e = launch_pdl(k_dwt1d<Tin, Tout, 1024, 128, false>, g, 128, s, p);
  } else {
    if (vec)
      e = launch_pdl(k_dwt1d<Tin, Tout, 4096, 256, true>, g, 256, s, p);
    else
      e = launch_pdl(k_dwt1d<Tin, Tout, 4096, 256, false>, g, 256, s, p);
  }
  return e;
}

template <typename Tin, typename Tout>
cudaError_t idwt1d_t(Pass p, int cfg, bool vec, cudaStream_t s) {
  if (cfg == kFast1) return dwt1d_fast_t<Tin, Tout>(p, false, s);
  const int CH = cfg == kC1024 ? 1024 : 4096;
  p.tiles_x = ceil_div(p.w, CH);
  p.tiles_y = 1;
  p.ntiles = p.batch * p.h * p.tiles_x;
  if (p.ntiles == 0) return cudaSuccess;
  const unsigned g = grid_for(p.ntiles, 0);
  cudaError_t e = cudaSuccess;
  if (cfg == kC1024) {
    if (vec)
      e = launch_pdl(k_idwt1d<Tin, Tout, 1024, 128, true>, g, 128, s, p);
    else
      e = launch_pdl(k_idwt1d<Tin, Tout, 1024, 128, false>, g, 128, s, p);
  } else {
    if (vec)
      e = launch_pdl(k_idwt1d<Tin, Tout, 4096, 256, true>, g, 256, s, p);
    else
      e = launch_pdl(k_idwt1d<Tin, Tout, 4096, 256, false>, g, 256, s, p);
  }
  return e;
}

// Dispatch on the output type for one input type.
#define FH_TOUT_SWITCH_FLOATS(CALL_F32, CALL_BF16, CALL_F16) \
  switch (tout) {                                            \
    case kF32: return CALL_F32;                              \
    case kBF16: return CALL_BF16;                            \
    case kF16: return CALL_F16;                              \
    default: return cudaErrorInvalidValue;                   \
  }

}  // namespace fh
