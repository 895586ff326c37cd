// haar_ragged.cuh -- one persistent launch over a ragged batch of images of
// different sizes and level counts.
//
// The work is cut into units of UH x UW pixels (one 32 x 32 block per warp,
// the same per-warp bodies as the strided-batch kernels; 64 x 128, 32 x 256,
// 64 x 64 or 128 x 128, picked by the autotuner).  A plan
// lists, per image, its first unit index; blocks take units from a global
// atomic counter, find the image by binary search, and transform.  The last
// block to finish resets the counter, so the launch can be replayed (for
// instance from a CUDA graph) without any host work; it also checks that
// every unit was handed out exactly once and records an error word if not.
#pragma once

#include <type_traits>

#include "haar_fast2d.cuh"
#include "haar_internal.h"

namespace fh {

// Takes the next unit; returns its index (>= total when the queue is empty)
// and the image it belongs to (shared by the whole block).
__device__ __forceinline__ long long ragged_next(const RaggedArgs& a, long long* s_unit,
                                                 int* s_img, int& img_out) {
  if (threadIdx.x == 0) {
    const long long u = (long long)atomicAdd(&a.hdr->next_unit, 1ull);
    int img = -1;
    if (u < a.total_units) {
      int64_t lo = 0, hi = a.n_imgs - 1;
      while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (a.imgs[mid].unit_begin <= u)
          lo = mid;
        else
          hi = mid - 1;
      }
      img = (int)lo;
    }
    *s_unit = u;
    *s_img = img;
  }
  __syncthreads();
  const long long u = *s_unit;
  img_out = *s_img;
  __syncthreads();  // nobody may refill s_unit / s_img before everyone read them
  return u;
}

// Called once per block after its loop, with the number of units it
// transformed.  The last block to finish checks that every unit was
// transformed exactly once and that the queue ran out exactly when expected,
// records an error word otherwise, and resets the counters for the next
// launch.
__device__ __forceinline__ void ragged_finish(const RaggedArgs& a, long long mine) {
  if (threadIdx.x == 0) {
    atomicAdd(&a.hdr->units_done, (unsigned long long)mine);
    __threadfence();
    const unsigned long long d = atomicAdd(&a.hdr->blocks_done, 1ull);
    if (d == gridDim.x - 1) {
      __threadfence();
      const unsigned long long total = (unsigned long long)a.total_units;
      const unsigned long long done = atomicAdd(&a.hdr->units_done, 0ull);
      const unsigned long long next = atomicAdd(&a.hdr->next_unit, 0ull);
      if (done != total || next != total + gridDim.x) atomicExch(&a.hdr->error, 1ull);
      atomicExch(&a.hdr->next_unit, 0ull);
      atomicExch(&a.hdr->units_done, 0ull);
      atomicExch(&a.hdr->blocks_done, 0ull);
    }
  }
}

template <typename Tin, typename Tout>
__device__ __forceinline__ Img2 ragged_image(const RaggedArgs& a, const RaggedImg& r) {
  Img2 im;
  im.src = static_cast<const Tin*>(a.in) + r.in_off;
  im.s_rs = r.in_rs;
  im.dst = static_cast<Tout*>(a.out) + r.out_off;
  im.d_rs = r.out_rs;
  im.h = r.h;
  im.w = r.w;
  return im;
}

// Both ragged kernels: FP32 arithmetic capped at 40 registers, 48 resident
// warps per SM (8-warp units, the 512-image batch: analysis 0.706 against
// 0.783 ms at 40 warps, synthesis 0.711 against 0.741 ms); FP64 is not
// capped.  A unit of NW warps is one block of 32 NW threads.
template <typename Tin, int NW>
constexpr int ragged_min_blocks() {
  return sizeof(typename AccT<Tin>::type) == 8 ? 1 : (48 / NW > 0 ? 48 / NW : 1);
}
template <typename Tin, typename Tout, int UH, int UW>
__global__ void __launch_bounds__(UH * UW / 32, ragged_min_blocks<Tin, (UH / 32) * (UW / 32)>())
    k_ragged_dwt2d(const RaggedArgs a) {
  pdl_wait();
  pdl_trigger();
  using A = typename AccT<Tin>::type;
  constexpr int WR = UH / 32, WC = UW / 32;
  __shared__ long long s_unit;
  __shared__ int s_img;
  __shared__ A s5[WR][WC];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t limit = a.total_units + gridDim.x;  // the queue hands out at most this many
  long long mine = 0;
  for (int64_t it = 0; it < limit; ++it) {
    int img;
    const long long u = ragged_next(a, &s_unit, &s_img, img);
    if (u >= a.total_units) break;
    ++mine;
    const RaggedImg r = a.imgs[img];
    Img2 im = ragged_image<Tin, Tout>(a, r);
    im.ll = im.dst;
    im.l_rs = im.d_rs;
    im.ll_acc = 0;
    const int64_t local = u - r.unit_begin;
    const int64_t uy = local / r.units_x, ux = local - uy * r.units_x;
    const int64_t y0 = uy * UH + (warp / WC) * 32, x0 = ux * UW + (warp % WC) * 32;
    const bool act = y0 < r.h && x0 < r.w;
    switch (r.levels) {
      case 1: if (act) dwt_block32<Tin, Tout, 1>(im, y0, x0, lane); break;
      case 2: if (act) dwt_block32<Tin, Tout, 2>(im, y0, x0, lane); break;
      case 3: if (act) dwt_block32<Tin, Tout, 3>(im, y0, x0, lane); break;
      case 4: if (act) dwt_block32<Tin, Tout, 4>(im, y0, x0, lane); break;
      case 5: if (act) dwt_block32<Tin, Tout, 5>(im, y0, x0, lane); break;
      case 6:
        if constexpr (WR % 2 == 0) {
          // the unit's (WR / 2) x (WC / 2) blocks of 64 x 64 finish level 6
          // from the LL5 values of their four warps
          const A l5 = act ? dwt_block32<Tin, Tout, 6>(im, y0, x0, lane) : A(0);
          if (lane == 0) s5[warp / WC][warp % WC] = l5;
          __syncthreads();
          if (threadIdx.x < (WR / 2) * (WC / 2)) {
            const int bi = threadIdx.x / (WC / 2), bj = threadIdx.x % (WC / 2);
            const int64_t by0 = uy * UH + 64 * bi, bx0 = ux * UW + 64 * bj;
            if (by0 < r.h && bx0 < r.w)
              dwt_level6<Tout>(im, s5[2 * bi][2 * bj], s5[2 * bi][2 * bj + 1],
                               s5[2 * bi + 1][2 * bj], s5[2 * bi + 1][2 * bj + 1], by0, bx0);
          }
          // (the barriers of ragged_next order these reads before the next
          // unit rewrites s5)
        }
        break;
      default: break;
    }
  }
  ragged_finish(a, mine);
}

template <typename Tin, typename Tout, int UH, int UW>
__global__ void __launch_bounds__(UH * UW / 32, ragged_min_blocks<Tin, (UH / 32) * (UW / 32)>())
    k_ragged_idwt2d(const RaggedArgs a) {
  pdl_wait();
  pdl_trigger();
  constexpr int WC = UW / 32;
  __shared__ long long s_unit;
  __shared__ int s_img;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t limit = a.total_units + gridDim.x;
  long long mine = 0;
  for (int64_t it = 0; it < limit; ++it) {
    int img;
    const long long u = ragged_next(a, &s_unit, &s_img, img);
    if (u >= a.total_units) break;
    ++mine;
    const RaggedImg r = a.imgs[img];
    Img2 im = ragged_image<Tin, Tout>(a, r);
    im.ll = const_cast<void*>(im.src);
    im.l_rs = im.s_rs;
    im.ll_acc = 0;
    const int64_t local = u - r.unit_begin;
    const int64_t uy = local / r.units_x, ux = local - uy * r.units_x;
    const int64_t y0 = uy * UH + (warp / WC) * 32, x0 = ux * UW + (warp % WC) * 32;
    if (y0 < r.h && x0 < r.w) {
      switch (r.levels) {
        case 1: idwt_block32<Tin, Tout, 1>(im, y0, x0, lane); break;
        case 2: idwt_block32<Tin, Tout, 2>(im, y0, x0, lane); break;
        case 3: idwt_block32<Tin, Tout, 3>(im, y0, x0, lane); break;
        case 4: idwt_block32<Tin, Tout, 4>(im, y0, x0, lane); break;
        case 5: idwt_block32<Tin, Tout, 5>(im, y0, x0, lane); break;
        case 6: idwt_block32<Tin, Tout, 6>(im, y0, x0, lane); break;
        default: break;
      }
    }
  }
  ragged_finish(a, mine);
}

template <typename Tin, typename Tout>
cudaError_t ragged_t(bool fwd, const RaggedArgs& a, int unit, unsigned grid, cudaStream_t s) {
  if (a.total_units == 0 || grid == 0) return cudaSuccess;
#define FH_RAGGED_UNIT(KERNEL)                                                                  \
  switch (unit) {                                                                               \
    case kUnit64x128: return launch_pdl(KERNEL<Tin, Tout, 64, 128>, grid, 256, s, a);          \
    case kUnit32x256: return launch_pdl(KERNEL<Tin, Tout, 32, 256>, grid, 256, s, a);          \
    case kUnit64x64: return launch_pdl(KERNEL<Tin, Tout, 64, 64>, grid, 128, s, a);            \
    case kUnit128x128: return launch_pdl(KERNEL<Tin, Tout, 128, 128>, grid, 512, s, a);        \
    default: return cudaErrorInvalidValue;                                                      \
  }
  if (fwd) {
    FH_RAGGED_UNIT(k_ragged_dwt2d)
  }
  if constexpr (std::is_same<Tin, uint8_t>::value) {
    return cudaErrorInvalidValue;  // coefficients are never stored as uint8
  } else {
    FH_RAGGED_UNIT(k_ragged_idwt2d)
  }
#undef FH_RAGGED_UNIT
}

}  // namespace fh
