// haar_denoise.cu -- wavelet shrinkage in one pass: analysis, thresholding of
// every detail coefficient (soft or hard; the low band is kept), synthesis.
// The signal or image is read once and the result written once; the
// coefficients live only in the registers of the warp that owns the block
// (the warp-block kernels of haar_fast1d.cuh and haar_roundtrip.cuh).
// The paper's use case is denoising of biosignals and images (Section VI);
// the shrinkage rule itself is not in the paper.
#include <cuda_runtime.h>

#include "fasthaar.h"
#include "haar_internal.h"
#include "haar_launch.cuh"
#include "haar_roundtrip.cuh"

namespace fh {

template <typename T>
__device__ __forceinline__ T shrink(T d, T t, bool hard) {
  const T a = fabs(d);
  if (hard) return a > t ? d : T(0);
  return a > t ? copysign(a - t, d) : T(0);
}

struct ShrinkArgs {
  Pass p;  // src = x, dst = y (same geometry); batch, h, w, levels
  double t;
  float t_f;  // t rounded once on the host
  int hard;
};

// ---- 1D: one warp per 256 samples ----
template <typename T, int L>
__global__ void __launch_bounds__(256) k_denoise1d(const ShrinkArgs a) {
  pdl_wait();
  pdl_trigger();
  int64_t sig, x0;
  if (!sig_block(a.p, sig, x0)) return;
  const int lane = threadIdx.x & 31;
  const Pass& p = a.p;
  const int64_t b = sig / p.h, y = sig - b * p.h;
  const T* src = static_cast<const T*>(p.src) + b * p.s_bs + y * p.s_rs;
  T* dst = static_cast<T*>(p.dst) + b * p.d_bs + y * p.d_rs;
  const int64_t px = x0 + 8 * lane;
  const T t = param<T>(a.t, a.t_f);
  const bool hard = a.hard != 0;
  T v[8];
  load8(src + px, v);
  // analysis into registers
  T a1[4], d1[4], a2[2], d2[2], dl[9], an = T(0);
#pragma unroll
  for (int k = 0; k < 4; ++k) fwd_pair(v[2 * k], v[2 * k + 1], a1[k], d1[k]);
  if constexpr (L >= 2) {
#pragma unroll
    for (int k = 0; k < 2; ++k) fwd_pair(a1[2 * k], a1[2 * k + 1], a2[k], d2[k]);
  }
  if constexpr (L >= 3) {
    fwd_pair(a2[0], a2[1], an, dl[3]);
#pragma unroll
    for (int l = 4; l <= L; ++l) {
      const int mask = 1 << (l - 4);
      T lo, hi;
      hpair1(an, (lane & mask) != 0, mask, lo, hi);
      an = lo;
      dl[l] = hi;
    }
  }
  // shrink the details
#pragma unroll
  for (int k = 0; k < 4; ++k) d1[k] = shrink(d1[k], t, hard);
  if constexpr (L >= 2) {
#pragma unroll
    for (int k = 0; k < 2; ++k) d2[k] = shrink(d2[k], t, hard);
  }
#pragma unroll
  for (int l = 3; l <= L; ++l) dl[l] = shrink(dl[l], t, hard);
  // synthesis back in registers
  if constexpr (L >= 3) {
    T w = an;
#pragma unroll
    for (int l = L; l >= 4; --l) w = inv_child1(w, dl[l], (int)((px >> (l - 1)) & 1));
    inv_pair(w, dl[3], a2[0], a2[1]);
  }
  if constexpr (L >= 2) {
#pragma unroll
    for (int k = 0; k < 2; ++k) inv_pair(a2[k], d2[k], a1[2 * k], a1[2 * k + 1]);
  }
  T o[8];
#pragma unroll
  for (int k = 0; k < 4; ++k) inv_pair(a1[k], d1[k], o[2 * k], o[2 * k + 1]);
  store8(dst + px, o);
}

// ---- 2D: one warp per 32 x 32 block ----
template <typename T>
struct OpShrink {
  T t;
  bool hard;
  __device__ __forceinline__ T operator()(T c, bool detail, bool) {
    return detail ? shrink(c, t, hard) : c;
  }
};

template <typename T, int L>
__global__ void __launch_bounds__(256) k_denoise2d(const ShrinkArgs a) {
  pdl_wait();
  pdl_trigger();
  const Pass& p = a.p;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t per = p.tiles_x * p.tiles_y;
  const int64_t bt = blockIdx.x;
  const int64_t b = bt / per, rr = bt - b * per;
  const int64_t cy = rr / p.tiles_x, cx = rr - cy * p.tiles_x;
  const int64_t y0 = cy * 32, x0 = cx * 256 + warp * 32;
  if (y0 >= p.h || x0 >= p.w) return;
  const int64_t py = y0 + 4 * (lane >> 2), px = x0 + 8 * (lane & 3);
  const T* src = static_cast<const T*>(p.src) + b * p.s_bs;
  T* dst = static_cast<T*>(p.dst) + b * p.d_bs + py * p.d_rs + px;
  WarpCoefs<T, L> k;
  warp_analysis<T, L>(src + py * p.s_rs + px, p.s_rs, lane, k);
  OpShrink<T> op{param<T>(a.t, a.t_f), a.hard != 0};
  warp_map<T, L>(lane, k, op);
  T o[4][8];
  warp_synthesis<T, L>(lane, py, px, k, o);
#pragma unroll
  for (int i = 0; i < 4; ++i) store8(dst + i * p.d_rs, o[i]);
}

template <typename T>
cudaError_t shrink_launch(bool two_d, ShrinkArgs a, cudaStream_t s) {
  Pass& p = a.p;
  if (two_d) {
    p.tiles_x = (p.w + 255) / 256;
    p.tiles_y = (p.h + 31) / 32;
    p.ntiles = p.batch * p.tiles_x * p.tiles_y;
  } else {
    p.tiles_x = (p.w + 2047) / 2048;
    p.tiles_y = 1;
    p.ntiles = p.batch * p.h * p.tiles_x;
  }
  if (p.ntiles == 0) return cudaSuccess;
  if (p.ntiles > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  const unsigned g = (unsigned)p.ntiles;
#define FH_SH2(LV) \
  case LV: return launch_pdl(k_denoise2d<T, LV>, g, 256, s, a);
#define FH_SH1(LV) \
  case LV: return launch_pdl(k_denoise1d<T, LV>, g, 256, s, a);
  if (two_d) {
    switch (p.levels) {
      FH_SH2(1) FH_SH2(2) FH_SH2(3) FH_SH2(4) FH_SH2(5)
      default: return cudaErrorInvalidValue;
    }
  }
  switch (p.levels) {
    FH_SH1(1) FH_SH1(2) FH_SH1(3) FH_SH1(4) FH_SH1(5) FH_SH1(6) FH_SH1(7) FH_SH1(8)
    default: return cudaErrorInvalidValue;
  }
#undef FH_SH1
#undef FH_SH2
}

}  // namespace fh

using namespace fh;

namespace {

int shrink_entry(const haar_desc* x, const haar_desc* y, int levels, double threshold, int mode,
                 void* stream, bool two_d) {
  if (!x || !y || x->reserved || y->reserved) return HAAR_EINVAL;
  if (x->dtype != y->dtype) return HAAR_EDTYPE;
  if (x->dtype != HAAR_F32 && x->dtype != HAAR_F64) return HAAR_EDTYPE;
  if (x->batch != y->batch || x->h != y->h || x->w != y->w) return HAAR_EINVAL;
  if (x->batch < 0 || x->h < 0 || x->w < 0 || x->batch_stride < 0 || x->row_stride < 0 ||
      y->batch_stride < 0 || y->row_stride < 0)
    return HAAR_EINVAL;
  if (mode != HAAR_THRESH_SOFT && mode != HAAR_THRESH_HARD) return HAAR_EINVAL;
  if (!(threshold >= 0.0)) return HAAR_EINVAL;
  if (levels < 1 || levels > (two_d ? 5 : 8)) return HAAR_EINVAL;
  if (x->batch == 0 || x->h == 0 || x->w == 0) return HAAR_OK;
  if (!x->ptr || !y->ptr) return HAAR_EINVAL;
  if (two_d ? (x->h % 32 || x->w % 32) : (x->w % 256)) return HAAR_ESHAPE;
  if (x->h > 1 && (x->row_stride < x->w || y->row_stride < y->w)) return HAAR_EINVAL;
  const int64_t rows = two_d ? x->h : 1;
  if (x->batch > 1 && (x->batch_stride < (rows - 1) * x->row_stride + x->w ||
                       y->batch_stride < (rows - 1) * y->row_stride + y->w))
    return HAAR_EINVAL;
  const int esz = x->dtype == HAAR_F64 ? 8 : 4;
  if (((uintptr_t)x->ptr | (uintptr_t)y->ptr) % 16 || (x->row_stride * esz) % 16 ||
      (y->row_stride * esz) % 16 || (x->batch_stride * esz) % 16 || (y->batch_stride * esz) % 16)
    return HAAR_EINVAL;
  const int64_t ex = (x->batch - 1) * x->batch_stride + (x->h - 1) * x->row_stride + x->w;
  const int64_t ey = (y->batch - 1) * y->batch_stride + (y->h - 1) * y->row_stride + y->w;
  const uintptr_t xl = (uintptr_t)x->ptr, yl = (uintptr_t)y->ptr;
  if (xl < yl + (uintptr_t)ey * esz && yl < xl + (uintptr_t)ex * esz) return HAAR_EALIAS;
  ShrinkArgs a{};
  a.p.src = x->ptr;
  a.p.s_bs = x->batch_stride;
  a.p.s_rs = x->row_stride;
  a.p.dst = y->ptr;
  a.p.d_bs = y->batch_stride;
  a.p.d_rs = y->row_stride;
  a.p.levels = levels;
  a.p.batch = x->batch;
  a.p.h = x->h;
  a.p.w = x->w;
  a.t = threshold;
  a.t_f = (float)threshold;
  a.hard = mode == HAAR_THRESH_HARD;
  const cudaError_t e = x->dtype == HAAR_F64
                            ? shrink_launch<double>(two_d, a, (cudaStream_t)stream)
                            : shrink_launch<float>(two_d, a, (cudaStream_t)stream);
  if (e != cudaSuccess) {
    set_last_cuda_error((int)e);
    return HAAR_ECUDA;
  }
  return HAAR_OK;
}

}  // namespace

extern "C" {

int haar_denoise_1d(const haar_desc* x, const haar_desc* y, int levels, double threshold,
                    int mode, void* cuda_stream) {
  return shrink_entry(x, y, levels, threshold, mode, cuda_stream, false);
}

int haar_denoise_2d(const haar_desc* x, const haar_desc* y, int levels, double threshold,
                    int mode, void* cuda_stream) {
  return shrink_entry(x, y, levels, threshold, mode, cuda_stream, true);
}

}  // extern "C"
