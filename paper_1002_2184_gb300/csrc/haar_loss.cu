// haar_loss.cu -- kernels and C ABI beyond the transform itself:
//  * FP64 verification reductions (energy, squared difference, max error);
//  * the pieces of the differentiable denoising loss
//      c = DWT(x), s = soft(c, t), xr = IDWT(s),
//      loss = mean((xr - x)^2) + lambda * mean(|s| over detail coefficients)
//    as separate elementwise kernels (for composing with autograd), and
//  * the same loss fused into the transforms' epilogues: two launches
//    forward, two backward, each a single streaming pass.
// None of this is in the paper; the transforms are.
#include <cuda_runtime.h>

#include "fasthaar.h"
#include "haar_internal.h"
#include "haar_launch.cuh"

namespace fh {

// ---------------------------------------------------------------------------
// Warp / block reductions into FP64 accumulators.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int m = 16; m; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int m = 16; m; m >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, m));
  return v;
}
// max of non-negative doubles: their bit patterns order the same way
__device__ __forceinline__ void atomic_max_nonneg(double* p, double v) {
  atomicMax(reinterpret_cast<unsigned long long*>(p), (unsigned long long)__double_as_longlong(v));
}

// ---------------------------------------------------------------------------
// Verification reductions: out[0] += sum a^2, out[1] += sum (a-b)^2,
// out[2] = max(out[2], max |a-b|), all in FP64.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_norms(const T* __restrict__ a, const T* __restrict__ b,
                                               int64_t n, double* out) {
  pdl_wait();
  pdl_trigger();
  double saa = 0.0, sdd = 0.0, mx = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double x = (double)to_acc(a[i]);
    saa += x * x;
    if (b) {
      const double d = x - (double)to_acc(b[i]);
      sdd += d * d;
      mx = fmax(mx, fabs(d));
    }
  }
  saa = warp_sum(saa);
  sdd = warp_sum(sdd);
  mx = warp_max(mx);
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(out, saa);
    if (b) {
      atomicAdd(out + 1, sdd);
      atomic_max_nonneg(out + 2, mx);
    }
  }
}

// Position (within its h x w image) of element i of a contiguous batch is a
// detail coefficient of an L-level Mallat layout unless it lies in LL_L.
__device__ __forceinline__ bool is_detail(int64_t i, int64_t h, int64_t w, int levels) {
  const int64_t x = i % w, y = (i / w) % h;
  return !(y < (h >> levels) && x < (w >> levels));
}

template <typename T>
__device__ __forceinline__ T soft(T v, T t) {
  const T a = fabs(v) - t;
  return a > T(0) ? copysign(a, v) : T(0);
}

// s = soft(c, t); l1[0] += sum over detail positions of |s|.
template <typename T>
__global__ void __launch_bounds__(256) k_soft(const T* __restrict__ c, T* __restrict__ s,
                                              int64_t n, int64_t h, int64_t w, int levels, T t,
                                              double* l1) {
  pdl_wait();
  pdl_trigger();
  T acc = T(0);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const T v = soft(c[i], t);
    s[i] = v;
    if (is_detail(i, h, w, levels)) acc += fabs(v);
  }
  if (l1) {
    const double tot = warp_sum((double)acc);
    if ((threadIdx.x & 31) == 0) atomicAdd(l1, tot);
  }
}

// g_c = (g_s + k * g_l1 * sign(s) * detail) * [s != 0]
template <typename T>
__global__ void __launch_bounds__(256) k_soft_bwd(const T* __restrict__ gs, const T* __restrict__ s,
                                                  T* __restrict__ gc, int64_t n, int64_t h,
                                                  int64_t w, int levels, T k,
                                                  const T* __restrict__ g_l1) {
  pdl_wait();
  pdl_trigger();
  const T lam = g_l1 ? k * g_l1[0] : T(0);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const T sv = s[i];
    T g = T(0);
    if (sv != T(0)) {
      g = gs[i];
      if (is_detail(i, h, w, levels)) g += sv > T(0) ? lam : -lam;
    }
    gc[i] = g;
  }
}

// g_a = k * g * (a - b), g_b = -g_a (either output may be absent)
template <typename T>
__global__ void __launch_bounds__(256) k_sqdiff_bwd(const T* __restrict__ a,
                                                    const T* __restrict__ b, T* ga, T* gb,
                                                    int64_t n, T k, const T* __restrict__ g) {
  pdl_wait();
  pdl_trigger();
  const T sc = g ? k * g[0] : k;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const T v = sc * (a[i] - b[i]);
    if (ga) ga[i] = v;
    if (gb) gb[i] = -v;
  }
}

// ---------------------------------------------------------------------------
// Fused loss: epilogues plugged into the warp-block transforms.
// ---------------------------------------------------------------------------
// Forward analysis: store s = soft(c, t); accumulate |s| over details.
template <typename T>
struct EpiSoft {
  T t;
  T l1;
  const T* base;
  __device__ __forceinline__ T f(T v, bool d) {
    const T s = soft(v, t);
    if (d) l1 += fabs(s);
    return s;
  }
  __device__ __forceinline__ void c4(T* p, const T v[4], bool d) {
    T o[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) o[k] = f(v[k], d);
    store4(p, o);
  }
  __device__ __forceinline__ void c2(T* p, const T v[2], bool d) {
    T o[2] = {f(v[0], d), f(v[1], d)};
    store2(p, o);
  }
  __device__ __forceinline__ void c1(T* p, T v, bool d) { *p = f(v, d); }
  __device__ __forceinline__ void px8(T* p, const T v[8]) { store8(p, v); }
};

// Forward synthesis: store r = xr - x; accumulate r^2.
template <typename T>
struct EpiResid {
  const T* x;     // same layout as the output
  const T* base;  // output base the offsets are taken from
  T sq;
  __device__ __forceinline__ void px8(T* p, const T v[8]) {
    T xv[8], r[8];
    load8(x + (p - base), xv);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      r[k] = v[k] - xv[k];
      sq += r[k] * r[k];
    }
    store8(p, r);
  }
  template <typename A>
  __device__ __forceinline__ void c4(T*, const A*, bool) {}
  template <typename A>
  __device__ __forceinline__ void c2(T*, const A*, bool) {}
  template <typename A>
  __device__ __forceinline__ void c1(T*, A, bool) {}
};

// Backward analysis of r: g_c = (scale * W r + lam * sign(s) * detail) * [s != 0].
template <typename T>
struct EpiGradC {
  const T* s;
  const T* base;
  T scale, lam;
  __device__ __forceinline__ T f(T v, T sv, bool d) {
    if (sv == T(0)) return T(0);
    T g = scale * v;
    if (d) g += sv > T(0) ? lam : -lam;
    return g;
  }
  __device__ __forceinline__ void c4(T* p, const T v[4], bool d) {
    T sv[4], o[4];
    load4(s + (p - base), sv);
#pragma unroll
    for (int k = 0; k < 4; ++k) o[k] = f(v[k], sv[k], d);
    store4(p, o);
  }
  __device__ __forceinline__ void c2(T* p, const T v[2], bool d) {
    T sv[2];
    load2(s + (p - base), sv);
    T o[2] = {f(v[0], sv[0], d), f(v[1], sv[1], d)};
    store2(p, o);
  }
  __device__ __forceinline__ void c1(T* p, T v, bool d) { *p = f(v, ld_scalar(s + (p - base)), d); }
  __device__ __forceinline__ void px8(T* p, const T v[8]) { store8(p, v); }
};

// Backward synthesis: g_x = W^T g_c - scale * r.
template <typename T>
struct EpiGradX {
  const T* r;
  const T* base;
  T scale;
  __device__ __forceinline__ void px8(T* p, const T v[8]) {
    T rv[8], o[8];
    load8(r + (p - base), rv);
#pragma unroll
    for (int k = 0; k < 8; ++k) o[k] = v[k] - scale * rv[k];
    store8(p, o);
  }
  template <typename A>
  __device__ __forceinline__ void c4(T*, const A*, bool) {}
  template <typename A>
  __device__ __forceinline__ void c2(T*, const A*, bool) {}
  template <typename A>
  __device__ __forceinline__ void c1(T*, A, bool) {}
};

struct DenoiseArgs {
  Pass p;             // src, dst of this launch; ll = dst; batch, h, w, levels
  const void* aux;    // second input read at the output's positions (x, s or r)
  double* acc;        // FP64 accumulators: [0] = sum |s_detail|, [1] = sum r^2
  const void* g;      // upstream gradient of the loss (device scalar) or null
  double k1, k2;      // per-launch constants (see the launchers)
};

template <typename T>
__device__ __forceinline__ T load_g(const void* g) {
  return g ? *static_cast<const T*>(g) : T(1);
}

// Tile decode shared by the four fused kernels (same geometry as the
// strided-batch fast kernels).
struct TileXY {
  int64_t b, cy, cx, y0, x0;
};
template <int WR, int WC>
__device__ __forceinline__ TileXY tile_xy(const Pass& p, int warp) {
  TileXY t;
  const int64_t per = p.tiles_x * p.tiles_y;
  const int64_t bt = blockIdx.x;
  t.b = bt / per;
  const int64_t rr = bt - t.b * per;
  t.cy = rr / p.tiles_x;
  t.cx = rr - t.cy * p.tiles_x;
  t.y0 = t.cy * (32 * WR) + (warp / WC) * 32;
  t.x0 = t.cx * (32 * WC) + (warp % WC) * 32;
  return t;
}

template <typename T, int L, typename Epi>
__device__ __forceinline__ void fused_analysis(const Pass& p, Epi& epi) {
  constexpr int WR = (L == 6) ? 2 : 1;
  constexpr int WC = 8 / WR;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const TileXY t = tile_xy<WR, WC>(p, warp);
  const Img2 im = pass_image<T, T>(p, t.b);
  // offsets into the second array are taken from the batch base (the
  // arrays share one contiguous layout)
  epi.base = static_cast<const T*>(p.dst);
  T l5 = T(0);
  if (t.y0 < p.h && t.x0 < p.w) l5 = dwt_block32<T, T, L>(im, t.y0, t.x0, lane, epi);
  if constexpr (L == 6) {
    __shared__ T s5[WR][WC];
    if (lane == 0) s5[warp / WC][warp % WC] = l5;
    __syncthreads();
    if (threadIdx.x < WC / 2) {
      const int j = threadIdx.x;
      const int64_t by0 = t.cy * 64, bx0 = t.cx * 128 + 64 * j;
      if (by0 < p.h && bx0 < p.w)
        dwt_level6<T>(im, s5[0][2 * j], s5[0][2 * j + 1], s5[1][2 * j], s5[1][2 * j + 1], by0,
                      bx0, epi);
    }
  }
}

template <typename T, int L, typename Epi>
__device__ __forceinline__ bool fused_synthesis(const Pass& p, Epi& epi) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const TileXY t = tile_xy<1, 8>(p, warp);
  if (t.y0 >= p.h || t.x0 >= p.w) return false;
  const Img2 im = pass_image<T, T>(p, t.b);
  epi.base = static_cast<const T*>(p.dst);
  idwt_block32<T, T, L>(im, t.y0, t.x0, lane, epi);
  return true;
}

// Forward, launch 1: x -> s.  k1 = threshold.
template <typename T, int L>
__global__ void __launch_bounds__(256) k_denoise_a(const DenoiseArgs a) {
  pdl_wait();
  pdl_trigger();
  EpiSoft<T> epi{(T)a.k1, T(0), nullptr};
  fused_analysis<T, L>(a.p, epi);
  const double tot = warp_sum((double)epi.l1);
  if ((threadIdx.x & 31) == 0) atomicAdd(a.acc, tot);
}

// Forward, launch 2: s -> r = IDWT(s) - x.
template <typename T, int L>
__global__ void __launch_bounds__(256) k_denoise_b(const DenoiseArgs a) {
  pdl_wait();
  pdl_trigger();
  EpiResid<T> epi{static_cast<const T*>(a.aux), nullptr, T(0)};
  if (!fused_synthesis<T, L>(a.p, epi)) return;  // whole warp outside the image
  const double tot = warp_sum((double)epi.sq);
  if ((threadIdx.x & 31) == 0) atomicAdd(a.acc + 1, tot);
}

// loss = acc[1] * k1 + acc[0] * k2 (k1 = 1/n, k2 = lambda/n_d); clears acc.
template <typename T>
__global__ void k_denoise_finalize(double* acc, T* loss, double k1, double k2) {
  pdl_wait();
  pdl_trigger();
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    *loss = (T)(acc[1] * k1 + acc[0] * k2);
    acc[0] = 0.0;
    acc[1] = 0.0;
  }
}

// Backward, launch 1: r -> g_c.  k1 = 2/n, k2 = lambda/n_d (times g).
template <typename T, int L>
__global__ void __launch_bounds__(256) k_denoise_c(const DenoiseArgs a) {
  pdl_wait();
  pdl_trigger();
  const T g = load_g<T>(a.g);
  EpiGradC<T> epi{static_cast<const T*>(a.aux), nullptr, (T)a.k1 * g, (T)a.k2 * g};
  fused_analysis<T, L>(a.p, epi);
}

// Backward, launch 2: g_c -> g_x = IDWT(g_c) - (2g/n) r.  k1 = 2/n.
template <typename T, int L>
__global__ void __launch_bounds__(256) k_denoise_d(const DenoiseArgs a) {
  pdl_wait();
  pdl_trigger();
  const T g = load_g<T>(a.g);
  EpiGradX<T> epi{static_cast<const T*>(a.aux), nullptr, (T)a.k1 * g};
  fused_synthesis<T, L>(a.p, epi);
}

template <typename T>
cudaError_t denoise_launch(int which, DenoiseArgs a, cudaStream_t s) {
  const bool ana = (which == 0 || which == 2);
  const int CH = (ana && a.p.levels == 6) ? 64 : 32, CW = (ana && a.p.levels == 6) ? 128 : 256;
  a.p.tiles_x = (a.p.w + CW - 1) / CW;
  a.p.tiles_y = (a.p.h + CH - 1) / CH;
  a.p.ntiles = a.p.batch * a.p.tiles_x * a.p.tiles_y;
  if (a.p.ntiles == 0) return cudaSuccess;
  if (a.p.ntiles > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  const unsigned g = (unsigned)a.p.ntiles;
#define FH_DENOISE_CASE(LV)                                                  \
  case LV:                                                                   \
    switch (which) {                                                         \
      case 0: return launch_pdl(k_denoise_a<T, LV>, g, 256, s, a);          \
      case 1: return launch_pdl(k_denoise_b<T, LV>, g, 256, s, a);          \
      case 2: return launch_pdl(k_denoise_c<T, LV>, g, 256, s, a);          \
      default: return launch_pdl(k_denoise_d<T, LV>, g, 256, s, a);         \
    }
  switch (a.p.levels) {
    FH_DENOISE_CASE(1)
    FH_DENOISE_CASE(2)
    FH_DENOISE_CASE(3)
    FH_DENOISE_CASE(4)
    FH_DENOISE_CASE(5)
    FH_DENOISE_CASE(6)
    default: return cudaErrorInvalidValue;
  }
#undef FH_DENOISE_CASE
}

inline unsigned ew_grid(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace fh

using namespace fh;

namespace {

int fail(cudaError_t e) {
  if (e == cudaSuccess) return HAAR_OK;
  set_last_cuda_error((int)e);
  return HAAR_ECUDA;
}

bool float_type(int dt) { return dt == HAAR_F32 || dt == HAAR_F64; }

// A contiguous batch: batch_stride = h*w, row_stride = w.
bool contiguous(const haar_desc* d) {
  return d->row_stride == d->w && (d->batch <= 1 || d->batch_stride == d->h * d->w);
}

int check_same(const haar_desc* a, const haar_desc* b) {
  if (!a || !b) return HAAR_EINVAL;
  if (a->reserved || b->reserved) return HAAR_EINVAL;
  if (a->dtype != b->dtype) return HAAR_EDTYPE;
  if (!float_type(a->dtype)) return HAAR_EDTYPE;
  if (a->batch != b->batch || a->h != b->h || a->w != b->w) return HAAR_EINVAL;
  if (a->batch < 0 || a->h < 0 || a->w < 0) return HAAR_EINVAL;
  if (!contiguous(a) || !contiguous(b)) return HAAR_EINVAL;
  const int64_t n = a->batch * a->h * a->w;
  if (n > 0 && (!a->ptr || !b->ptr)) return HAAR_EINVAL;
  return HAAR_OK;
}

int64_t numel(const haar_desc* d) { return d->batch * d->h * d->w; }

// The fused pipeline runs on the warp-block kernels: sides multiples of 32,
// 1..6 levels, 16-byte aligned contiguous arrays.
int check_fused(const haar_desc* d, int levels) {
  if (levels < 1 || levels > 6) return HAAR_EINVAL;
  if (d->h % 32 || d->w % 32) return HAAR_ESHAPE;
  if ((d->h & ((1 << levels) - 1)) || (d->w & ((1 << levels) - 1))) return HAAR_ESHAPE;
  if ((uintptr_t)d->ptr % 16) return HAAR_EINVAL;
  return HAAR_OK;
}

// One fused launch src -> dst.  The low band of the deepest level lives in
// the coefficient array: the destination of an analysis, the source of a
// synthesis.
Pass make_pass(const haar_desc* src, const haar_desc* dst, int levels, bool synthesis) {
  Pass p{};
  p.src = src->ptr;
  p.s_bs = src->h * src->w;
  p.s_rs = src->w;
  p.dst = dst->ptr;
  p.d_bs = dst->h * dst->w;
  p.d_rs = dst->w;
  p.ll = synthesis ? src->ptr : dst->ptr;
  p.l_bs = p.d_bs;
  p.l_rs = p.d_rs;
  p.ll_acc = 0;
  p.levels = levels;
  p.batch = src->batch;
  p.h = src->h;
  p.w = src->w;
  return p;
}

cudaError_t denoise_dispatch(int dtype, int which, const DenoiseArgs& a, cudaStream_t s) {
  return dtype == HAAR_F64 ? denoise_launch<double>(which, a, s)
                           : denoise_launch<float>(which, a, s);
}

}  // namespace

extern "C" {

int haar_norms_f64(const void* a, const void* b, int dtype, int64_t n, double* out3,
                   void* cuda_stream) {
  if (n < 0 || (n > 0 && (!a || !out3))) return HAAR_EINVAL;
  if (n == 0) return HAAR_OK;
  const cudaStream_t s = (cudaStream_t)cuda_stream;
  const unsigned g = ew_grid(n);
  cudaError_t e;
  switch (dtype) {
    case HAAR_F32:
      e = launch_pdl(k_norms<float>, g, 256, s, (const float*)a, (const float*)b, n, out3);
      break;
    case HAAR_F64:
      e = launch_pdl(k_norms<double>, g, 256, s, (const double*)a, (const double*)b, n, out3);
      break;
    case HAAR_BF16:
      e = launch_pdl(k_norms<__nv_bfloat16>, g, 256, s, (const __nv_bfloat16*)a,
                     (const __nv_bfloat16*)b, n, out3);
      break;
    case HAAR_F16:
      e = launch_pdl(k_norms<__half>, g, 256, s, (const __half*)a, (const __half*)b, n, out3);
      break;
    case HAAR_U8:
      e = launch_pdl(k_norms<uint8_t>, g, 256, s, (const uint8_t*)a, (const uint8_t*)b, n, out3);
      break;
    default:
      return HAAR_EDTYPE;
  }
  return fail(e);
}

int haar_soft_threshold(const haar_desc* c, const haar_desc* s, int levels, double threshold,
                        double* l1_acc, void* cuda_stream) {
  int rc = check_same(c, s);
  if (rc) return rc;
  if (levels < 0 || levels > 62 || !(threshold >= 0.0)) return HAAR_EINVAL;
  const int64_t n = numel(c);
  if (n == 0) return HAAR_OK;
  const cudaStream_t st = (cudaStream_t)cuda_stream;
  const unsigned g = ew_grid(n);
  if (c->dtype == HAAR_F64)
    return fail(launch_pdl(k_soft<double>, g, 256, st, (const double*)c->ptr, (double*)s->ptr, n,
                           c->h, c->w, levels, threshold, l1_acc));
  return fail(launch_pdl(k_soft<float>, g, 256, st, (const float*)c->ptr, (float*)s->ptr, n, c->h,
                         c->w, levels, (float)threshold, l1_acc));
}

int haar_soft_threshold_backward(const haar_desc* g_s, const haar_desc* s, const haar_desc* g_c,
                                 int levels, double l1_scale, const void* g_l1,
                                 void* cuda_stream) {
  int rc = check_same(g_s, s);
  if (!rc) rc = check_same(s, g_c);
  if (rc) return rc;
  if (levels < 0 || levels > 62) return HAAR_EINVAL;
  const int64_t n = numel(s);
  if (n == 0) return HAAR_OK;
  const cudaStream_t st = (cudaStream_t)cuda_stream;
  const unsigned g = ew_grid(n);
  if (s->dtype == HAAR_F64)
    return fail(launch_pdl(k_soft_bwd<double>, g, 256, st, (const double*)g_s->ptr,
                           (const double*)s->ptr, (double*)g_c->ptr, n, s->h, s->w, levels,
                           l1_scale, (const double*)g_l1));
  return fail(launch_pdl(k_soft_bwd<float>, g, 256, st, (const float*)g_s->ptr,
                         (const float*)s->ptr, (float*)g_c->ptr, n, s->h, s->w, levels,
                         (float)l1_scale, (const float*)g_l1));
}

int haar_sq_diff_backward(const haar_desc* a, const haar_desc* b, const haar_desc* g_a,
                          const haar_desc* g_b, double scale, const void* g,
                          void* cuda_stream) {
  int rc = check_same(a, b);
  if (rc) return rc;
  if (g_a && (rc = check_same(a, g_a))) return rc;
  if (g_b && (rc = check_same(a, g_b))) return rc;
  const int64_t n = numel(a);
  if (n == 0 || (!g_a && !g_b)) return HAAR_OK;
  const cudaStream_t st = (cudaStream_t)cuda_stream;
  const unsigned gr = ew_grid(n);
  if (a->dtype == HAAR_F64)
    return fail(launch_pdl(k_sqdiff_bwd<double>, gr, 256, st, (const double*)a->ptr,
                           (const double*)b->ptr, g_a ? (double*)g_a->ptr : (double*)nullptr,
                           g_b ? (double*)g_b->ptr : (double*)nullptr, n, scale,
                           (const double*)g));
  return fail(launch_pdl(k_sqdiff_bwd<float>, gr, 256, st, (const float*)a->ptr,
                         (const float*)b->ptr, g_a ? (float*)g_a->ptr : (float*)nullptr,
                         g_b ? (float*)g_b->ptr : (float*)nullptr, n, (float)scale,
                         (const float*)g));
}

int haar_denoise_forward(const haar_desc* x, const haar_desc* s, const haar_desc* r, int levels,
                         double threshold, double l1_weight, double* acc2, void* loss,
                         void* cuda_stream) {
  int rc = check_same(x, s);
  if (!rc) rc = check_same(x, r);
  if (rc) return rc;
  if (!acc2 || !loss || !(threshold >= 0.0)) return HAAR_EINVAL;
  const int64_t n = numel(x);
  if (n == 0) return HAAR_OK;
  if ((rc = check_fused(x, levels)) || (rc = check_fused(s, levels)) ||
      (rc = check_fused(r, levels)))
    return rc;
  const cudaStream_t st = (cudaStream_t)cuda_stream;
  const int64_t nd = x->batch * (x->h * x->w - (x->h >> levels) * (x->w >> levels));
  DenoiseArgs a{};
  a.acc = acc2;
  a.p = make_pass(x, s, levels, false);  // x -> s
  a.k1 = threshold;
  cudaError_t e = denoise_dispatch(x->dtype, 0, a, st);
  if (e == cudaSuccess) {
    a.p = make_pass(s, r, levels, true);  // s -> r
    a.aux = x->ptr;
    e = denoise_dispatch(x->dtype, 1, a, st);
  }
  if (e == cudaSuccess) {
    const double k1 = 1.0 / (double)n, k2 = nd ? l1_weight / (double)nd : 0.0;
    if (x->dtype == HAAR_F64)
      e = launch_pdl(k_denoise_finalize<double>, 1, 32, st, acc2, (double*)loss, k1, k2);
    else
      e = launch_pdl(k_denoise_finalize<float>, 1, 32, st, acc2, (float*)loss, k1, k2);
  }
  return fail(e);
}

int haar_denoise_backward(const haar_desc* r, const haar_desc* s, const haar_desc* g_c,
                          const haar_desc* g_x, int levels, double l1_weight, const void* g_loss,
                          void* cuda_stream) {
  int rc = check_same(r, s);
  if (!rc) rc = check_same(r, g_c);
  if (!rc) rc = check_same(r, g_x);
  if (rc) return rc;
  const int64_t n = numel(r);
  if (n == 0) return HAAR_OK;
  if ((rc = check_fused(r, levels)) || (rc = check_fused(s, levels)) ||
      (rc = check_fused(g_c, levels)) || (rc = check_fused(g_x, levels)))
    return rc;
  const cudaStream_t st = (cudaStream_t)cuda_stream;
  const int64_t nd = r->batch * (r->h * r->w - (r->h >> levels) * (r->w >> levels));
  DenoiseArgs a{};
  a.g = g_loss;
  a.p = make_pass(r, g_c, levels, false);  // r -> g_c
  a.aux = s->ptr;
  a.k1 = 2.0 / (double)n;
  a.k2 = nd ? l1_weight / (double)nd : 0.0;
  cudaError_t e = denoise_dispatch(r->dtype, 2, a, st);
  if (e == cudaSuccess) {
    a.p = make_pass(g_c, g_x, levels, true);  // g_c -> g_x
    a.aux = r->ptr;
    e = denoise_dispatch(r->dtype, 3, a, st);
  }
  return fail(e);
}

}  // extern "C"
