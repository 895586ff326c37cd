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
#include "haar_roundtrip.cuh"

namespace fh {

// ---------------------------------------------------------------------------
// Warp / block reductions into FP64 accumulators.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int m = 16; m; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
  return v;
}
template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
  for (int m = 16; m; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
  return v;
}
// Sums over the block of two values per thread, added once into out[0] and
// out[1] (FP64): warp shuffles and one shared-memory slot per warp and value
// in the values' own type, one barrier, then one conversion and one FP64
// atomic per value and block (atomics from every warp to one address would
// serialise).  FP64 arithmetic is a slow pipe on this GPU, so it stays out
// of the per-thread work; an fp32 block partial is a tree sum of at most
// 8192 terms (40 roundings deep).  Every thread of the block calls it, once,
// as its last step (the slots are not reused).  (Two one-value reductions,
// each with its own barrier pair, took the forward from 18.0 to 18.7 us on
// 32 x 3 x 512^2.)
template <typename T>
__device__ __forceinline__ void block_sums_to(T v0, T v1, double* out) {
  __shared__ T part[2][32];
  v0 = warp_sum_t(v0);
  v1 = warp_sum_t(v1);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    part[0][warp] = v0;
    part[1][warp] = v1;
  }
  __syncthreads();
  if (warp == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    T t0 = lane < nw ? part[0][lane] : T(0), t1 = lane < nw ? part[1][lane] : T(0);
    t0 = warp_sum_t(t0);
    t1 = warp_sum_t(t1);
    if (lane == 0) {
      atomicAdd(out, (double)t0);
      atomicAdd(out + 1, (double)t1);
    }
  }
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
// Fused loss by recomputation.
//
// W is orthonormal (W W^T = I), so with c = W x and s = soft(c, t):
//   r = W^T s - x = W^T (s - c) = -W^T clamp(c, -t, t)
//   d loss / d x  = W^T q,   q = [|c| > t] * lam' * sign(c) * [detail]
//                              + [|c| <= t] * (2 g / n) * c,   lam' = lam g / n_d
// (g: upstream gradient; n pixels, n_d detail coefficients).  Neither s nor
// r has to be stored: the forward reads x and produces only the loss sums
// (with |r|^2 = |clamp(c, -t, t)|^2 it needs no synthesis), the backward
// reads x and writes the gradient.  Each is one kernel in which a warp takes
// its 32 x 32 block through the analysis (registers and shuffles, as
// dwt_block32) and maps every coefficient in place; the backward then runs
// the synthesis back in registers (each lane holds every coarse coefficient
// on its own path after the shuffles).
// ---------------------------------------------------------------------------
// Forward: since r = -W^T clamp(c, -t, t) and W is orthonormal, Parseval
// gives |r|^2 = |clamp(c, -t, t)|^2, so the forward needs no synthesis: it
// sums min(|c|, t)^2 over every coefficient and |soft(c)| = max(|c| - t, 0)
// over the details, each coefficient once (the owner copy).
template <typename T>
struct OpEnergy {
  T t, l1, sq;
  __device__ __forceinline__ T operator()(T c, bool detail, bool owner) {
    const T a = fabs(c) - t;
    if (owner) {
      if (detail && a > T(0)) l1 += a;
      const T m = a > T(0) ? t : fabs(c);
      sq += m * m;
    }
    return c;
  }
};

// Backward map: c -> [|c| > t] lam sign(c) [detail] + [|c| <= t] scale c.
template <typename T>
struct OpGradient {
  T t, scale, lam;
  __device__ __forceinline__ T operator()(T c, bool detail, bool) {
    if (fabs(c) > t) return detail ? copysign(lam, c) : T(0);
    return scale * c;
  }
};

struct DenoiseArgs {
  const void* x;
  void* gx;          // backward output (same layout as x)
  int64_t batch, h, w;
  int64_t tiles_x, tiles_y, ntiles;
  double* acc;       // forward sums: [0] = sum |s_detail|, [1] = sum r^2
  const void* g;     // upstream gradient (device scalar) or null (= 1)
  double t, k_scale, k_lam;  // threshold; 2/n; lam/n_d
  float t_f, k_scale_f, k_lam_f;  // the same, rounded once on the host
  int levels;        // 1..5
};


template <typename T>
__device__ __forceinline__ T load_g(const void* g) {
  return g ? *static_cast<const T*>(g) : T(1);
}

// Block of 8 warps side by side: 32 x 256 pixels of one image.
__device__ __forceinline__ bool dn_block(const DenoiseArgs& a, int64_t& off, int64_t& py,
                                         int64_t& px) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t per = a.tiles_x * a.tiles_y;
  const int64_t bt = blockIdx.x;
  const int64_t b = bt / per, rr = bt - b * per;
  const int64_t cy = rr / a.tiles_x, cx = rr - cy * a.tiles_x;
  const int64_t y0 = cy * 32, x0 = cx * 256 + warp * 32;
  py = y0 + 4 * (lane >> 2);
  px = x0 + 8 * (lane & 3);
  off = b * a.h * a.w;
  return y0 < a.h && x0 < a.w;
}

// The forward (read-only, analysis + sums) with FP32 arithmetic is capped at
// 40 registers for 6 resident blocks per SM (0.0197 against 0.0206 ms on
// 32 x 3 x 512^2); the backward spills under the same cap, so it has none.
template <typename T>
constexpr int loss_min_blocks() {
  return sizeof(T) == 8 ? 1 : 6;
}
template <typename T, int L>
__global__ void __launch_bounds__(256, loss_min_blocks<T>()) k_denoise_loss(const DenoiseArgs a) {
  pdl_wait();
  pdl_trigger();
  const int lane = threadIdx.x & 31;
  int64_t off, py, px;
  OpEnergy<T> op{param<T>(a.t, a.t_f), T(0), T(0)};
  if (dn_block(a, off, py, px)) {  // warps outside the image contribute zeros
    const T* x = static_cast<const T*>(a.x) + off;
    WarpCoefs<T, L> k;
    warp_analysis<T, L>(x + py * a.w + px, a.w, lane, k);
    warp_map<T, L>(lane, k, op);
  }
  block_sums_to(op.l1, op.sq, a.acc);  // acc[0] += sum |s_detail|, acc[1] += sum r^2
}

template <typename T, int L>
__global__ void __launch_bounds__(256) k_denoise_grad(const DenoiseArgs a) {
  pdl_wait();
  pdl_trigger();
  const int lane = threadIdx.x & 31;
  int64_t off, py, px;
  if (!dn_block(a, off, py, px)) return;
  const T g = load_g<T>(a.g);
  const T* x = static_cast<const T*>(a.x) + off;
  WarpCoefs<T, L> k;
  warp_analysis<T, L>(x + py * a.w + px, a.w, lane, k);
  OpGradient<T> op{param<T>(a.t, a.t_f), param<T>(a.k_scale, a.k_scale_f) * g,
                   param<T>(a.k_lam, a.k_lam_f) * g};
  warp_map<T, L>(lane, k, op);
  T o[4][8];
  warp_synthesis<T, L>(lane, py, px, k, o);
  T* gx = static_cast<T*>(a.gx) + off + py * a.w + px;
#pragma unroll
  for (int i = 0; i < 4; ++i) store8(gx + i * a.w, o[i]);
}

// loss = acc[1] / n + lam / n_d * acc[0]; clears acc for the next call.
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

template <typename T>
cudaError_t denoise_launch(bool grad, DenoiseArgs a, cudaStream_t s) {
  a.tiles_x = (a.w + 255) / 256;
  a.tiles_y = (a.h + 31) / 32;
  a.ntiles = a.batch * a.tiles_x * a.tiles_y;
  if (a.ntiles == 0) return cudaSuccess;
  if (a.ntiles > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  const unsigned g = (unsigned)a.ntiles;
#define FH_DN_CASE(LV)                                                                   \
  case LV:                                                                               \
    return grad ? launch_pdl(k_denoise_grad<T, LV>, g, 256, s, a)                        \
                : launch_pdl(k_denoise_loss<T, LV>, g, 256, s, a);
  switch (a.levels) {
    FH_DN_CASE(1)
    FH_DN_CASE(2)
    FH_DN_CASE(3)
    FH_DN_CASE(4)
    FH_DN_CASE(5)
    default: return cudaErrorInvalidValue;
  }
#undef FH_DN_CASE
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

// The fused loss runs on the warp-block kernels: sides multiples of 32,
// 1..5 levels (one warp per 32 x 32 block), 16-byte aligned contiguous arrays.
int check_fused(const haar_desc* d, int levels) {
  if (levels < 1 || levels > 5) return HAAR_EINVAL;
  if (d->h % 32 || d->w % 32) return HAAR_ESHAPE;
  if ((d->h & ((1 << levels) - 1)) || (d->w & ((1 << levels) - 1))) return HAAR_ESHAPE;
  if ((uintptr_t)d->ptr % 16) return HAAR_EINVAL;
  return HAAR_OK;
}

cudaError_t denoise_dispatch(int dtype, bool grad, const DenoiseArgs& a, cudaStream_t s) {
  return dtype == HAAR_F64 ? denoise_launch<double>(grad, a, s) : denoise_launch<float>(grad, a, s);
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

int haar_denoise_forward(const haar_desc* x, int levels, double threshold, double l1_weight,
                         double* acc2, void* loss, void* cuda_stream) {
  int rc = check_same(x, x);
  if (rc) return rc;
  if (!acc2 || !loss || !(threshold >= 0.0)) return HAAR_EINVAL;
  const int64_t n = numel(x);
  if (n == 0) return HAAR_OK;
  if ((rc = check_fused(x, levels))) return rc;
  const cudaStream_t st = (cudaStream_t)cuda_stream;
  const int64_t nd = x->batch * (x->h * x->w - (x->h >> levels) * (x->w >> levels));
  DenoiseArgs a{};
  a.x = x->ptr;
  a.batch = x->batch;
  a.h = x->h;
  a.w = x->w;
  a.acc = acc2;
  a.t = threshold;
  a.t_f = (float)threshold;
  a.levels = levels;
  cudaError_t e = denoise_dispatch(x->dtype, false, a, st);
  if (e == cudaSuccess) {
    const double k1 = 1.0 / (double)n, k2 = nd ? l1_weight / (double)nd : 0.0;
    if (x->dtype == HAAR_F64)
      e = launch_pdl(k_denoise_finalize<double>, 1, 32, st, acc2, (double*)loss, k1, k2);
    else
      e = launch_pdl(k_denoise_finalize<float>, 1, 32, st, acc2, (float*)loss, k1, k2);
  }
  return fail(e);
}

int haar_denoise_backward(const haar_desc* x, const haar_desc* g_x, int levels, double threshold,
                          double l1_weight, const void* g_loss, void* cuda_stream) {
  int rc = check_same(x, g_x);
  if (rc) return rc;
  if (!(threshold >= 0.0)) return HAAR_EINVAL;
  const int64_t n = numel(x);
  if (n == 0) return HAAR_OK;
  if ((rc = check_fused(x, levels)) || (rc = check_fused(g_x, levels))) return rc;
  const uintptr_t xl = (uintptr_t)x->ptr, gl = (uintptr_t)g_x->ptr;
  const uintptr_t bytes = (uintptr_t)n * (uintptr_t)(x->dtype == HAAR_F64 ? 8 : 4);
  if (xl < gl + bytes && gl < xl + bytes) return HAAR_EALIAS;
  const int64_t nd = x->batch * (x->h * x->w - (x->h >> levels) * (x->w >> levels));
  DenoiseArgs a{};
  a.x = x->ptr;
  a.gx = g_x->ptr;
  a.batch = x->batch;
  a.h = x->h;
  a.w = x->w;
  a.g = g_loss;
  a.t = threshold;
  a.k_scale = 2.0 / (double)n;
  a.k_lam = nd ? l1_weight / (double)nd : 0.0;
  a.t_f = (float)a.t;
  a.k_scale_f = (float)a.k_scale;
  a.k_lam_f = (float)a.k_lam;
  a.levels = levels;
  return fail(denoise_dispatch(x->dtype, true, a, (cudaStream_t)cuda_stream));
}

}  // extern "C"
