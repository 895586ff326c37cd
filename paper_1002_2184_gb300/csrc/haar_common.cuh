// haar_common.cuh -- storage types, vector load/store policies and the
// 2x2 / pair butterflies shared by every Fast Haar kernel.
//
// Arithmetic is always FP32 (FP64 for the double instantiation used by
// gradient checks); storage may be fp32, bf16, fp16 or uint8 (input only).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace fh {

// ---------------------------------------------------------------------------
// Programmatic dependent launch.  Every kernel is launched with programmatic
// stream serialisation allowed, so the next kernel in the stream can be
// scheduled while this one drains.  pdl_wait() blocks until all prerequisite
// grids have completed and their memory is visible; every kernel calls it
// before its first global memory access, so ordering is exactly that of
// plain stream order.  pdl_trigger() lets the next grid begin launching.
// Both are no-ops for a grid launched without the attribute.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Launch `kernel<<<grid, block, 0, stream>>>(args...)` with programmatic
// stream serialisation allowed (see pdl_wait).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), unsigned grid, unsigned block,
                              cudaStream_t stream, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<Args&&>(args)...);
}

// A kernel parameter in the arithmetic type.  Parameters travel as double
// plus a copy rounded to float once on the host, so that fp32 kernels never
// convert from double per thread (FP64 is a slow pipe on this GPU).
template <typename T>
__device__ __forceinline__ T param(double d, float f);
template <>
__device__ __forceinline__ float param<float>(double, float f) { return f; }
template <>
__device__ __forceinline__ double param<double>(double d, float) { return d; }

// ---------------------------------------------------------------------------
// Accumulator type per storage type.
// ---------------------------------------------------------------------------
template <typename T> struct AccT { using type = float; };
template <> struct AccT<double> { using type = double; };

__device__ __forceinline__ float to_acc(float v) { return v; }
__device__ __forceinline__ double to_acc(double v) { return v; }
__device__ __forceinline__ float to_acc(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_acc(__half v) { return __half2float(v); }
__device__ __forceinline__ float to_acc(uint8_t v) { return (float)v; }

template <typename T> __device__ __forceinline__ T from_acc(float v);
template <> __device__ __forceinline__ float from_acc<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_acc<__nv_bfloat16>(float v) {
  return __float2bfloat16_rn(v);
}
template <> __device__ __forceinline__ __half from_acc<__half>(float v) {
  return __float2half_rn(v);
}
template <typename T> __device__ __forceinline__ T from_acc(double v);
template <> __device__ __forceinline__ double from_acc<double>(double v) { return v; }

// ---------------------------------------------------------------------------
// Read-only streaming loads (inputs never alias outputs: the C-ABI checks).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float ld_scalar(const float* p) { return __ldg(p); }
__device__ __forceinline__ double ld_scalar(const double* p) { return __ldg(p); }
__device__ __forceinline__ float ld_scalar(const __nv_bfloat16* p) {
  return __bfloat162float(__ldg(p));
}
__device__ __forceinline__ float ld_scalar(const __half* p) { return __half2float(__ldg(p)); }
__device__ __forceinline__ float ld_scalar(const uint8_t* p) { return (float)__ldg(p); }

template <typename T, typename A>
__device__ __forceinline__ void st_scalar(T* p, A v) { *p = from_acc<T>(v); }

// 8 consecutive elements -> accumulators.  Alignment: 16 B for fp32, bf16,
// fp16 and fp64 rows, 8 B for uint8 rows (the host checks it).
__device__ __forceinline__ void load8(const float* p, float v[8]) {
  float4 a = __ldg(reinterpret_cast<const float4*>(p));
  float4 b = __ldg(reinterpret_cast<const float4*>(p) + 1);
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}
__device__ __forceinline__ void load8(const double* p, double v[8]) {
  const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    double2 a = __ldg(q + k);
    v[2 * k] = a.x;
    v[2 * k + 1] = a.y;
  }
}
__device__ __forceinline__ void load8(const __nv_bfloat16* p, float v[8]) {
  uint4 u = __ldg(reinterpret_cast<const uint4*>(p));
  const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    __nv_bfloat162 h2 = *reinterpret_cast<const __nv_bfloat162*>(&w[k]);
    float2 f = __bfloat1622float2(h2);
    v[2 * k] = f.x;
    v[2 * k + 1] = f.y;
  }
}
__device__ __forceinline__ void load8(const __half* p, float v[8]) {
  uint4 u = __ldg(reinterpret_cast<const uint4*>(p));
  const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    __half2 h2 = *reinterpret_cast<const __half2*>(&w[k]);
    float2 f = __half22float2(h2);
    v[2 * k] = f.x;
    v[2 * k + 1] = f.y;
  }
}
// Byte k of w as a float, exactly: one byte permute builds the bit pattern
// of 2^23 + byte (the byte lands in the low mantissa bits under the exponent
// of 2^23), one subtraction removes 2^23.
__device__ __forceinline__ float u8_to_f32(uint32_t w, int k) {
  return __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7540u + (unsigned)k)) - 8388608.0f;
}
__device__ __forceinline__ void load8(const uint8_t* p, float v[8]) {
  uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    v[k] = u8_to_f32(u.x, k);
    v[4 + k] = u8_to_f32(u.y, k);
  }
}

// 4 consecutive elements -> accumulators (coefficient bands; no uint8).
__device__ __forceinline__ void load4(const float* p, float v[4]) {
  float4 a = __ldg(reinterpret_cast<const float4*>(p));
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
}
__device__ __forceinline__ void load4(const double* p, double v[4]) {
  const double2* q = reinterpret_cast<const double2*>(p);
  double2 a = __ldg(q), b = __ldg(q + 1);
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void load4(const __nv_bfloat16* p, float v[4]) {
  uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
  float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.x));
  float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.y));
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void load4(const __half* p, float v[4]) {
  uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
  float2 a = __half22float2(*reinterpret_cast<const __half2*>(&u.x));
  float2 b = __half22float2(*reinterpret_cast<const __half2*>(&u.y));
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

// 2 consecutive coefficients -> accumulators (8 B fp32, 4 B bf16/fp16, 16 B fp64).
__device__ __forceinline__ void load2(const float* p, float v[2]) {
  float2 a = __ldg(reinterpret_cast<const float2*>(p));
  v[0] = a.x; v[1] = a.y;
}
__device__ __forceinline__ void load2(const double* p, double v[2]) {
  double2 a = __ldg(reinterpret_cast<const double2*>(p));
  v[0] = a.x; v[1] = a.y;
}
__device__ __forceinline__ void load2(const __nv_bfloat16* p, float v[2]) {
  float2 a = __bfloat1622float2(__ldg(reinterpret_cast<const __nv_bfloat162*>(p)));
  v[0] = a.x; v[1] = a.y;
}
__device__ __forceinline__ void load2(const __half* p, float v[2]) {
  float2 a = __half22float2(__ldg(reinterpret_cast<const __half2*>(p)));
  v[0] = a.x; v[1] = a.y;
}

// accumulators -> 4 consecutive elements (16 B fp32, 8 B bf16/fp16, 32 B fp64).
__device__ __forceinline__ void store4(float* p, const float v[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void store4(double* p, const double v[4]) {
  double2* q = reinterpret_cast<double2*>(p);
  q[0] = make_double2(v[0], v[1]);
  q[1] = make_double2(v[2], v[3]);
}
__device__ __forceinline__ uint32_t pack2(__nv_bfloat16*, float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}
__device__ __forceinline__ uint32_t pack2(__half*, float a, float b) {
  __half2 h = __floats2half2_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}
__device__ __forceinline__ void store4(__nv_bfloat16* p, const float v[4]) {
  *reinterpret_cast<uint2*>(p) = make_uint2(pack2(p, v[0], v[1]), pack2(p, v[2], v[3]));
}
__device__ __forceinline__ void store4(__half* p, const float v[4]) {
  *reinterpret_cast<uint2*>(p) = make_uint2(pack2(p, v[0], v[1]), pack2(p, v[2], v[3]));
}

// accumulators -> 2 consecutive elements.
__device__ __forceinline__ void store2(float* p, const float v[2]) {
  *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
}
__device__ __forceinline__ void store2(double* p, const double v[2]) {
  *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
}
__device__ __forceinline__ void store2(__nv_bfloat16* p, const float v[2]) {
  *reinterpret_cast<uint32_t*>(p) = pack2(p, v[0], v[1]);
}
__device__ __forceinline__ void store2(__half* p, const float v[2]) {
  *reinterpret_cast<uint32_t*>(p) = pack2(p, v[0], v[1]);
}

// accumulators -> 8 consecutive elements.
// Eight fp32 values: when the address allows it, one 32-byte store (a whole
// sector, Blackwell's 256-bit st), so no sector is written in two halves by
// two instructions; else two 16-byte stores.
__device__ __forceinline__ void store8(float* p, const float v[8]) {
  if (((uintptr_t)p & 31) == 0) {
    asm volatile("st.global.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "f"(v[0]),
                 "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7])
                 : "memory");
    return;
  }
  store4(p, v);
  store4(p + 4, v + 4);
}
__device__ __forceinline__ void store8(double* p, const double v[8]) {
  if (((uintptr_t)p & 31) == 0) {  // two whole sectors
    asm volatile("st.global.v4.f64 [%0], {%1,%2,%3,%4};" ::"l"(p), "d"(v[0]), "d"(v[1]),
                 "d"(v[2]), "d"(v[3])
                 : "memory");
    asm volatile("st.global.v4.f64 [%0], {%1,%2,%3,%4};" ::"l"(p + 4), "d"(v[4]), "d"(v[5]),
                 "d"(v[6]), "d"(v[7])
                 : "memory");
    return;
  }
  store4(p, v);
  store4(p + 4, v + 4);
}
__device__ __forceinline__ void store8(__nv_bfloat16* p, const float v[8]) {
  *reinterpret_cast<uint4*>(p) = make_uint4(pack2(p, v[0], v[1]), pack2(p, v[2], v[3]),
                                            pack2(p, v[4], v[5]), pack2(p, v[6], v[7]));
}
__device__ __forceinline__ void store8(__half* p, const float v[8]) {
  *reinterpret_cast<uint4*>(p) = make_uint4(pack2(p, v[0], v[1]), pack2(p, v[2], v[3]),
                                            pack2(p, v[4], v[5]), pack2(p, v[6], v[7]));
}

// ---------------------------------------------------------------------------
// Butterflies.
//
// 1D (Fig. 4 and Eq. 19): the down-sampler sits at the input, so one even/odd
// pair gives both bands directly:
//   d0 = (x0 + x1) s,  d1 = (x1 - x0) s;   x0 = (d0 - d1) s,  x1 = (d0 + d1) s
// with s = RN_fp32(1/sqrt(2)) (RN_fp64 for the double instantiation).
//
// 2D: the row pass followed by the column pass on one 2x2 block [[a, b],
// [c, d]] collapses to four sums with an exact factor 1/2 (s * s = 1/2):
//   LL = (a+b+c+d)/2, Hx = (b-a+d-c)/2, Hy = (c+d-a-b)/2, HH = (a-b-c+d)/2.
// ---------------------------------------------------------------------------
template <typename A> struct Consts;
template <> struct Consts<float> {
  static __device__ __forceinline__ float s() { return 0.70710678118654752440f; }
};
template <> struct Consts<double> {
  static __device__ __forceinline__ double s() { return 0.70710678118654752440; }
};

template <typename A>
__device__ __forceinline__ void fwd_pair(A x0, A x1, A& d0, A& d1) {
  const A s = Consts<A>::s();
  d0 = (x0 + x1) * s;
  d1 = (x1 - x0) * s;
}
template <typename A>
__device__ __forceinline__ void inv_pair(A d0, A d1, A& x0, A& x1) {
  const A s = Consts<A>::s();
  x0 = (d0 - d1) * s;
  x1 = (d0 + d1) * s;
}

template <typename A>
__device__ __forceinline__ void fwd_quad(A a, A b, A c, A d, A& ll, A& hx, A& hy, A& hh) {
  const A h = A(0.5);
  A p = a + b, q = c + d, r = b - a, t = d - c;
  ll = (p + q) * h;
  hy = (q - p) * h;
  hx = (r + t) * h;
  hh = (t - r) * h;
}
template <typename A>
__device__ __forceinline__ void inv_quad(A ll, A hx, A hy, A hh, A& a, A& b, A& c, A& d) {
  const A h = A(0.5);
  A s1 = ll - hy, s2 = hx - hh, t1 = ll + hy, t2 = hx + hh;
  a = (s1 - s2) * h;
  b = (s1 + s2) * h;
  c = (t1 - t2) * h;
  d = (t1 + t2) * h;
}

}  // namespace fh
