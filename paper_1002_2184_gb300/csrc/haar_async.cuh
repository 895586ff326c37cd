// haar_async.cuh -- asynchronous global -> shared staging with cp.async
// (16-byte copies issued by every thread, one wait at the end) for the
// kernels that work on a staged window of a row: the K-tap bank and the
// undecimated transform.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace fh {

// elements per 16-byte copy
template <typename T>
__host__ __device__ constexpr int fvec() { return 16 / (int)sizeof(T); }

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
template <int B>
__device__ __forceinline__ void cp_async_small(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(d), "l"(src), "n"(B)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// Stage positions [s, s + cnt) of a sequence of period P stored at `row`
// into dst[sh + i], sh = s mod (16 / sizeof(T)).  Inside the sequence and
// with a 16-byte aligned row the copy is made of aligned 16-byte pieces
// (which may also bring a few neighbours, inside [0, P)); otherwise, e.g. for
// windows that wrap around, each element is copied on its own.  Returns sh.
// NT: the number of threads sharing the copy (a compile-time stride).
template <int NT, typename T>
__device__ __forceinline__ int stage(T* dst, const T* row, int64_t P, int64_t s, int cnt, int tid) {
  constexpr int V = fvec<T>();
  const int sh = (int)(s & (V - 1));  // s mod V, also for negative s (two's complement)
  const bool vec = ((uintptr_t)row % 16 == 0) && (P % V == 0) && s >= 0 && s + cnt <= P;
  if (vec) {
    // one 32-bit shared and one global address, both advanced per copy
    const T* src = row + (s - sh) + tid * V;
    unsigned d = (unsigned)__cvta_generic_to_shared(dst) + tid * 16u;
    const int nv = (sh + cnt + V - 1) / V;
    for (int i = tid; i < nv; i += NT, src += NT * V, d += NT * 16u)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
  } else {
    for (int i = tid; i < cnt; i += NT) {
      int64_t gpos = (s + i) % P;
      if (gpos < 0) gpos += P;
      cp_async_small<(int)sizeof(T)>(dst + sh + i, row + gpos);
    }
  }
  return sh;
}

}  // namespace fh
