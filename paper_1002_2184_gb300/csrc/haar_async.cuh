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

// Before a kernel's dependency wait: ask L2 for `bytes` from p, one 128-byte
// line per thread in turn (a hint only: the loads after the wait see every
// earlier write), so that a launch's first reads overlap the previous
// launch's drain.  NT threads share the lines.
template <int NT>
__device__ __forceinline__ void warm_l2(const void* p, int64_t bytes, int tid) {
  const char* c = static_cast<const char*>(p);
  for (int64_t o = (int64_t)tid * 128; o < bytes; o += (int64_t)NT * 128)
    asm volatile("prefetch.global.L2 [%0];" ::"l"(c + o) : "memory");
}

// Copy n elements from src to dst, both 16-byte aligned, as ceil(n / V)
// 16-byte pieces shared by NT threads (one 32-bit shared and one global
// address, both advanced per copy).
template <int NT, typename T>
__device__ __forceinline__ void stage_span(T* dst, const T* src, int n, int tid) {
  constexpr int V = fvec<T>();
  src += tid * V;
  unsigned d = (unsigned)__cvta_generic_to_shared(dst) + tid * 16u;
  const int nv = (n + V - 1) / V;
  for (int i = tid; i < nv; i += NT, src += NT * V, d += NT * 16u)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}

// Stage positions [s, s + cnt) of a sequence of period P stored at `row`
// into dst[sh + i], sh = s mod (16 / sizeof(T)).  With a 16-byte aligned row
// and P a multiple of 16 bytes, the window is a run [s mod P, P) followed by
// whole periods and a last partial run from 0 (a window longer than the
// period wraps several times), and each run is copied in aligned 16-byte
// pieces (which may also bring a few neighbours, inside [0, P)): every run
// after the first starts at dst[sh + done] with done = P - (s mod P) + a
// multiple of P, a multiple of 16 bytes.  Windows of more than 8 periods, or
// unaligned rows, copy each element on its own.  Returns sh.  NT: the number
// of threads sharing the copy (a compile-time stride).
template <int NT, typename T>
__device__ __forceinline__ int stage(T* dst, const T* row, int64_t P, int64_t s, int cnt, int tid) {
  constexpr int V = fvec<T>();
  const int sh = (int)(s & (V - 1));  // s mod V, also for negative s (two's complement)
  if ((uintptr_t)row % 16 == 0 && P % V == 0 && cnt <= 8 * P) {
    int64_t s0 = s < 0 ? s + P : s;  // windows start at most one period early
    if (s0 < 0 || s0 >= P) {         // any other start: a 64-bit remainder
      s0 = s % P;
      if (s0 < 0) s0 += P;
    }
    int done = (int)min((int64_t)cnt, P - s0);
    stage_span<NT>(dst, row + (s0 - sh), sh + done, tid);
    while (done < cnt) {
      const int len = (int)min((int64_t)(cnt - done), P);
      stage_span<NT>(dst + sh + done, row, len, tid);
      done += len;
    }
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
