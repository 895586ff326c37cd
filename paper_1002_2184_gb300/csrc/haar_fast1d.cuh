// haar_fast1d.cuh -- register/warp-shuffle 1D Fast Haar kernels for signals
// whose length is a multiple of 256.
//
// Each warp owns 256 consecutive samples; each lane owns 8 of them, read or
// written as two 16-byte vectors.  Analysis: levels 1-3 run inside the lane
// (the even/odd pairs of Fig. 4, four, then two, then one); levels 4-8 pair
// lanes lane^1, ^2, ^4, ^8, ^16 through warp shuffles.  Synthesis (Eq. 19)
// needs no communication: a lane loads its own level-1..3 details and the
// (warp-shared) coarser ones, and walks down to its 8 samples.  The pair
// butterflies are fwd_pair / inv_pair, so results are bit-identical to the
// shared-memory chunk kernels.
#pragma once

#include <type_traits>

#include "haar_internal.h"
#include "haar_kernels.cuh"

namespace fh {

// One 1D signal of a pass (pointers offset to the row).
struct Sig1 {
  const void* src;
  void* dst;
  void* ll;  // a_L destination (analysis) or source (synthesis)
  int ll_acc;
  int64_t n;
};

// Both lanes of a pair (lane, lane^mask) get lo = (left + right) s and
// hi = (right - left) s, as fwd_pair computes them.
template <typename A>
__device__ __forceinline__ void hpair1(A v, bool right, int mask, A& lo, A& hi) {
  const A s = Consts<A>::s();
  const A o = __shfl_xor_sync(0xffffffffu, v, mask);
  lo = (v + o) * s;
  hi = (right ? v - o : o - v) * s;
}

// The child `c` (0 = even, 1 = odd sample) of one pair: inv_pair's outputs.
template <typename A>
__device__ __forceinline__ A inv_child1(A a, A d, int c) {
  const A s = Consts<A>::s();
  return (c ? a + d : a - d) * s;
}

template <typename T, typename A>
__device__ __forceinline__ void put_ll1(const Sig1& g, int64_t i, A v) {
  if (g.ll_acc)
    static_cast<A*>(g.ll)[i] = v;
  else
    st_scalar(static_cast<T*>(g.ll) + i, v);
}

template <typename Tin, typename A>
__device__ __forceinline__ A get_ll1(const Sig1& g, int64_t i) {
  if (g.ll_acc) return static_cast<const A*>(g.ll)[i];
  return ld_scalar(static_cast<const Tin*>(g.ll) + i);
}

// Analysis of one 256-sample block (x0 = first sample) by one warp.
template <typename Tin, typename Tout, int L>
__device__ __forceinline__ void dwt_block256(const Sig1& g, int64_t x0, int lane) {
  using A = typename AccT<Tin>::type;
  static_assert(L >= 1 && L <= 8, "one warp fuses 1..8 levels");
  const int64_t px = x0 + 8 * lane, n = g.n;
  Tout* dst = static_cast<Tout*>(g.dst);
  A v[8];
  load8(static_cast<const Tin*>(g.src) + px, v);
  A a1[4], d1[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) fwd_pair(v[2 * k], v[2 * k + 1], a1[k], d1[k]);
  store4(dst + (n >> 1) + (px >> 1), d1);
  if constexpr (L == 1) {
    if (!g.ll_acc) {
      store4(static_cast<Tout*>(g.ll) + (px >> 1), a1);
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) put_ll1<Tout>(g, (px >> 1) + k, a1[k]);
    }
    return;
  }
  A a2[2], d2[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) fwd_pair(a1[2 * k], a1[2 * k + 1], a2[k], d2[k]);
  store2(dst + (n >> 2) + (px >> 2), d2);
  if constexpr (L == 2) {
    if (!g.ll_acc) {
      store2(static_cast<Tout*>(g.ll) + (px >> 2), a2);
    } else {
      put_ll1<Tout>(g, (px >> 2), a2[0]);
      put_ll1<Tout>(g, (px >> 2) + 1, a2[1]);
    }
    return;
  }
  A a, d;
  fwd_pair(a2[0], a2[1], a, d);
  st_scalar(dst + (n >> 3) + (px >> 3), d);
#pragma unroll
  for (int l = 4; l <= L; ++l) {
    const int mask = 1 << (l - 4);
    A lo, hi;
    hpair1(a, (lane & mask) != 0, mask, lo, hi);
    a = lo;
    if ((lane & (2 * mask - 1)) == 0) st_scalar(dst + (n >> l) + (px >> l), hi);
  }
  if ((lane & ((1 << (L - 3)) - 1)) == 0) put_ll1<Tout>(g, px >> L, a);
}

// Synthesis of one 256-sample block by one warp (lanes independent).
template <typename Tin, typename Tout, int L>
__device__ __forceinline__ void idwt_block256(const Sig1& g, int64_t x0, int lane) {
  using A = typename AccT<Tin>::type;
  static_assert(L >= 1 && L <= 8, "one warp undoes 1..8 levels");
  const int64_t px = x0 + 8 * lane, n = g.n;
  const Tin* src = static_cast<const Tin*>(g.src);
  A d1[4], a1[4], d2[2], a2[2];
  A dl[9];
  A aL = A(0);
  load4(src + (n >> 1) + (px >> 1), d1);
  if constexpr (L == 1) {
    if (!g.ll_acc) {
      load4(static_cast<const Tin*>(g.ll) + (px >> 1), a1);
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) a1[k] = get_ll1<Tin, A>(g, (px >> 1) + k);
    }
  } else {
    load2(src + (n >> 2) + (px >> 2), d2);
    if constexpr (L == 2) {
      if (!g.ll_acc) {
        load2(static_cast<const Tin*>(g.ll) + (px >> 2), a2);
      } else {
        a2[0] = get_ll1<Tin, A>(g, px >> 2);
        a2[1] = get_ll1<Tin, A>(g, (px >> 2) + 1);
      }
    } else {
#pragma unroll
      for (int l = 3; l <= L; ++l) dl[l] = ld_scalar(src + (n >> l) + (px >> l));
      aL = get_ll1<Tin, A>(g, px >> L);
    }
  }
  if constexpr (L >= 3) {
    A v = aL;
#pragma unroll
    for (int l = L; l >= 4; --l) v = inv_child1(v, dl[l], (int)((px >> (l - 1)) & 1));
    inv_pair(v, dl[3], a2[0], a2[1]);
  }
  if constexpr (L >= 2) {
#pragma unroll
    for (int k = 0; k < 2; ++k) inv_pair(a2[k], d2[k], a1[2 * k], a1[2 * k + 1]);
  }
  A o[8];
#pragma unroll
  for (int k = 0; k < 4; ++k) inv_pair(a1[k], d1[k], o[2 * k], o[2 * k + 1]);
  store8(static_cast<Tout*>(g.dst) + px, o);
}

// Blocks of 8 warps = 2048 samples of one signal.
__device__ __forceinline__ bool sig_block(const Pass& p, int64_t& sig, int64_t& x0) {
  const int warp = threadIdx.x >> 5;
  const int64_t t = blockIdx.x;
  sig = t / p.tiles_x;
  x0 = (t - sig * p.tiles_x) * 2048 + warp * 256;
  return x0 < p.w;
}

template <typename Tin, typename Tout>
__device__ __forceinline__ Sig1 pass_signal(const Pass& p, int64_t sig, bool analysis) {
  using A = typename AccT<Tin>::type;
  const int64_t b = sig / p.h, y = sig - b * p.h;
  Sig1 g;
  g.src = static_cast<const Tin*>(p.src) + b * p.s_bs + y * p.s_rs;
  g.dst = static_cast<Tout*>(p.dst) + b * p.d_bs + y * p.d_rs;
  const int64_t lo = b * p.l_bs + y * p.l_rs;
  if (p.ll_acc)
    g.ll = static_cast<A*>(p.ll) + lo;
  else if (analysis)
    g.ll = static_cast<Tout*>(p.ll) + lo;
  else
    g.ll = const_cast<Tin*>(static_cast<const Tin*>(p.ll) + lo);
  g.ll_acc = p.ll_acc;
  g.n = p.w;
  return g;
}

template <typename Tin, typename Tout, int L>
__global__ void __launch_bounds__(256) k_dwt1d_fast(const Pass p) {
  pdl_wait();
  pdl_trigger();
  int64_t sig, x0;
  if (!sig_block(p, sig, x0)) return;
  dwt_block256<Tin, Tout, L>(pass_signal<Tin, Tout>(p, sig, true), x0, threadIdx.x & 31);
}

template <typename Tin, typename Tout, int L>
__global__ void __launch_bounds__(256) k_idwt1d_fast(const Pass p) {
  pdl_wait();
  pdl_trigger();
  int64_t sig, x0;
  if (!sig_block(p, sig, x0)) return;
  idwt_block256<Tin, Tout, L>(pass_signal<Tin, Tout>(p, sig, false), x0, threadIdx.x & 31);
}

template <typename Tin, typename Tout>
cudaError_t dwt1d_fast_t(Pass p, bool fwd, cudaStream_t s) {
  p.tiles_x = (p.w + 2047) / 2048;
  p.tiles_y = 1;
  p.ntiles = p.batch * p.h * p.tiles_x;
  if (p.ntiles == 0) return cudaSuccess;
  if (p.ntiles > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  const unsigned g = (unsigned)p.ntiles;
#define FH_F1_CASE(LV)                                                     \
  case LV:                                                                 \
    if (fwd) return launch_pdl(k_dwt1d_fast<Tin, Tout, LV>, g, 256, s, p); \
    if constexpr (std::is_same<Tin, uint8_t>::value)                       \
      return cudaErrorInvalidValue; /* coefficients are never uint8 */     \
    else                                                                   \
      return launch_pdl(k_idwt1d_fast<Tin, Tout, LV>, g, 256, s, p);
  switch (p.levels) {
    FH_F1_CASE(1)
    FH_F1_CASE(2)
    FH_F1_CASE(3)
    FH_F1_CASE(4)
    FH_F1_CASE(5)
    FH_F1_CASE(6)
    FH_F1_CASE(7)
    FH_F1_CASE(8)
    default: return cudaErrorInvalidValue;
  }
#undef FH_F1_CASE
}

}  // namespace fh
