// haar_filter.cu -- the down-sample-first (polyphase) two-channel bank for
// any even-length orthogonal low-pass filter h[0..K-1], K in {2, 4, 6, 8}
// (Haar, Daubechies-4/6/8, ...), 1D, periodic boundary, multi-level Mallat
// layout [a_L | d_L | ... | d_1].
//
// The paper derives the polyphase split for the two-tap Haar filter and
// states the decomposition for a general filter (Section III, Eq. 7).  With
// the down-sampler moved in front, each output is formed from the K input
// samples it actually depends on and the decimated outputs are never
// computed:
//   a[n] = sum_k h[k] x[(2n + k) mod N],   d[n] = sum_k g[k] x[(2n + k) mod N],
//   g[k] = (-1)^(k+1) h[K-1-k]   (for K = 2 the detail sign of Eq. 9),
//   x[2n + p] = sum_i h[p + 2i] a[n - i] + g[p + 2i] d[n - i],  i < K/2.
//
// Work is cut into chunks of 4096 level-0 positions (4096 / 2^l coefficients
// at level l; 8192 with K >= 6).  Analysis: the chunk plus
// a right halo of (K - 2)(2^L - 1) samples (wrapped) is staged in shared
// memory with asynchronous 16-byte copies and every level is fused there,
// two levels per pass: a thread takes 8 consecutive inputs of level l, makes
// 4 outputs of level l + 1 in registers (and the K - 2 low-pass ones after
// them: made again for K <= 4, taken from the next lanes for K >= 6) and
// from those 2 outputs of level l + 2, so level l + 1 never touches shared
// memory.  Synthesis: a_L and the window of every d_l the
// chunk needs (K/2 - 1 extra coefficients per level on the left) are staged
// in one go and the levels run coarsest first, also two per pass; the last
// pass (levels 2 and 1) writes the output.
#include <cuda_runtime.h>

#include "fasthaar.h"
#include "haar_internal.h"
#include "haar_async.cuh"
#include "haar_kernels.cuh"

namespace fh {

constexpr int kFMaxLevels = 10;
constexpr int kFMaxTaps = 8;

// Analysis chunk and block.  A chunk recomputes a right halo of
// (K - 2)(2^L - 1) samples for its coarser levels, so the longer filters
// take chunks twice as long (the same 32 samples per thread).
template <int K>
__host__ __device__ constexpr int fchunk_a() { return K >= 6 ? 8192 : 4096; }
template <int K>
__host__ __device__ constexpr int fthreads_a() { return K >= 6 ? 256 : 128; }
// Synthesis chunk (level-0 positions per block) and block.  The passes
// over the coarse levels, the windows' left extensions and the per-block
// set-up are the same for every chunk, so the longer filters, whose passes
// cost the most, take chunks twice as long (the same 32 outputs per thread).
template <int K>
__host__ __device__ constexpr int fchunk_s() { return K >= 6 ? 8192 : 4096; }
template <int K>
__host__ __device__ constexpr int fthreads_s() { return K >= 6 ? 256 : 128; }

struct FilterArgs {
  const void* in;
  void* out;
  int64_t rows, n;
  int levels;
  int64_t chunks;
  double h[kFMaxTaps], g[kFMaxTaps];
  float hf[kFMaxTaps], gf[kFMaxTaps];  // the same, rounded once on the host
  int woff[kFMaxLevels + 2];           // synthesis: offset of staged window w (a_L, d_L, ..., d_1)
  int e[kFMaxLevels + 1];              // synthesis: e_l of the window starts (host-computed)
};

template <typename T> struct FVec2;
template <> struct FVec2<float> { using type = float2; };
template <> struct FVec2<double> { using type = double2; };
template <typename T> struct FVec16;
template <> struct FVec16<float> { using type = float4; };
template <> struct FVec16<double> { using type = double2; };


__host__ __device__ constexpr int fround(int v, int m) { return (v + m - 1) / m * m; }


// ---- shared-memory footprints (host and device agree on these) ----
// analysis: staged window (chunk + right halo) and one quarter-size buffer
// for a_2, a_6, ... (a_4, a_8, ... go back to the first); both with 16
// elements of slack for the reads past the end
template <typename T, int K>
__host__ __device__ constexpr int fdwt_cap_a(int L) {
  return fround(fchunk_a<K>() + (K - 2) * ((1 << L) - 1) + 16, fvec<T>());
}
template <typename T, int K>
__host__ __device__ constexpr int fdwt_cap_b(int L) {
  return fround(fchunk_a<K>() / 4 + (K - 2) * ((1 << L) - 1) / 4 + 16, fvec<T>());
}
// synthesis: the window of level l (a_l or d_l) spans (chunk >> l) + at most
// 2 (K/2 - 1) + 1 positions; every window is staged with a 16-byte slack and
// room for the 8-wide reads of level 1 past its end
template <typename T, int K>
__host__ __device__ constexpr int fidwt_seg_cap(int l) {
  return fround((fchunk_s<K>() >> l) + 2 * (K / 2 - 1) + 2 + 2 * fvec<T>() + 8, fvec<T>());
}
template <typename T, int K>
__host__ __device__ constexpr int fidwt_stage_cap(int L) {
  int t = fidwt_seg_cap<T, K>(L);  // a_L
  for (int l = 1; l <= L; ++l) t += fidwt_seg_cap<T, K>(l);
  return t;
}
// synthesis intermediates: a_2, a_6, a_10 in the big buffer, a_4, a_8 in the
// small one (a pass reads one and writes the other); each holds its window,
// the 8 values a unit writes past it and the reads past it
template <typename T, int K>
__host__ __device__ constexpr int fidwt_big_cap() {
  return fround((fchunk_s<K>() >> 2) + 4 * (K / 2 - 1) + 16 + 2 * fvec<T>(), fvec<T>());
}
template <typename T, int K>
__host__ __device__ constexpr int fidwt_small_cap() {
  return fround((fchunk_s<K>() >> 4) + 4 * (K / 2 - 1) + 16 + 2 * fvec<T>(), fvec<T>());
}
// e_l of the synthesis window start lo(l) = (m0 >> l) - e_l: e_0 = 0,
// e_l = ceil(e_{l-1} / 2) + K/2 - 1 (the same for every chunk)
template <int K>
__host__ __device__ constexpr int fe(int l) {
  int e = 0;
  for (int i = 0; i < l; ++i) e = (e + 1) / 2 + K / 2 - 1;
  return e;
}

// ---- analysis ----
// One level: from the input A of this level (chunk + right halo r) the
// low-pass outputs go to lo_dst, the details of the chunk to dl.
template <typename T, int K, int NT>
__device__ __forceinline__ void dwt_level(const T* A, T* lo_dst, T* dl, int half, int m,
                                          const T* h, const T* g, int tid) {
  using V2 = typename FVec2<T>::type;
  const V2* A2 = reinterpret_cast<const V2*>(A);
  if constexpr (K <= 4) {
    // two neighbouring outputs j, j + 1 per thread share K/2 + 1 pair loads
    for (int p = tid; 2 * p < m; p += NT) {
      T v[K + 2];
#pragma unroll
      for (int t = 0; t <= K / 2; ++t) {
        const V2 w = A2[2 * p + t];
        v[2 * t] = w.x;
        v[2 * t + 1] = w.y;
      }
      T lo0 = T(0), hi0 = T(0), lo1 = T(0), hi1 = T(0);
#pragma unroll
      for (int k = 0; k < K; ++k) {
        lo0 = fma(h[k], v[k], lo0);
        hi0 = fma(g[k], v[k], hi0);
        lo1 = fma(h[k], v[k + 2], lo1);
        hi1 = fma(g[k], v[k + 2], hi1);
      }
      const int j = 2 * p;
      lo_dst[j] = lo0;
      if (j + 1 < m) lo_dst[j + 1] = lo1;
      if (j < half) dl[j] = hi0;
      if (j + 1 < half) dl[j + 1] = hi1;
    }
  } else {
    // longer filters: one output per thread, neighbouring threads read
    // neighbouring pairs (no bank conflicts)
    for (int j = tid; j < m; j += NT) {
      T lo = T(0), hi = T(0);
#pragma unroll
      for (int t = 0; t < K / 2; ++t) {
        const V2 w = A2[j + t];
        lo = fma(h[2 * t], w.x, lo);
        lo = fma(h[2 * t + 1], w.y, lo);
        hi = fma(g[2 * t], w.x, hi);
        hi = fma(g[2 * t + 1], w.y, hi);
      }
      lo_dst[j] = lo;
      if (j < half) dl[j] = hi;
    }
  }
}

// Two levels in one pass, a thread per unit (the form for K <= 4).  X holds
// this level's input: len samples of the chunk and a right halo r; m2 =
// len/4 + r2 outputs of level l + 2 are made (r2 = (r - 3(K - 2)) / 4, the
// halo the levels after it need).  Unit u reads X[8u, 8u + 3K + 2):
// a_{l+1}[4u + j] for j < K + 2 (the last K - 2 belong to the next unit as
// well and are made twice), d_{l+1}[4u + j] for j < 4, then a_{l+2} and
// d_{l+2} at 2u and 2u + 1.  Outputs past the ends (m2, len/2, len/4) are
// computed from the buffer's slack and not stored: the last unit reads up
// to X[len + r + 5] (fp32) or X[len + r + 3] (fp64), inside the 16 elements
// of slack every staging buffer has.
template <typename T, int K, bool DETAILS = true>
__device__ __forceinline__ void pair_unit(const T* X, int u, const T* h, const T* g, T (&e1)[4],
                                          T (&a2)[2], T (&e2)[2]) {
  using VT = typename FVec16<T>::type;
  constexpr int V = fvec<T>();
  constexpr int NW = (3 * K + 2 + V - 1) / V;  // 16-byte loads per unit
  T x[NW * V];
#pragma unroll
  for (int i = 0; i < NW; ++i)
    *reinterpret_cast<VT*>(x + i * V) = reinterpret_cast<const VT*>(X + 8 * u)[i];
  T a1[K + 2];
#pragma unroll
  for (int j = 0; j < K + 2; ++j) {
    T s = T(0);
#pragma unroll
    for (int k = 0; k < K; ++k) s = fma(h[k], x[2 * j + k], s);
    a1[j] = s;
  }
  if constexpr (DETAILS) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      T s = T(0);
#pragma unroll
      for (int k = 0; k < K; ++k) s = fma(g[k], x[2 * j + k], s);
      e1[j] = s;
    }
  }
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    T s = T(0), d = T(0);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      s = fma(h[k], a1[2 * j + k], s);
      if constexpr (DETAILS) d = fma(g[k], a1[2 * j + k], d);
    }
    a2[j] = s;
    e2[j] = d;
  }
}

// Units u < len/8 have all their outputs inside: with VEC (every output
// vector aligned) they store without a guard.  The rest -- the halo units,
// whose only stored outputs are a_{l+2}, and the last unit of a ragged
// chunk -- store one by one under guards.
template <typename T, int K, int NT, bool VEC>
__device__ __forceinline__ void dwt_pair_rc(const T* X, T* lo, T* d1, T* d2, int len, int m2,
                                            const T* h, const T* g, int tid) {
  using V2 = typename FVec2<T>::type;
  const int nfull = VEC ? len >> 3 : 0;
  for (int u = tid; u < nfull; u += NT) {
    T e1[4], a2[2], e2[2];
    pair_unit<T, K>(X, u, h, g, e1, a2, e2);
    if constexpr (sizeof(T) == 4) {
      *reinterpret_cast<float4*>(d1 + 4 * u) = make_float4(e1[0], e1[1], e1[2], e1[3]);
    } else {
      *reinterpret_cast<V2*>(d1 + 4 * u) = V2{e1[0], e1[1]};
      *reinterpret_cast<V2*>(d1 + 4 * u + 2) = V2{e1[2], e1[3]};
    }
    *reinterpret_cast<V2*>(d2 + 2 * u) = V2{e2[0], e2[1]};
    *reinterpret_cast<V2*>(lo + 2 * u) = V2{a2[0], a2[1]};
  }
  const int n1 = len >> 1, n2 = len >> 2;
  for (int u = nfull + tid; 2 * u < m2; u += NT) {
    T e1[4], a2[2], e2[2];
    if (4 * u < n1) {  // a ragged chunk's last unit, or any unit without VEC
      pair_unit<T, K>(X, u, h, g, e1, a2, e2);
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (4 * u + i < n1) d1[4 * u + i] = e1[i];
#pragma unroll
      for (int i = 0; i < 2; ++i)
        if (2 * u + i < n2) d2[2 * u + i] = e2[i];
    } else {  // a halo unit: only its low-pass outputs are kept
      pair_unit<T, K, false>(X, u, h, g, e1, a2, e2);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
      if (2 * u + i < m2) lo[2 * u + i] = a2[i];
  }
}

// The arithmetic of one unit on every lane of the warp: 4 outputs of level
// l + 1 from the lane's inputs xs[0, K + 6), the K - 2 after them from the
// next lanes, then 2 of level l + 2.  Without DETAILS only the low-pass
// outputs are made.
template <typename T, int K, bool DETAILS>
__device__ __forceinline__ void sh_unit(const T* xs, const T* h, const T* g, T (&e1)[4],
                                        T (&a2)[2], T (&e2)[2]) {
  using VT = typename FVec16<T>::type;
  constexpr int V = fvec<T>();
  constexpr int NW = (K + 6 + V - 1) / V;  // 16-byte loads per unit
  T x[NW * V];
#pragma unroll
  for (int i = 0; i < NW; ++i) *reinterpret_cast<VT*>(x + i * V) = reinterpret_cast<const VT*>(xs)[i];
  T a1[K + 2];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    T s = T(0);
#pragma unroll
    for (int k = 0; k < K; ++k) s = fma(h[k], x[2 * j + k], s);
    a1[j] = s;
  }
  if constexpr (DETAILS) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      T s = T(0);
#pragma unroll
      for (int k = 0; k < K; ++k) s = fma(g[k], x[2 * j + k], s);
      e1[j] = s;
    }
  }
#pragma unroll
  for (int j = 0; j < K - 2; ++j) a1[4 + j] = __shfl_down_sync(0xffffffffu, a1[j % 4], 1 + j / 4);
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    T s = T(0);
#pragma unroll
    for (int k = 0; k < K; ++k) s = fma(h[k], a1[2 * j + k], s);
    a2[j] = s;
  }
  if constexpr (DETAILS) {
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      T d = T(0);
#pragma unroll
      for (int k = 0; k < K; ++k) d = fma(g[k], a1[2 * j + k], d);
      e2[j] = d;
    }
  }
}

template <typename T>
__device__ __forceinline__ void put_unit(T* d1, T* d2, T* lo, const T (&e1)[4], const T (&a2)[2],
                                         const T (&e2)[2]) {
  using V2 = typename FVec2<T>::type;
  if constexpr (sizeof(T) == 4) {
    *reinterpret_cast<float4*>(d1) = make_float4(e1[0], e1[1], e1[2], e1[3]);
  } else {
    *reinterpret_cast<V2*>(d1) = V2{e1[0], e1[1]};
    *reinterpret_cast<V2*>(d1 + 2) = V2{e1[2], e1[3]};
  }
  *reinterpret_cast<V2*>(d2) = V2{e2[0], e2[1]};
  *reinterpret_cast<V2*>(lo) = V2{a2[0], a2[1]};
}

// Two levels in one pass, a warp at a time (the form for K >= 6, where the
// values made twice above are most of the work).  X holds this level's
// input: len samples of the chunk and a right halo r; m2 = len/4 + r2
// outputs of level l + 2 are made (r2 = (r - 3(K - 2)) / 4, the halo the
// levels after it need) by U = ceil(m2 / 2) units.  Unit u makes
// a_{l+1}[4u + j] and d_{l+1}[4u + j] (j < 4) from X[8u, 8u + K + 6), then
// a_{l+2} and d_{l+2} at 2u, 2u + 1, which also read a_{l+1}[4u + 4,
// 4u + K + 2): the first values of units u + 1 and u + 2, taken from the
// next lanes with shuffles.  A warp pass covers W = 32 - R units; its last
// R = ceil((K - 2) / 4) lanes only make values for their neighbours.
// Outputs past the ends (m2, len/2, len/4) come from the buffer's slack and
// are not stored; lanes past the last unit read as the R-th lane after it,
// so reads end at X[len + r + 9], inside the 16 elements of slack every
// staging buffer has.
//
// With VEC (every output vector aligned) the passes whose units all lie
// inside the chunk (base + W <= len/8) run first in a loop of their own:
// no clamp (lanes W.. read unit len/8 + R - 1 at most, and U >= len/8), the
// details kept, whole-vector stores without guards, and addresses that
// advance by a fixed stride.  The remaining passes (halo units, whose only
// stored outputs are a_{l+2}, and a ragged end) check each store.
template <typename T, int K, int NT, bool VEC>
__device__ __forceinline__ void dwt_pair_sh(const T* X, T* lo, T* d1, T* d2, int len, int m2,
                                            const T* h, const T* g, int tid) {
  constexpr int R = (K - 2 + 3) / 4;
  constexpr int W = 32 - R;
  constexpr int S = (NT / 32) * W;  // units one pass of the block covers
  const int lane = tid & 31;
  const int U = (m2 + 1) / 2, n1 = len >> 1, n2 = len >> 2;
  int base = (tid >> 5) * W;
  if constexpr (VEC) {
    const int nfull = len >> 3;
    const T* xs = X + 8 * (base + lane);
    T* d1p = d1 + 4 * (base + lane);
    T* d2p = d2 + 2 * (base + lane);
    T* lop = lo + 2 * (base + lane);
    // unrolled twice: 8-tap analysis 74.0 -> 75.5 % of measured HBM
#pragma unroll 2
    for (; base + W <= nfull; base += S) {
      T e1[4], a2[2], e2[2];
      sh_unit<T, K, true>(xs, h, g, e1, a2, e2);
      if (lane < W) put_unit(d1p, d2p, lop, e1, a2, e2);
      xs += 8 * S;
      d1p += 4 * S;
      d2p += 2 * S;
      lop += 2 * S;
    }
  }
  for (; base < U; base += S) {
    const int u = base + lane;
    const T* xs = X + 8 * min(u, U - 1 + R);
    T e1[4] = {}, a2[2], e2[2] = {};
    // a pass past len/8 units keeps no details (halo units feed the coarser
    // levels' low-pass outputs only); the same for the whole warp
    if (4 * base < n1) sh_unit<T, K, true>(xs, h, g, e1, a2, e2);
    else sh_unit<T, K, false>(xs, h, g, e1, a2, e2);
    if (lane < W) {
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (4 * u + i < n1) d1[4 * u + i] = e1[i];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        if (2 * u + i < n2) d2[2 * u + i] = e2[i];
        if (2 * u + i < m2) lo[2 * u + i] = a2[i];
      }
    }
  }
}

template <typename T, int K, int NT, bool VEC>
__device__ __forceinline__ void dwt_pair(const T* X, T* lo, T* d1, T* d2, int len, int m2,
                                         const T* h, const T* g, int tid) {
  if constexpr (K >= 6) dwt_pair_sh<T, K, NT, VEC>(X, lo, d1, d2, len, m2, h, g, tid);
  else dwt_pair_rc<T, K, NT, VEC>(X, lo, d1, d2, len, m2, h, g, tid);
}

// One step on NT threads: the low-pass outputs go to shared memory (Y) or,
// on the last level, to the output; VEC when every output vector of a full
// unit is aligned.
template <typename T, int K, int NT>
__device__ __forceinline__ void dwt_pair_step(const T* X, T* Y, T* out, T* d1, T* d2, bool last,
                                              int len, int m2, const T* h, const T* g, int tid) {
  const bool vec = (uintptr_t)d1 % 16 == 0 && (uintptr_t)d2 % (2 * sizeof(T)) == 0 &&
                   (uintptr_t)out % (2 * sizeof(T)) == 0;
  if (!last) {
    if (vec) dwt_pair<T, K, NT, true>(X, Y, d1, d2, len, m2, h, g, tid);
    else dwt_pair<T, K, NT, false>(X, Y, d1, d2, len, m2, h, g, tid);
  } else {
    if (vec) dwt_pair<T, K, NT, true>(X, out, d1, d2, len, m2, h, g, tid);
    else dwt_pair<T, K, NT, false>(X, out, d1, d2, len, m2, h, g, tid);
  }
}

template <typename T, int K>
__global__ void __launch_bounds__(fthreads_a<K>()) k_filter_dwt(const FilterArgs a) {
  constexpr int NT = fthreads_a<K>(), CH = fchunk_a<K>();
  {
    // before the dependency wait, ask L2 for the chunk and its right halo
    // (up to the row's end; 64 x 2^20 fp32, 8 levels: Daubechies-4
    // analysis 97 -> 99 %, 8 taps 75.5 -> 77 % of measured HBM)
    const unsigned ch = (unsigned)a.chunks;
    const int64_t rw = blockIdx.x / ch, kk = (int64_t)(blockIdx.x % ch) * CH;
    const int64_t end = min(a.n, kk + CH + (K - 2) * ((1 << a.levels) - 1));
    warm_l2<NT>(static_cast<const T*>(a.in) + rw * a.n + kk, (end - kk) * (int64_t)sizeof(T),
                threadIdx.x);
  }
  pdl_wait();
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int L = a.levels;
  T* A = reinterpret_cast<T*>(smem_raw);
  T* B = A + fdwt_cap_a<T, K>(L);
  T h[K], g[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    h[k] = param<T>(a.h[k], a.hf[k]);
    g[k] = param<T>(a.g[k], a.gf[k]);
  }
  const unsigned chunks = (unsigned)a.chunks;
  const int64_t row = blockIdx.x / chunks, k0 = (int64_t)(blockIdx.x % chunks) * CH;
  const int64_t n = a.n;
  const int C = (int)min((int64_t)CH, n - k0);
  T* out = static_cast<T*>(a.out) + row * n;
  // the chunk and the (K - 2)(2^L - 1) samples to its right that the coarser
  // levels' filters reach; k0 is a multiple of 16 bytes, so no shift
  int r = (K - 2) * ((1 << L) - 1);
  stage<NT>(A, static_cast<const T*>(a.in) + row * n, n, k0, C + r, threadIdx.x);
  cp_async_wait_all();
  __syncthreads();
  T* X = A;
  T* Y = B;
  int len = C, l = 0;  // l levels done; X holds a_l (len of the chunk, halo r)
  bool solo = false;   // warp 0 alone from here on
  // pairs of levels
  for (; L - l >= 2; l += 2) {
    const int r2 = (r - 3 * (K - 2)) / 4;
    const int m2 = len / 4 + r2;
    T* d1 = out + (n >> (l + 1)) + (k0 >> (l + 1));
    T* d2 = out + (n >> (l + 2)) + (k0 >> (l + 2));
    T* lo = out + (k0 >> L);
    const bool last = l + 2 == L;
    if (!solo && (m2 + 1) / 2 > 64) {
      dwt_pair_step<T, K, NT>(X, Y, lo, d1, d2, last, len, m2, h, g, threadIdx.x);
      __syncthreads();
    } else {
      // at most 64 units: warp 0 alone, the other warps are done
      if (threadIdx.x >= 32) return;
      solo = true;
      dwt_pair_step<T, K, 32>(X, Y, lo, d1, d2, last, len, m2, h, g, threadIdx.x);
      __syncwarp();
    }
    T* t = X;
    X = Y;
    Y = t;
    len /= 4;
    r = r2;
  }
  // an odd number of levels: the coarsest one alone
  if (l < L) {
    const int half = len / 2;
    T* lo = out + (k0 >> L);
    T* dl = out + (n >> L) + (k0 >> L);
    if (!solo && half > 64) {
      dwt_level<T, K, NT>(X, lo, dl, half, half, h, g, threadIdx.x);
    } else if (threadIdx.x < 32) {
      dwt_level<T, K, 32>(X, lo, dl, half, half, h, g, threadIdx.x);
    }
  }
}

// ---- synthesis ----
// Window of level l: positions [lo(l), (m0 + C) >> l), lo(l) = (m0 >> l) - e_l.
// A "window-origin" pointer W has W[k] = the value at lo(l) + k.  Pairs of
// level l - 1 are q = lo(l) + HL + i; pair i reads a_l and d_l at window
// indices i + HL - t (t < K/2) and writes a_{l-1} at window indices
// 2i + p - (e_{l-1} mod 2).
//
// One level: pairs (2q, 2q+1) of level l-1, q = q0 + i, written to B[4p ..]
// (B index = window index + (e_{l-1} mod 2)); two pairs per thread share
// their loads.
template <typename T, int K, int NT>
__device__ __forceinline__ void idwt_level(const T* Acur, const T* D, T* B, int np,
                                           const T* h, const T* g, int tid) {
  constexpr int HL = K / 2 - 1;
  for (int p = tid; 2 * p < np; p += NT) {
    const int b1 = HL + 2 * p + 1;  // window index of the second pair
    T av[K / 2 + 1], dv[K / 2 + 1];
#pragma unroll
    for (int i = 0; i <= K / 2; ++i) {
      av[i] = Acur[b1 - i];
      dv[i] = D[b1 - i];
    }
    T e0 = T(0), o0 = T(0), e1 = T(0), o1 = T(0);
#pragma unroll
    for (int t = 0; t < K / 2; ++t) {
      e1 = fma(h[2 * t], av[t], e1);
      e1 = fma(g[2 * t], dv[t], e1);
      o1 = fma(h[2 * t + 1], av[t], o1);
      o1 = fma(g[2 * t + 1], dv[t], o1);
      e0 = fma(h[2 * t], av[t + 1], e0);
      e0 = fma(g[2 * t], dv[t + 1], e0);
      o0 = fma(h[2 * t + 1], av[t + 1], o0);
      o0 = fma(g[2 * t + 1], dv[t + 1], o0);
    }
    T* b = B + 4 * p;
    b[0] = e0;
    b[1] = o0;
    if (2 * p + 1 < np) {
      b[2] = e1;
      b[3] = o1;
    }
  }
}

// Two levels in one pass (l and l - 1): a unit makes pairs i' = 4u .. 4u + 3
// of level l - 1, i.e. 8 values of a_{l-2}.  They read a_{l-1} at window
// indices 4u .. 4u + 3 + HL, which come from the NP pairs of level l that
// start at 2u (made in registers; with ODD = e_{l-1} mod 2 the window index
// 4u + j is value j + ODD of those pairs), and those read a_l, d_l at window
// indices 2u .. 2u + NP - 1 + HL.  av, dv: a_l, d_l from 2u; d1: d_{l-1}
// from 4u.  y[2k + p] is output p of pair 4u + k.
template <int K, bool ODD>
struct SynShape {
  static constexpr int HL = K / 2 - 1;
  static constexpr int NP = (5 + HL + (ODD ? 1 : 0)) / 2;
  static constexpr int NA = NP + HL;
};

template <typename T, int K, bool ODD>
__device__ __forceinline__ void syn_unit(const T (&av)[SynShape<K, ODD>::NA],
                                         const T (&dv)[SynShape<K, ODD>::NA], const T (&d1)[K / 2 + 3],
                                         const T* h, const T* g, T (&y)[8]) {
  using S = SynShape<K, ODD>;
  constexpr int HL = S::HL;
  T z[2 * S::NP];
#pragma unroll
  for (int i = 0; i < S::NP; ++i) {
    T e = T(0), o = T(0);
#pragma unroll
    for (int t = 0; t < K / 2; ++t) {
      e = fma(h[2 * t], av[i + HL - t], e);
      e = fma(g[2 * t], dv[i + HL - t], e);
      o = fma(h[2 * t + 1], av[i + HL - t], o);
      o = fma(g[2 * t + 1], dv[i + HL - t], o);
    }
    z[2 * i] = e;
    z[2 * i + 1] = o;
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    T e = T(0), o = T(0);
#pragma unroll
    for (int t = 0; t < K / 2; ++t) {
      const T a = z[k + HL - t + (ODD ? 1 : 0)], d = d1[k + HL - t];
      e = fma(h[2 * t], a, e);
      e = fma(g[2 * t], d, e);
      o = fma(h[2 * t + 1], a, o);
      o = fma(g[2 * t + 1], d, o);
    }
    y[2 * k] = e;
    y[2 * k + 1] = o;
  }
}

// A coarse pass (levels l, l - 1 with l - 2 >= 2): window-origin pointers,
// element loads, 8 values per unit to P[8u ..] (P index = window index +
// (e_{l-2} mod 2), 16-byte aligned).
template <typename T, int K, int NT, bool ODD>
__device__ __forceinline__ void idwt_pair(const T* Aw, const T* Dw, const T* Dw1, T* P, int units,
                                          const T* h, const T* g, int tid) {
  using S = SynShape<K, ODD>;
  using VT = typename FVec16<T>::type;
  constexpr int V = fvec<T>();
  for (int u = tid; u < units; u += NT) {
    T av[S::NA], dv[S::NA], d1[K / 2 + 3];
#pragma unroll
    for (int s = 0; s < S::NA; ++s) {
      av[s] = Aw[2 * u + s];
      dv[s] = Dw[2 * u + s];
    }
#pragma unroll
    for (int j = 0; j < K / 2 + 3; ++j) d1[j] = Dw1[4 * u + j];
    T y[8];
    syn_unit<T, K, ODD>(av, dv, d1, h, g, y);
#pragma unroll
    for (int i = 0; i < 8 / V; ++i) {
      VT w;
      if constexpr (sizeof(T) == 4) w = make_float4(y[4 * i], y[4 * i + 1], y[4 * i + 2], y[4 * i + 3]);
      else w = VT{y[2 * i], y[2 * i + 1]};
      reinterpret_cast<VT*>(P + 8 * u)[i] = w;
    }
  }
}

// 8 consecutive output values at a unit's start, whose alignment is that of
// the chunk start (units are 8 values, chunks 4096 or 8192): one 256-bit store (AL =
// 32), 16-byte stores (AL = 16) or element stores (AL = 0).
template <typename T, int AL>
__device__ __forceinline__ void put8(T* p, const T (&y)[8]) {
  if constexpr (AL == 32 && sizeof(T) == 4) {
    asm volatile("st.global.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "f"(y[0]),
                 "f"(y[1]), "f"(y[2]), "f"(y[3]), "f"(y[4]), "f"(y[5]), "f"(y[6]), "f"(y[7])
                 : "memory");
  } else if constexpr (AL == 32) {
    asm volatile("st.global.v4.f64 [%0], {%1,%2,%3,%4};" ::"l"(p), "d"(y[0]), "d"(y[1]),
                 "d"(y[2]), "d"(y[3])
                 : "memory");
    asm volatile("st.global.v4.f64 [%0], {%1,%2,%3,%4};" ::"l"(p + 4), "d"(y[4]), "d"(y[5]),
                 "d"(y[6]), "d"(y[7])
                 : "memory");
  } else if constexpr (AL == 16) {
    store4(p, y);
    store4(p + 4, y + 4);
  } else {
#pragma unroll
    for (int i = 0; i < 8; ++i) p[i] = y[i];
  }
}

// The last pass (levels 2 and 1), straight to the output.  Every window
// shift is a compile-time constant here (e_1 and e_2 depend on K only), so
// a_2 and d_2 come in 2-element and d_1 in 16-byte aligned vectors from the
// buffer starts Ab, D2b, D1b.  a_2 sits in the big buffer (shift e_2 mod 2)
// or, for two levels, in its staged window.
template <typename T, int K, int NT, bool A_STAGED, int AL>
__device__ __forceinline__ void idwt_pair_last(const T* Ab, const T* D2b, const T* D1b, T* xo,
                                               int np1, const T* h, const T* g, int tid) {
  using V2 = typename FVec2<T>::type;
  using VT = typename FVec16<T>::type;
  constexpr int V = fvec<T>();
  constexpr int e1 = fe<K>(1), e2 = fe<K>(2);
  constexpr bool ODD = e1 & 1;
  using S = SynShape<K, ODD>;
  constexpr int SA = A_STAGED ? ((-e2) & (V - 1)) : (e2 & 1);
  constexpr int SD2 = (-e2) & (V - 1);
  constexpr int SD1 = (-e1) & (V - 1);
  constexpr int NLA = (SA + S::NA + 1) / 2, NLD = (SD2 + S::NA + 1) / 2;
  static_assert(SD1 + K / 2 + 3 <= 8, "d_1 reads stay inside the 8 loaded values");
  for (int u = tid; 4 * u < np1; u += NT) {
    T ra[2 * NLA], rd[2 * NLD], r1[8];
#pragma unroll
    for (int i = 0; i < NLA; ++i) {
      const V2 w = reinterpret_cast<const V2*>(Ab + 2 * u)[i];
      ra[2 * i] = w.x;
      ra[2 * i + 1] = w.y;
    }
#pragma unroll
    for (int i = 0; i < NLD; ++i) {
      const V2 w = reinterpret_cast<const V2*>(D2b + 2 * u)[i];
      rd[2 * i] = w.x;
      rd[2 * i + 1] = w.y;
    }
#pragma unroll
    for (int i = 0; i < 8 / V; ++i)
      *reinterpret_cast<VT*>(r1 + i * V) = reinterpret_cast<const VT*>(D1b + 4 * u)[i];
    T av[S::NA], dv[S::NA], d1[K / 2 + 3];
#pragma unroll
    for (int s = 0; s < S::NA; ++s) {
      av[s] = ra[s + SA];
      dv[s] = rd[s + SD2];
    }
#pragma unroll
    for (int j = 0; j < K / 2 + 3; ++j) d1[j] = r1[j + SD1];
    T y[8];
    syn_unit<T, K, ODD>(av, dv, d1, h, g, y);
    T* xp = xo + 8 * u;
    if (4 * u + 3 < np1) {
      put8<T, AL>(xp, y);
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (4 * u + k < np1) {
          xp[2 * k] = y[2 * k];
          xp[2 * k + 1] = y[2 * k + 1];
        }
    }
  }
}

// One level alone (a single-level transform): a thread makes 4 pairs from
// the staged a_1 and d_1 windows (shift (-HL) mod V for both).
template <typename T, int K, int NT, int AL>
__device__ __forceinline__ void idwt_level1(const T* A1, const T* D1, T* xo, int np, const T* h,
                                            const T* g, int tid) {
  using VT = typename FVec16<T>::type;
  constexpr int V = fvec<T>();
  constexpr int HL = K / 2 - 1;
  constexpr int SD = (-HL) & (V - 1);
  for (int p = tid; 4 * p < np; p += NT) {
    T ra[8], rd[8];
#pragma unroll
    for (int i = 0; i < 8 / V; ++i) {
      *reinterpret_cast<VT*>(ra + i * V) = reinterpret_cast<const VT*>(A1 + 4 * p)[i];
      *reinterpret_cast<VT*>(rd + i * V) = reinterpret_cast<const VT*>(D1 + 4 * p)[i];
    }
    T y[8];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      T e = T(0), o = T(0);
#pragma unroll
      for (int t = 0; t < K / 2; ++t) {
        const T av = ra[HL + k - t + SD], dv = rd[HL + k - t + SD];
        e = fma(h[2 * t], av, e);
        e = fma(g[2 * t], dv, e);
        o = fma(h[2 * t + 1], av, o);
        o = fma(g[2 * t + 1], dv, o);
      }
      y[2 * k] = e;
      y[2 * k + 1] = o;
    }
    T* xp = xo + 8 * p;
    if (4 * p + 3 < np) {
      put8<T, AL>(xp, y);
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (4 * p + k < np) {
          xp[2 * k] = y[2 * k];
          xp[2 * k + 1] = y[2 * k + 1];
        }
    }
  }
}

template <typename T, int K>
__global__ void __launch_bounds__(fthreads_s<K>()) k_filter_idwt(const FilterArgs a) {
  constexpr int V = fvec<T>(), CH = fchunk_s<K>(), NT = fthreads_s<K>();
  {
    const unsigned ch = (unsigned)a.chunks;
    const int64_t rw = blockIdx.x / ch, mm = (int64_t)(blockIdx.x % ch) * CH;
    const int64_t cc = min((int64_t)CH, a.n - mm);
    const T* cr = static_cast<const T*>(a.in) + rw * a.n;
    // before the dependency wait, ask L2 for the chunk's d_1 and d_2 (three
    // quarters of what the block reads; Daubechies-4 synthesis 96 -> 98 %,
    // 6 taps 89 -> 92 %)
    warm_l2<NT>(cr + (a.n >> 1) + (mm >> 1), (cc >> 1) * (int64_t)sizeof(T), threadIdx.x);
    if (a.levels >= 2)
      warm_l2<NT>(cr + (a.n >> 2) + (mm >> 2), (cc >> 2) * (int64_t)sizeof(T), threadIdx.x);
  }
  pdl_wait();
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int L = a.levels;
  T* S = reinterpret_cast<T*>(smem_raw);
  T* Pbig = S + fidwt_stage_cap<T, K>(L);
  T* Psmall = Pbig + fidwt_big_cap<T, K>();
  auto P = [&](int l) { return ((l >> 1) & 1) ? Pbig : Psmall; };  // holds a_l, l even
  T h[K], g[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    h[k] = param<T>(a.h[k], a.hf[k]);
    g[k] = param<T>(a.g[k], a.gf[k]);
  }
  const unsigned chunks = (unsigned)a.chunks;
  const int64_t row = blockIdx.x / chunks, m0 = (int64_t)(blockIdx.x % chunks) * CH;
  const int64_t n = a.n;
  const int C = (int)min((int64_t)CH, n - m0);
  const int64_t end = m0 + C;
  const T* c = static_cast<const T*>(a.in) + row * n;
  T* x = static_cast<T*>(a.out) + row * n;
  // stage the windows a_L, d_L, ..., d_1: window w by warp w mod 4, at the
  // offset the host computed, then one wait for everything
  {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int w = warp; w <= L; w += NT / 32) {
      const int l = w == 0 ? L : L + 1 - w;
      const int64_t nl = n >> l, s = (m0 >> l) - a.e[l];
      stage<32>(S + a.woff[w], w == 0 ? c : c + nl, nl, s, (int)((end >> l) - s), lane);
    }
  }
  cp_async_wait_all();
  __syncthreads();
  const int al = (uintptr_t)(x + m0) % 32 == 0 ? 32 : (uintptr_t)(x + m0) % 16 == 0 ? 16 : 0;
  auto win = [&](int l) {  // window-origin pointer of the staged d_l
    return S + a.woff[L + 1 - l] + ((-a.e[l]) & (V - 1));
  };
  if (L == 1) {
    const T *A1 = S + a.woff[0], *D1 = S + a.woff[1];
    if (al == 32) idwt_level1<T, K, NT, 32>(A1, D1, x + m0, C >> 1, h, g, threadIdx.x);
    else if (al == 16) idwt_level1<T, K, NT, 16>(A1, D1, x + m0, C >> 1, h, g, threadIdx.x);
    else idwt_level1<T, K, NT, 0>(A1, D1, x + m0, C >> 1, h, g, threadIdx.x);
    return;
  }
  // passes of at most 64 units run on warp 0 alone; the block waits for
  // them before its next pass
  bool warp0_wrote = false;
  auto phase = [&](int units) {
    if (units <= 64) {
      warp0_wrote = true;
      return threadIdx.x < 32 ? 1 : 0;  // 1: warp 0 runs it, 0: skip
    }
    if (warp0_wrote) __syncthreads();
    warp0_wrote = false;
    return 2;  // the whole block
  };
  const T* Aw = S + a.woff[0] + ((-a.e[L]) & (V - 1));  // a_L
  int l = L;
  if (L & 1) {  // an odd number of levels: level L alone first
    const int em = a.e[L - 1];
    const int np = (C >> L) + (em + 1) / 2;
    T* B = P(L - 1);
    const int ph = phase((np + 1) / 2);
    if (ph == 1) {
      idwt_level<T, K, 32>(Aw, win(L), B, np, h, g, threadIdx.x);
      __syncwarp();
    } else if (ph == 2) {
      idwt_level<T, K, NT>(Aw, win(L), B, np, h, g, threadIdx.x);
      __syncthreads();
    }
    Aw = B + (em & 1);
    l = L - 1;
  }
  for (; l >= 4; l -= 2) {
    const int e2 = a.e[l - 2];
    const bool odd = a.e[l - 1] & 1;
    const int units = ((C >> (l - 1)) + (e2 + 1) / 2 + 3) / 4;
    T* B = P(l - 2);
    const int ph = phase(units);
    if (ph != 0) {
      if (ph == 1) {
        if (odd) idwt_pair<T, K, 32, true>(Aw, win(l), win(l - 1), B, units, h, g, threadIdx.x);
        else idwt_pair<T, K, 32, false>(Aw, win(l), win(l - 1), B, units, h, g, threadIdx.x);
        __syncwarp();
      } else {
        if (odd)
          idwt_pair<T, K, NT, true>(Aw, win(l), win(l - 1), B, units, h, g, threadIdx.x);
        else
          idwt_pair<T, K, NT, false>(Aw, win(l), win(l - 1), B, units, h, g, threadIdx.x);
        __syncthreads();
      }
    }
    Aw = B + (e2 & 1);
  }
  if (warp0_wrote) __syncthreads();
  // levels 2 and 1 to the output
  if (L == 2) {
    const T *Ab = S + a.woff[0], *D2 = S + a.woff[1], *D1 = S + a.woff[2];
    if (al == 32)
      idwt_pair_last<T, K, NT, true, 32>(Ab, D2, D1, x + m0, C >> 1, h, g, threadIdx.x);
    else if (al == 16)
      idwt_pair_last<T, K, NT, true, 16>(Ab, D2, D1, x + m0, C >> 1, h, g, threadIdx.x);
    else
      idwt_pair_last<T, K, NT, true, 0>(Ab, D2, D1, x + m0, C >> 1, h, g, threadIdx.x);
  } else {
    const T *Ab = P(2), *D2 = S + a.woff[L - 1], *D1 = S + a.woff[L];
    if (al == 32)
      idwt_pair_last<T, K, NT, false, 32>(Ab, D2, D1, x + m0, C >> 1, h, g, threadIdx.x);
    else if (al == 16)
      idwt_pair_last<T, K, NT, false, 16>(Ab, D2, D1, x + m0, C >> 1, h, g, threadIdx.x);
    else
      idwt_pair_last<T, K, NT, false, 0>(Ab, D2, D1, x + m0, C >> 1, h, g, threadIdx.x);
  }
}

template <typename T, int K>
size_t filter_smem(bool fwd, int L) {
  const int elems = fwd ? fdwt_cap_a<T, K>(L) + fdwt_cap_b<T, K>(L)
                        : fidwt_stage_cap<T, K>(L) + fidwt_big_cap<T, K>() + fidwt_small_cap<T, K>();
  return (size_t)elems * sizeof(T);
}

template <typename T, int K>
cudaError_t filter_launch_k(bool fwd, FilterArgs a, cudaStream_t s) {
  const int chunk = fwd ? fchunk_a<K>() : fchunk_s<K>();
  a.chunks = (a.n + chunk - 1) / chunk;
  const int64_t total = a.rows * a.chunks;
  if (total == 0) return cudaSuccess;
  if (total > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  const size_t smem = filter_smem<T, K>(fwd, a.levels);
  auto kern = fwd ? k_filter_dwt<T, K> : k_filter_idwt<T, K>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)total);
  cfg.blockDim = dim3(fwd ? fthreads_a<K>() : fthreads_s<K>());
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, a);
}

// Offsets of the synthesis windows a_L, d_L, ..., d_1 in the staging area,
// and the e_l of their starts.
template <typename T, int K>
void window_offsets_k(FilterArgs& a) {
  int off = 0;
  for (int w = 0; w <= a.levels; ++w) {
    const int l = w == 0 ? a.levels : a.levels + 1 - w;
    a.woff[w] = off;
    off += fidwt_seg_cap<T, K>(l);
  }
  for (int l = 0; l <= a.levels; ++l) a.e[l] = fe<K>(l);
}
template <typename T>
cudaError_t window_offsets(FilterArgs& a, int K) {
  switch (K) {
    case 2: window_offsets_k<T, 2>(a); return cudaSuccess;
    case 4: window_offsets_k<T, 4>(a); return cudaSuccess;
    case 6: window_offsets_k<T, 6>(a); return cudaSuccess;
    case 8: window_offsets_k<T, 8>(a); return cudaSuccess;
  }
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t filter_launch(bool fwd, FilterArgs a, int K, cudaStream_t s) {
  switch (K) {
    case 2: return filter_launch_k<T, 2>(fwd, a, s);
    case 4: return filter_launch_k<T, 4>(fwd, a, s);
    case 6: return filter_launch_k<T, 6>(fwd, a, s);
    case 8: return filter_launch_k<T, 8>(fwd, a, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace fh

using namespace fh;

namespace {

int filter_entry(const void* in, void* out, int dtype, int64_t rows, int64_t n, int levels,
                 const double* lowpass, int ntaps, void* stream, bool fwd) {
  if (dtype != HAAR_F32 && dtype != HAAR_F64) return HAAR_EDTYPE;
  if (rows < 0 || n < 0 || levels < 1 || levels > kFMaxLevels) return HAAR_EINVAL;
  if (!lowpass || (ntaps != 2 && ntaps != 4 && ntaps != 6 && ntaps != 8)) return HAAR_EINVAL;
  if (rows == 0 || n == 0) return HAAR_OK;
  if (!in || !out) return HAAR_EINVAL;
  if (n & (((int64_t)1 << levels) - 1)) return HAAR_ESHAPE;
  const size_t esz = dtype == HAAR_F64 ? 8 : 4;
  const uintptr_t bytes = (uintptr_t)rows * (uintptr_t)n * esz;
  const uintptr_t il = (uintptr_t)in, ol = (uintptr_t)out;
  if (il < ol + bytes && ol < il + bytes) return HAAR_EALIAS;
  FilterArgs a{};
  a.in = in;
  a.out = out;
  a.rows = rows;
  a.n = n;
  a.levels = levels;
  for (int k = 0; k < ntaps; ++k) {
    a.h[k] = lowpass[k];
    a.g[k] = ((k & 1) ? 1.0 : -1.0) * lowpass[ntaps - 1 - k];  // (-1)^(k+1) h[K-1-k]
    a.hf[k] = (float)a.h[k];
    a.gf[k] = (float)a.g[k];
  }
  const cudaError_t e0 = dtype == HAAR_F64 ? window_offsets<double>(a, ntaps)
                                           : window_offsets<float>(a, ntaps);
  if (e0 != cudaSuccess) return HAAR_EINVAL;
  const cudaError_t e = dtype == HAAR_F64 ? filter_launch<double>(fwd, a, ntaps, (cudaStream_t)stream)
                                          : filter_launch<float>(fwd, a, ntaps, (cudaStream_t)stream);
  if (e != cudaSuccess) {
    set_last_cuda_error((int)e);
    return HAAR_ECUDA;
  }
  return HAAR_OK;
}

}  // namespace

extern "C" {

int haar_filter_dwt_1d(const void* x, void* coef, int dtype, int64_t rows, int64_t n, int levels,
                       const double* lowpass, int ntaps, void* cuda_stream) {
  return filter_entry(x, coef, dtype, rows, n, levels, lowpass, ntaps, cuda_stream, true);
}

int haar_filter_idwt_1d(const void* coef, void* x, int dtype, int64_t rows, int64_t n,
                        int levels, const double* lowpass, int ntaps, void* cuda_stream) {
  return filter_entry(coef, x, dtype, rows, n, levels, lowpass, ntaps, cuda_stream, false);
}

}  // extern "C"
