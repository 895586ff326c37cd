// haar_fast2d.cuh -- register/warp-shuffle 2D Fast Haar kernels for images
// whose sides are multiples of 32 (every workload of interest).
//
// Each warp owns a 32 x 32 pixel block; each lane owns a 4-row x 8-column
// micro-block (lane = 4 * ty + tx, ty = 0..7, tx = 0..3), read or written as
// four 8-wide row segments with 16-byte accesses.
//
// Analysis: levels 1 and 2 run inside the lane's registers (straight from
// the loads, Fig. 4 applied along rows and then columns); levels 3, 4 and 5
// pair lanes with warp shuffles (partners lane^4 / lane^1,^8 / lane^2,^16);
// a sixth level pairs the four warps of a 64 x 64 block through 32 bytes of
// shared memory.  No other shared memory and no other barrier is used.
//
// Synthesis (Eq. 19 along columns, then rows) needs no communication at all:
// each lane issues all of its loads up front -- its own level-1 and level-2
// detail coefficients and the (warp-shared, broadcast) coarser ones -- and
// walks the coarse levels down to its own micro-block.
//
// The butterflies perform exactly the same floating-point operations, in
// the same order, as fwd_quad / inv_quad, so results are bit-identical to
// the generic kernels.
#pragma once

#include "haar_internal.h"
#include "haar_kernels.cuh"

namespace fh {

// Mallat band addressing of one image: level-l band coordinates (row, col).
template <typename T>
struct Bands {
  T* base;
  int64_t rs, h, w;
  __device__ __forceinline__ T* hx(int l, int64_t row, int64_t col) const {
    return base + row * rs + (w >> l) + col;
  }
  __device__ __forceinline__ T* hy(int l, int64_t row, int64_t col) const {
    return base + ((h >> l) + row) * rs + col;
  }
  __device__ __forceinline__ T* hh(int l, int64_t row, int64_t col) const {
    return base + ((h >> l) + row) * rs + (w >> l) + col;
  }
};

// Horizontal half of a 2x2 butterfly across lanes lane and lane^mask:
// both lanes get lo = left + right and hi = right - left.
template <typename A>
__device__ __forceinline__ void hpair(A v, bool right, int mask, A& lo, A& hi) {
  const A o = __shfl_xor_sync(0xffffffffu, v, mask);
  lo = v + o;
  hi = right ? v - o : o - v;
}

// Vertical half across lanes lane and lane^mask (top/bottom rows' lo, hi):
// both lanes get the four bands, as fwd_quad computes them.
template <typename A>
__device__ __forceinline__ void vpair(A lo, A hi, bool bottom, int mask, A& ll, A& hx, A& hy,
                                      A& hh) {
  const A h = A(0.5);
  const A olo = __shfl_xor_sync(0xffffffffu, lo, mask);
  const A ohi = __shfl_xor_sync(0xffffffffu, hi, mask);
  ll = (lo + olo) * h;
  hy = (bottom ? lo - olo : olo - lo) * h;
  hx = (hi + ohi) * h;
  hh = (bottom ? hi - ohi : ohi - hi) * h;
}

// One output of the inverse butterfly: the child (qy, qx) of a coarse
// coefficient, with the same operations as inv_quad.
template <typename A>
__device__ __forceinline__ A inv_child(A ll, A hx, A hy, A hh, int qy, int qx) {
  const A sy = qy ? A(1) : A(-1), sx = qx ? A(1) : A(-1);
  const A s1 = fma(sy, hy, ll);  // ll -/+ hy, exactly rounded
  const A s2 = fma(sy, hh, hx);  // hx -/+ hh
  return fma(sx, s2, s1) * A(0.5);
}

// Output epilogues.  The block functions hand every value they produce to
// an epilogue object before it is stored: coefficients with a flag saying
// whether they are detail (true) or low-pass (false), output pixels in rows
// of eight.  EpiStore stores them unchanged; the fused loss pipeline
// (haar_denoise.cu) substitutes epilogues that transform, read a second
// array at the same position, and accumulate sums.
struct EpiStore {
  template <typename T, typename A>
  __device__ __forceinline__ void c4(T* p, const A v[4], bool) { store4(p, v); }
  template <typename T, typename A>
  __device__ __forceinline__ void c2(T* p, const A v[2], bool) { store2(p, v); }
  template <typename T, typename A>
  __device__ __forceinline__ void c1(T* p, A v, bool) { st_scalar(p, v); }
  template <typename T, typename A>
  __device__ __forceinline__ void px8(T* p, const A v[8]) { store8(p, v); }
};

// One image of a pass (pointers already offset to the batch item).
struct Img2 {
  const void* src;
  int64_t s_rs;
  void* dst;
  int64_t d_rs;
  void* ll;  // LL destination (analysis) or source (synthesis)
  int64_t l_rs;
  int ll_acc;  // 1: ll is accumulator typed (workspace), 0: coefficient typed
  int64_t h, w;
};

template <typename Tout, typename A>
__device__ __forceinline__ void put_ll(const Img2& im, int64_t row, int64_t col, A v) {
  const int64_t off = row * im.l_rs + col;
  if (im.ll_acc)
    static_cast<A*>(im.ll)[off] = v;
  else
    st_scalar(static_cast<Tout*>(im.ll) + off, v);
}

template <typename Tin, typename A>
__device__ __forceinline__ A get_ll(const Img2& im, int64_t row, int64_t col) {
  const int64_t off = row * im.l_rs + col;
  if (im.ll_acc) return static_cast<const A*>(im.ll)[off];
  return ld_scalar(static_cast<const Tin*>(im.ll) + off);
}

// A low-pass output: through the epilogue into the coefficient array, or
// unchanged into an accumulator-typed workspace (an intermediate band).
template <typename Tout, typename A, typename Epi>
__device__ __forceinline__ void put_ll_epi(const Img2& im, int64_t row, int64_t col, A v,
                                           Epi& epi) {
  if (im.ll_acc)
    static_cast<A*>(im.ll)[row * im.l_rs + col] = v;
  else
    epi.c1(static_cast<Tout*>(im.ll) + row * im.l_rs + col, v, false);
}

// ---------------------------------------------------------------------------
// Analysis of one 32 x 32 block by one warp: levels 1..min(L, 5), every
// band stored; returns LL5 (used by a sixth level when L = 6).
// ---------------------------------------------------------------------------
template <typename Tin, typename Tout, int L, typename Epi = EpiStore>
__device__ __forceinline__ typename AccT<Tin>::type dwt_block32(const Img2& im, int64_t y0,
                                                                int64_t x0, int lane,
                                                                Epi&& epi = Epi()) {
  using A = typename AccT<Tin>::type;
  static_assert(L >= 1 && L <= 6, "one warp fuses 1..6 levels");
  const int tx = lane & 3, ty = lane >> 2;
  const Bands<Tout> out{static_cast<Tout*>(im.dst), im.d_rs, im.h, im.w};
  const int64_t py = y0 + 4 * ty, px = x0 + 8 * tx;
  A l5 = A(0);

  const Tin* src = static_cast<const Tin*>(im.src) + py * im.s_rs + px;
  A v[4][8];
#pragma unroll
  for (int r = 0; r < 4; ++r) load8(src + r * im.s_rs, v[r]);

  // ---- level 1: eight 2x2 blocks per lane ----
  A l1[2][4];
#pragma unroll
  for (int rp = 0; rp < 2; ++rp) {
    A hx[4], hy[4], hh[4];
#pragma unroll
    for (int c = 0; c < 4; ++c)
      fwd_quad(v[2 * rp][2 * c], v[2 * rp][2 * c + 1], v[2 * rp + 1][2 * c],
               v[2 * rp + 1][2 * c + 1], l1[rp][c], hx[c], hy[c], hh[c]);
    const int64_t row = (py >> 1) + rp, col = px >> 1;
    epi.c4(out.hx(1, row, col), hx, true);
    epi.c4(out.hy(1, row, col), hy, true);
    epi.c4(out.hh(1, row, col), hh, true);
  }
  if constexpr (L == 1) {
#pragma unroll
    for (int rp = 0; rp < 2; ++rp) {
      const int64_t row = (py >> 1) + rp, col = px >> 1;
      if (!im.ll_acc) {
        epi.c4(static_cast<Tout*>(im.ll) + row * im.l_rs + col, l1[rp], false);
      } else {
#pragma unroll
        for (int c = 0; c < 4; ++c) put_ll<Tout>(im, row, col + c, l1[rp][c]);
      }
    }
  } else {
    // ---- level 2: two 2x2 blocks of LL1 per lane ----
    A l2[2];
    {
      A hx[2], hy[2], hh[2];
#pragma unroll
      for (int c = 0; c < 2; ++c)
        fwd_quad(l1[0][2 * c], l1[0][2 * c + 1], l1[1][2 * c], l1[1][2 * c + 1], l2[c], hx[c],
                 hy[c], hh[c]);
      const int64_t row = py >> 2, col = px >> 2;
      epi.c2(out.hx(2, row, col), hx, true);
      epi.c2(out.hy(2, row, col), hy, true);
      epi.c2(out.hh(2, row, col), hh, true);
    }
    if constexpr (L == 2) {
      const int64_t row = py >> 2, col = px >> 2;
      if (!im.ll_acc) {
        epi.c2(static_cast<Tout*>(im.ll) + row * im.l_rs + col, l2, false);
      } else {
        put_ll<Tout>(im, row, col, l2[0]);
        put_ll<Tout>(im, row, col + 1, l2[1]);
      }
    } else {
      // ---- level 3: horizontal pair in the lane, vertical pair lane^4 ----
      A l3, x3, y3, z3;
      vpair(l2[0] + l2[1], l2[1] - l2[0], (ty & 1) != 0, 4, l3, x3, y3, z3);
      const int64_t r3 = py >> 3, c3 = px >> 3;
      const bool own3 = (ty & 1) == 0;
      if (own3) {
        epi.c1(out.hx(3, r3, c3), x3, true);
        epi.c1(out.hy(3, r3, c3), y3, true);
        epi.c1(out.hh(3, r3, c3), z3, true);
      }
      if constexpr (L == 3) {
        if (own3) put_ll_epi<Tout>(im, r3, c3, l3, epi);
      } else {
        // ---- level 4: pairs lane^1 (columns) and lane^8 (rows) ----
        A lo, hi, l4, x4, y4, z4;
        hpair(l3, (tx & 1) != 0, 1, lo, hi);
        vpair(lo, hi, ((ty >> 1) & 1) != 0, 8, l4, x4, y4, z4);
        const int64_t r4 = py >> 4, c4 = px >> 4;
        const bool own4 = (ty & 3) == 0 && (tx & 1) == 0;
        if (own4) {
          epi.c1(out.hx(4, r4, c4), x4, true);
          epi.c1(out.hy(4, r4, c4), y4, true);
          epi.c1(out.hh(4, r4, c4), z4, true);
        }
        if constexpr (L == 4) {
          if (own4) put_ll_epi<Tout>(im, r4, c4, l4, epi);
        } else {
          // ---- level 5: pairs lane^2 (columns) and lane^16 (rows) ----
          A lo5, hi5, x5, y5, z5;
          hpair(l4, (tx & 2) != 0, 2, lo5, hi5);
          vpair(lo5, hi5, (ty & 4) != 0, 16, l5, x5, y5, z5);
          if (lane == 0) {
            const int64_t r5 = py >> 5, c5 = px >> 5;
            epi.c1(out.hx(5, r5, c5), x5, true);
            epi.c1(out.hy(5, r5, c5), y5, true);
            epi.c1(out.hh(5, r5, c5), z5, true);
            if constexpr (L == 5) put_ll_epi<Tout>(im, r5, c5, l5, epi);
          }
        }
      }
    }
  }
  return l5;
}

// Level 6 of one 64 x 64 block from the LL5 of its four 32 x 32 blocks.
template <typename Tout, typename A, typename Epi = EpiStore>
__device__ __forceinline__ void dwt_level6(const Img2& im, A tl, A tr, A bl, A br, int64_t by0,
                                           int64_t bx0, Epi&& epi = Epi()) {
  const Bands<Tout> out{static_cast<Tout*>(im.dst), im.d_rs, im.h, im.w};
  A l6, x6, y6, z6;
  fwd_quad(tl, tr, bl, br, l6, x6, y6, z6);
  const int64_t r6 = by0 >> 6, c6 = bx0 >> 6;
  epi.c1(out.hx(6, r6, c6), x6, true);
  epi.c1(out.hy(6, r6, c6), y6, true);
  epi.c1(out.hh(6, r6, c6), z6, true);
  put_ll_epi<Tout>(im, r6, c6, l6, epi);
}

// ---------------------------------------------------------------------------
// Synthesis of one 32 x 32 block by one warp (any L <= 6): every load is
// issued first -- the coarse coefficients, needed first, then the level-2
// and level-1 details -- and the lanes do not communicate.
// ---------------------------------------------------------------------------
template <typename Tin, typename Tout, int L, typename Epi = EpiStore>
__device__ __forceinline__ void idwt_block32(const Img2& im, int64_t y0, int64_t x0, int lane,
                                             Epi&& epi = Epi()) {
  using A = typename AccT<Tin>::type;
  static_assert(L >= 1 && L <= 6, "one warp undoes 1..6 levels");
  const int tx = lane & 3, ty = lane >> 2;
  const Bands<const Tin> in{static_cast<const Tin*>(im.src), im.s_rs, im.h, im.w};
  const int64_t py = y0 + 4 * ty, px = x0 + 8 * tx;

  A d1x[2][4], d1y[2][4], d1z[2][4];
  A ll1[2][4];
  A ll2[2];
  A d2x[2], d2y[2], d2z[2];
  A cxv[7], cyv[7], czv[7];  // levels 3..L
  A llL = A(0);
  if constexpr (L == 1) {
#pragma unroll
    for (int rp = 0; rp < 2; ++rp) {
      const int64_t row = (py >> 1) + rp, col = px >> 1;
      if (!im.ll_acc) {
        load4(static_cast<const Tin*>(im.ll) + row * im.l_rs + col, ll1[rp]);
      } else {
#pragma unroll
        for (int c = 0; c < 4; ++c) ll1[rp][c] = get_ll<Tin, A>(im, row, col + c);
      }
    }
  } else {
    const int64_t row = py >> 2, col = px >> 2;
    load2(in.hx(2, row, col), d2x);
    load2(in.hy(2, row, col), d2y);
    load2(in.hh(2, row, col), d2z);
    if constexpr (L == 2) {
      if (!im.ll_acc) {
        load2(static_cast<const Tin*>(im.ll) + row * im.l_rs + col, ll2);
      } else {
        ll2[0] = get_ll<Tin, A>(im, row, col);
        ll2[1] = get_ll<Tin, A>(im, row, col + 1);
      }
    } else {
#pragma unroll
      for (int l = 3; l <= L; ++l) {
        const int64_t r = py >> l, c = px >> l;
        cxv[l] = ld_scalar(in.hx(l, r, c));
        cyv[l] = ld_scalar(in.hy(l, r, c));
        czv[l] = ld_scalar(in.hh(l, r, c));
      }
      llL = get_ll<Tin, A>(im, py >> L, px >> L);
    }
  }

#pragma unroll
  for (int rp = 0; rp < 2; ++rp) {
    const int64_t row = (py >> 1) + rp, col = px >> 1;
    load4(in.hx(1, row, col), d1x[rp]);
    load4(in.hy(1, row, col), d1y[rp]);
    load4(in.hh(1, row, col), d1z[rp]);
  }
  // ---- coarse levels: walk down to this lane's LL2 pair ----
  if constexpr (L >= 3) {
    A v = llL;
#pragma unroll
    for (int l = L; l >= 4; --l)
      v = inv_child(v, cxv[l], cyv[l], czv[l], (int)((py >> (l - 1)) & 1),
                    (int)((px >> (l - 1)) & 1));
    const int qy = (int)((py >> 2) & 1);
    ll2[0] = inv_child(v, cxv[3], cyv[3], czv[3], qy, 0);
    ll2[1] = inv_child(v, cxv[3], cyv[3], czv[3], qy, 1);
  }
  // ---- level 2: LL1 (2 x 4) ----
  if constexpr (L >= 2) {
#pragma unroll
    for (int c = 0; c < 2; ++c)
      inv_quad(ll2[c], d2x[c], d2y[c], d2z[c], ll1[0][2 * c], ll1[0][2 * c + 1], ll1[1][2 * c],
               ll1[1][2 * c + 1]);
  }
  // ---- level 1: the 4 x 8 micro-block ----
  Tout* dst = static_cast<Tout*>(im.dst) + py * im.d_rs + px;
#pragma unroll
  for (int rp = 0; rp < 2; ++rp) {
    A o0[8], o1[8];
#pragma unroll
    for (int c = 0; c < 4; ++c)
      inv_quad(ll1[rp][c], d1x[rp][c], d1y[rp][c], d1z[rp][c], o0[2 * c], o0[2 * c + 1],
               o1[2 * c], o1[2 * c + 1]);
    epi.px8(dst + (2 * rp) * im.d_rs, o0);
    epi.px8(dst + (2 * rp + 1) * im.d_rs, o1);
  }
}

// One batch item of a pass.  A coefficient-typed low band is an output of
// the analysis (Tout) but an input of the synthesis (Tin): the batch offset
// is scaled by that type.
template <typename Tin, typename Tout>
__device__ __forceinline__ Img2 pass_image(const Pass& p, int64_t b, bool analysis) {
  using A = typename AccT<Tin>::type;
  Img2 im;
  im.src = static_cast<const Tin*>(p.src) + b * p.s_bs;
  im.s_rs = p.s_rs;
  im.dst = static_cast<Tout*>(p.dst) + b * p.d_bs;
  im.d_rs = p.d_rs;
  im.ll = p.ll_acc   ? (void*)(static_cast<A*>(p.ll) + b * p.l_bs)
          : analysis ? (void*)(static_cast<Tout*>(p.ll) + b * p.l_bs)
                     : (void*)(const_cast<Tin*>(static_cast<const Tin*>(p.ll)) + b * p.l_bs);
  im.l_rs = p.l_rs;
  im.ll_acc = p.ll_acc;
  im.h = p.h;
  im.w = p.w;
  return im;
}

// ---------------------------------------------------------------------------
// Strided-batch kernels.  Analysis block of warps: 1 x 4 (32 x 128 px) for
// L <= 5, 2 x 4 (64 x 128 px) for L = 6.  Synthesis: 1 x 4 for every L.
// Four-warp blocks finish a launch with a finer tail than eight-warp ones
// (4096^2 fp32, 5 levels: DWT + IDWT 41.45 against 42.12 us); two-warp
// blocks measured the same as four.  The launch bounds below declare 256
// threads, which fixes the register caps they state.
// ---------------------------------------------------------------------------
// Analysis: inputs of at most 2 bytes carry half the bytes per instruction
// or less, so more resident warps hide more latency: registers capped for 6
// blocks per SM (bf16 64 x 2048^2, 4 levels: 0.167 against 0.191 ms).  fp32
// keeps its 5 blocks (42 registers; a cap for 6 measured slower); fp64, the
// verification path, is not capped.
template <typename Tin>
constexpr int dwt_min_blocks() {
  return sizeof(Tin) <= 2 ? 6 : sizeof(Tin) == 4 ? 5 : 1;
}
template <typename Tin, typename Tout, int L>
__global__ void __launch_bounds__(256, dwt_min_blocks<Tin>()) k_dwt2d_fast(const Pass p) {
  pdl_wait();
  pdl_trigger();
  using A = typename AccT<Tin>::type;
  constexpr int WR = (L == 6) ? 2 : 1;
  constexpr int WC = 4;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t per = p.tiles_x * p.tiles_y;
  const int64_t t = blockIdx.x;
  const int64_t b = t / per, rr = t - b * per;
  const int64_t cy = rr / p.tiles_x, cx = rr - cy * p.tiles_x;
  const int64_t y0 = cy * (32 * WR) + (warp / WC) * 32;
  const int64_t x0 = cx * (32 * WC) + (warp % WC) * 32;
  const Img2 im = pass_image<Tin, Tout>(p, b, true);
  A l5 = A(0);
  if (y0 < p.h && x0 < p.w) l5 = dwt_block32<Tin, Tout, L>(im, y0, x0, lane);
  if constexpr (L == 6) {
    __shared__ A s5[WR][WC];
    if (lane == 0) s5[warp / WC][warp % WC] = l5;
    __syncthreads();
    if (threadIdx.x < WC / 2) {
      const int j = threadIdx.x;
      const int64_t by0 = cy * 64, bx0 = cx * 128 + 64 * j;
      if (by0 < p.h && bx0 < p.w)
        dwt_level6<Tout>(im, s5[0][2 * j], s5[0][2 * j + 1], s5[1][2 * j], s5[1][2 * j + 1],
                         by0, bx0);
    }
  }
}

// Synthesis with FP32 arithmetic: registers capped for 6 resident blocks per
// SM (40 registers; measured 2 % faster than 5 blocks at 42 registers on the
// 4096^2 fp32 case).  FP64 arithmetic needs twice the registers: no cap.
template <typename Tin>
constexpr int idwt_min_blocks() {
  return sizeof(typename AccT<Tin>::type) == 8 ? 1 : 6;
}
template <typename Tin, typename Tout, int L>
__global__ void __launch_bounds__(256, idwt_min_blocks<Tin>()) k_idwt2d_fast(const Pass p) {
  pdl_wait();
  pdl_trigger();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t per = p.tiles_x * p.tiles_y;
  const int64_t t = blockIdx.x;
  const int64_t b = t / per, rr = t - b * per;
  const int64_t cy = rr / p.tiles_x, cx = rr - cy * p.tiles_x;
  const int64_t y0 = cy * 32, x0 = cx * 128 + warp * 32;
  if (y0 >= p.h || x0 >= p.w) return;
  idwt_block32<Tin, Tout, L>(pass_image<Tin, Tout>(p, b, false), y0, x0, lane);
}

template <typename Tin, typename Tout>
cudaError_t dwt2d_fast_t(Pass p, cudaStream_t s) {
  const int CH = p.levels == 6 ? 64 : 32, CW = 128;
  p.tiles_x = (p.w + CW - 1) / CW;
  p.tiles_y = (p.h + CH - 1) / CH;
  p.ntiles = p.batch * p.tiles_x * p.tiles_y;
  if (p.ntiles == 0) return cudaSuccess;
  if (p.ntiles > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  const unsigned g = (unsigned)p.ntiles;
  cudaError_t e = cudaSuccess;
  switch (p.levels) {
    case 1: e = launch_pdl(k_dwt2d_fast<Tin, Tout, 1>, g, 128, s, p); break;
    case 2: e = launch_pdl(k_dwt2d_fast<Tin, Tout, 2>, g, 128, s, p); break;
    case 3: e = launch_pdl(k_dwt2d_fast<Tin, Tout, 3>, g, 128, s, p); break;
    case 4: e = launch_pdl(k_dwt2d_fast<Tin, Tout, 4>, g, 128, s, p); break;
    case 5: e = launch_pdl(k_dwt2d_fast<Tin, Tout, 5>, g, 128, s, p); break;
    case 6: e = launch_pdl(k_dwt2d_fast<Tin, Tout, 6>, g, 256, s, p); break;
    default: return cudaErrorInvalidValue;
  }
  return e;
}

template <typename Tin, typename Tout>
cudaError_t idwt2d_fast_t(Pass p, cudaStream_t s) {
  p.tiles_x = (p.w + 127) / 128;
  p.tiles_y = (p.h + 31) / 32;
  p.ntiles = p.batch * p.tiles_x * p.tiles_y;
  if (p.ntiles == 0) return cudaSuccess;
  if (p.ntiles > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  const unsigned g = (unsigned)p.ntiles;
  cudaError_t e = cudaSuccess;
  switch (p.levels) {
    case 1: e = launch_pdl(k_idwt2d_fast<Tin, Tout, 1>, g, 128, s, p); break;
    case 2: e = launch_pdl(k_idwt2d_fast<Tin, Tout, 2>, g, 128, s, p); break;
    case 3: e = launch_pdl(k_idwt2d_fast<Tin, Tout, 3>, g, 128, s, p); break;
    case 4: e = launch_pdl(k_idwt2d_fast<Tin, Tout, 4>, g, 128, s, p); break;
    case 5: e = launch_pdl(k_idwt2d_fast<Tin, Tout, 5>, g, 128, s, p); break;
    case 6: e = launch_pdl(k_idwt2d_fast<Tin, Tout, 6>, g, 128, s, p); break;
    default: return cudaErrorInvalidValue;
  }
  return e;
}

}  // namespace fh
