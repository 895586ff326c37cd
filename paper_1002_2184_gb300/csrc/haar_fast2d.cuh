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
// dwt_block32_regs takes the lane's 4 x 8 micro-block already loaded (rows
// py .. py + 3, columns px .. px + 7 with py = y0 + 4 ty, px = x0 + 8 tx).
template <typename Tin, typename Tout, int L, typename Epi = EpiStore>
__device__ __forceinline__ typename AccT<Tin>::type dwt_block32_regs(
    const Img2& im, int64_t y0, int64_t x0, int lane, typename AccT<Tin>::type (&v)[4][8],
    Epi&& epi = Epi()) {
  using A = typename AccT<Tin>::type;
  static_assert(L >= 1 && L <= 6, "one warp fuses 1..6 levels");
  const int tx = lane & 3, ty = lane >> 2;
  const Bands<Tout> out{static_cast<Tout*>(im.dst), im.d_rs, im.h, im.w};
  const int64_t py = y0 + 4 * ty, px = x0 + 8 * tx;
  A l5 = A(0);

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

template <typename Tin, typename Tout, int L, typename Epi = EpiStore>
__device__ __forceinline__ typename AccT<Tin>::type dwt_block32(const Img2& im, int64_t y0,
                                                                int64_t x0, int lane,
                                                                Epi&& epi = Epi()) {
  using A = typename AccT<Tin>::type;
  const int tx = lane & 3, ty = lane >> 2;
  const Tin* src = static_cast<const Tin*>(im.src) + (y0 + 4 * ty) * im.s_rs + x0 + 8 * tx;
  A v[4][8];
#pragma unroll
  for (int r = 0; r < 4; ++r) load8(src + r * im.s_rs, v[r]);
  return dwt_block32_regs<Tin, Tout, L>(im, y0, x0, lane, v, static_cast<Epi&&>(epi));
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
// L2 warm-up before the dependency wait.  Every kernel starts with
// griddepcontrol.wait, which holds it until the previous kernel in the stream
// has finished; a block launched early (programmatic dependent launch) would
// otherwise sit idle while the previous kernel drains, and the memory system
// would restart from empty once the wait returns.  A block therefore first
// asks L2 for the lines it is about to read (a prefetch is only a hint: the
// loads after the wait still see every write of the previous kernel, since
// L2 is the point of coherence), so the next launch's reads overlap the
// previous launch's last writes.  One prefetch per whole 128-byte line:
// several blocks or warps asking for parts of the same line measured slower
// than no prefetch at all.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void l2_prefetch(const char* p, int bytes) {
  if ((((uintptr_t)p | (unsigned)bytes) & 15u) == 0) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
  } else {
    for (int o = 0; o < bytes; o += 128)
      asm volatile("prefetch.global.L2 [%0];" ::"l"(p + o) : "memory");
  }
}

// One 128-byte piece of a band row: piece j of `row` of a band whose rows
// start at base (pitch in bytes) and hold row_bytes bytes in this block.
__device__ __forceinline__ void pf_piece(const char* base, int64_t pitch, int row, int j,
                                         int64_t row_bytes) {
  const int64_t off = (int64_t)j << 7;
  const int64_t rest = row_bytes - off;
  if (rest > 0) l2_prefetch(base + row * pitch + off, (int)(rest < 128 ? rest : 128));
}

// The analysis block's input: 32 * WR rows of 32 * WC samples, one 128-byte
// piece per thread (the pieces are numbered row-major and dealt out over
// the block's threads).
template <typename Tin, int WR, int WC>
__device__ __forceinline__ void dwt_prefetch(const Pass& p, int64_t b, int64_t by0,
                                             int64_t bx0) {
  constexpr int NL = (32 * WC * (int)sizeof(Tin) + 127) / 128;
  const int64_t rows = p.h - by0 < 32 * WR ? p.h - by0 : 32 * WR;
  const int64_t cols = p.w - bx0 < 32 * WC ? p.w - bx0 : 32 * WC;
  const char* base = reinterpret_cast<const char*>(static_cast<const Tin*>(p.src) + b * p.s_bs +
                                                   by0 * p.s_rs + bx0);
  const int64_t pitch = p.s_rs * (int64_t)sizeof(Tin);
  for (int s = threadIdx.x; s < rows * NL; s += blockDim.x)
    pf_piece(base, pitch, s / NL, s % NL, cols * (int64_t)sizeof(Tin));
}

// The synthesis block's level-1 detail rows (16 rows of each band), level-2
// rows (8 per band) and, for one or two levels, its low-band rows: deeper
// levels are 1/16 of the data or less.  Pieces are dealt out one per thread
// in the order level 1, level 2, low band.  (A version that built a table
// of rectangles per block and looped over it measured 21.3 against 19.4 us
// for this flat form, 4096^2 fp32, 5 levels.)
template <typename Tin, typename A, int L, int WC>
__device__ __forceinline__ void idwt_prefetch(const Pass& p, int64_t b, int64_t by0,
                                              int64_t bx0) {
  constexpr int ES = (int)sizeof(Tin);
  constexpr int NL1 = (16 * WC * ES + 127) / 128, NL2 = (8 * WC * ES + 127) / 128;
  constexpr int N1 = 3 * 16 * NL1, N2 = L >= 2 ? 3 * 8 * NL2 : 0;
  constexpr int NLL = L == 1 ? 16 * NL1 : (L == 2 ? 8 * NL2 : 0);
  const char* c = reinterpret_cast<const char*>(static_cast<const Tin*>(p.src) + b * p.s_bs);
  const int64_t pitch = p.s_rs * ES;
  const int64_t w1 = p.w >> 1, h1 = p.h >> 1, w2 = p.w >> 2, h2 = p.h >> 2;
  const int64_t c1 = bx0 >> 1, r1 = by0 >> 1, c2 = bx0 >> 2, r2 = by0 >> 2;
  const int64_t rb1 = (w1 - c1 < 16 * WC ? w1 - c1 : 16 * WC) * ES;
  const int64_t rb2 = (w2 - c2 < 8 * WC ? w2 - c2 : 8 * WC) * ES;
  for (int s = threadIdx.x; s < N1 + N2 + NLL; s += blockDim.x) {
    if (s < N1) {
      const int band = s / (16 * NL1), q = s - band * (16 * NL1);
      const int64_t row = r1 + (band ? h1 : 0), col = c1 + (band != 1 ? w1 : 0);
      pf_piece(c + (row * p.s_rs + col) * ES, pitch, q / NL1, q % NL1, rb1);
    } else if (s < N1 + N2) {
      const int t = s - N1, band = t / (8 * NL2), q = t - band * (8 * NL2);
      const int64_t row = r2 + (band ? h2 : 0), col = c2 + (band != 1 ? w2 : 0);
      pf_piece(c + (row * p.s_rs + col) * ES, pitch, q / NL2, q % NL2, rb2);
    } else {
      const int t = s - N1 - N2;
      const int64_t lsz = p.ll_acc ? (int64_t)sizeof(A) : (int64_t)ES;
      const char* ll = static_cast<const char*>(p.ll) + b * p.l_bs * lsz;
      const int64_t lpitch = p.l_rs * lsz;
      if constexpr (L == 1) {
        const int64_t rb = rb1 / ES * lsz;
        const int nl = (int)((rb + 127) >> 7);
        if (t < 16 * nl) pf_piece(ll + (r1 * p.l_rs + c1) * lsz, lpitch, t / nl, t % nl, rb);
      } else {
        const int64_t rb = rb2 / ES * lsz;
        const int nl = (int)((rb + 127) >> 7);
        if (t < 8 * nl) pf_piece(ll + (r2 * p.l_rs + c2) * lsz, lpitch, t / nl, t % nl, rb);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Strided-batch kernels.  A block is WC warps side by side (WC x 32 columns)
// and, for the analysis with a sixth level, two such rows (64 rows, so the
// four LL5 values of each 64 x 64 block meet in 32 bytes of shared memory).
// WARPS is the number of resident warps per SM the register cap is set for
// (0: no cap).  PF selects the L2 warm-up: 0 none, 1 every block, 2 the
// blocks of the first wave only (p.pf_blocks), which are the ones that can
// start while the previous kernel drains.
// ---------------------------------------------------------------------------
// Batch item and tile row / column of this block.  The launcher keeps the
// tile count below 2^31, so 32-bit divisions suffice (a 64-bit division is
// a long instruction sequence, paid by every warp).
__device__ __forceinline__ void block_coords(const Pass& p, int64_t& b, int64_t& cy,
                                             int64_t& cx) {
  const uint32_t t = blockIdx.x, per = (uint32_t)(p.tiles_x * p.tiles_y);
  const uint32_t tx = (uint32_t)p.tiles_x;
  const uint32_t bb = t / per, rr = t - bb * per;
  const uint32_t yy = rr / tx;
  b = bb;
  cy = yy;
  cx = rr - yy * tx;
}

template <int WR, int WC, int WARPS>
constexpr int fast_min_blocks() {
  return WARPS == 0 ? 1 : (WARPS / (WR * WC) > 0 ? WARPS / (WR * WC) : 1);
}

template <typename Tin, typename Tout, int L, int WC, int WARPS, int PF>
__global__ void __launch_bounds__(32 * WC * (L == 6 ? 2 : 1),
                                  fast_min_blocks<(L == 6 ? 2 : 1), WC, WARPS>())
    k_dwt2d_fast(const Pass p) {
  using A = typename AccT<Tin>::type;
  constexpr int WR = (L == 6) ? 2 : 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t t = blockIdx.x;
  int64_t b, cy, cx;
  block_coords(p, b, cy, cx);
  const int64_t by0 = cy * (32 * WR), bx0 = cx * (32 * WC);
  if (PF == 1 || (PF == 2 && t < p.pf_blocks)) dwt_prefetch<Tin, WR, WC>(p, b, by0, bx0);
  pdl_wait();
  pdl_trigger();
  const int64_t y0 = by0 + (warp / WC) * 32;
  const int64_t x0 = bx0 + (warp % WC) * 32;
  const Img2 im = pass_image<Tin, Tout>(p, b, true);
  A l5 = A(0);
  if (y0 < p.h && x0 < p.w) l5 = dwt_block32<Tin, Tout, L>(im, y0, x0, lane);
  if constexpr (L == 6) {
    __shared__ A s5[WR][WC];
    if (lane == 0) s5[warp / WC][warp % WC] = l5;
    __syncthreads();
    if (threadIdx.x < WC / 2) {
      const int j = threadIdx.x;
      const int64_t y6 = by0, x6 = bx0 + 64 * j;
      if (y6 < p.h && x6 < p.w)
        dwt_level6<Tout>(im, s5[0][2 * j], s5[0][2 * j + 1], s5[1][2 * j], s5[1][2 * j + 1], y6,
                         x6);
    }
  }
}

template <typename Tin, typename Tout, int L, int WC, int WARPS, int PF>
__global__ void __launch_bounds__(32 * WC, fast_min_blocks<1, WC, WARPS>())
    k_idwt2d_fast(const Pass p) {
  using A = typename AccT<Tin>::type;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t t = blockIdx.x;
  int64_t b, cy, cx;
  block_coords(p, b, cy, cx);
  const int64_t by0 = cy * 32, bx0 = cx * (32 * WC);
  if (PF == 1 || (PF == 2 && t < p.pf_blocks)) idwt_prefetch<Tin, A, L, WC>(p, b, by0, bx0);
  pdl_wait();
  pdl_trigger();
  const int64_t y0 = by0, x0 = bx0 + warp * 32;
  if (y0 >= p.h || x0 >= p.w) return;
  idwt_block32<Tin, Tout, L>(pass_image<Tin, Tout>(p, b, false), y0, x0, lane);
}

// SM count of the current device (cached per device).
int fast_sm_count();

// Launchers for one configuration; the blocks of the first wave are the
// SM count times the resident blocks per SM the register cap allows.
template <typename Tin, typename Tout, int WC, int WARPS, int PF>
cudaError_t dwt2d_fast_cfg(Pass p, cudaStream_t s) {
  const int CH = p.levels == 6 ? 64 : 32, CW = 32 * WC;
  p.tiles_x = (p.w + CW - 1) / CW;
  p.tiles_y = (p.h + CH - 1) / CH;
  p.ntiles = p.batch * p.tiles_x * p.tiles_y;
  if (p.ntiles == 0) return cudaSuccess;
  if (p.ntiles > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  const int wr = p.levels == 6 ? 2 : 1;
  p.pf_blocks = (int64_t)fast_sm_count() * (WARPS ? WARPS / (wr * WC) : 1);
  const unsigned g = (unsigned)p.ntiles;
  cudaError_t e = cudaSuccess;
  switch (p.levels) {
#define FH_DWT_CASE(LV)                                                                       \
  case LV:                                                                                    \
    e = launch_pdl(k_dwt2d_fast<Tin, Tout, LV, WC, WARPS, PF>, g, 32 * WC * (LV == 6 ? 2 : 1), \
                   s, p);                                                                     \
    break;
    FH_DWT_CASE(1)
    FH_DWT_CASE(2)
    FH_DWT_CASE(3)
    FH_DWT_CASE(4)
    FH_DWT_CASE(5)
    FH_DWT_CASE(6)
#undef FH_DWT_CASE
    default: return cudaErrorInvalidValue;
  }
  return e;
}

template <typename Tin, typename Tout, int WC, int WARPS, int PF>
cudaError_t idwt2d_fast_cfg(Pass p, cudaStream_t s) {
  const int CW = 32 * WC;
  p.tiles_x = (p.w + CW - 1) / CW;
  p.tiles_y = (p.h + 31) / 32;
  p.ntiles = p.batch * p.tiles_x * p.tiles_y;
  if (p.ntiles == 0) return cudaSuccess;
  if (p.ntiles > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  p.pf_blocks = (int64_t)fast_sm_count() * (WARPS ? WARPS / WC : 1);
  const unsigned g = (unsigned)p.ntiles;
  const unsigned nt = 32 * WC;
  cudaError_t e = cudaSuccess;
  switch (p.levels) {
#define FH_IDWT_CASE(LV)                                                          \
  case LV:                                                                        \
    e = launch_pdl(k_idwt2d_fast<Tin, Tout, LV, WC, WARPS, PF>, g, nt, s, p);     \
    break;
    FH_IDWT_CASE(1)
    FH_IDWT_CASE(2)
    FH_IDWT_CASE(3)
    FH_IDWT_CASE(4)
    FH_IDWT_CASE(5)
    FH_IDWT_CASE(6)
#undef FH_IDWT_CASE
    default: return cudaErrorInvalidValue;
  }
  return e;
}

// The configuration used per storage type, measured on 4096^2 fp32 with 5
// levels (one image per launch, where the warm-up matters most) and on the
// 64 x 2048^2 batch with 4 levels (fraction of the measured copy bandwidth):
//  * fp32 analysis: 2-warp blocks, 32 resident warps (64 registers; 24 and
//    48 warps were 1-2 % slower), warm-up in every block: 4096^2 19.5 us
//    (101 %) against 21.7 us without; batch 106 % against 105 %;
//  * fp32 synthesis: 2-warp blocks, 40 warps (48 registers), every block:
//    4096^2 19.4 against 21.6 us; batch 106 % against 105 %;
//  * 16-bit storage: 48 warps, warm-up in the first wave only (in every
//    block it costs more issue than it saves when a block moves half the
//    bytes: bf16 analysis 88 %, synthesis 86 %; first wave only 95 % and
//    101 %, none 95 % and 101 %); a synthesis writing fp32 keeps it in every
//    block (104 % against 103 %);
//  * uint8 input: 4-warp blocks (a block row is one 128-byte line), 48
//    warps, first wave only (79 %: bound by instruction issue at 3 bytes per
//    pixel, not by the warm-up);
//  * FP64 (the verification path): no register cap.
template <typename Tin> struct DwtCfg {
  static constexpr int WC = sizeof(Tin) == 1 ? 4 : 2;
  static constexpr int WARPS = sizeof(Tin) == 8 ? 0 : (sizeof(Tin) == 4 ? 32 : 48);
  static constexpr int PF = sizeof(Tin) >= 4 ? 1 : 2;
};
template <typename Tin, typename Tout> struct IdwtCfg {
  static constexpr int WC = sizeof(Tin) == 2 ? 4 : 2;
  static constexpr int WARPS = sizeof(Tin) == 8 ? 0 : (sizeof(Tin) == 4 ? 40 : 48);
  static constexpr int PF = (sizeof(Tin) >= 4 || sizeof(Tout) >= 4) ? 1 : 2;
};

template <typename Tin, typename Tout>
cudaError_t dwt2d_fast_t(Pass p, cudaStream_t s) {
  using C = DwtCfg<Tin>;
  return dwt2d_fast_cfg<Tin, Tout, C::WC, C::WARPS, C::PF>(p, s);
}
template <typename Tin, typename Tout>
cudaError_t idwt2d_fast_t(Pass p, cudaStream_t s) {
  using C = IdwtCfg<Tin, Tout>;
  return idwt2d_fast_cfg<Tin, Tout, C::WC, C::WARPS, C::PF>(p, s);
}

}  // namespace fh
