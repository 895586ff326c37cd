// haar_fast2d_wide.cuh -- 2D Fast Haar analysis of 1- and 2-byte images
// with a wide micro-block per lane.
//
// At one or two bytes per input pixel the analysis moves 3 or 4 bytes per
// pixel, so the register/warp-shuffle kernel of haar_fast2d.cuh, whose
// per-lane costs (addresses, shuffles, predicates, the coarse levels) are
// paid for every 4 x 8 pixels, runs out of instruction issue before HBM is
// busy.  Here a lane owns 4 rows x 16 columns instead: one or two 16-byte
// loads per row, level-1 details leave as 8 consecutive coefficients (one
// 16-byte store for 16-bit coefficients), and every coarse level costs half
// as much per pixel.  A warp covers 32 rows x 64 columns (lane = 4 ty + tx,
// rows 4 ty .., columns 16 tx ..):
//   level 1, 2: in the lane (2 x 8 -> 1 x 4 low-pass values);
//   level 3:    pairs of columns in the lane, rows with lane ^ 4;
//   level 4:    the lane's two level-3 columns, rows with lane ^ 8;
//   level 5:    columns with lane ^ 1, rows with lane ^ 16.
// Every butterfly performs exactly the operations of fwd_quad (the pair
// sums and differences first, then the scaled sums), so the coefficients
// are bit-identical to those of the other 2D kernels.
#pragma once

#include "haar_fast2d.cuh"

namespace fh {

// 16 consecutive input samples of one row, kept in their storage type until
// the row pair is transformed: one 16-byte load for bytes, two for 16-bit
// samples.
template <typename Tin> struct Row16 {
  uint4 u[sizeof(Tin)];
};
template <typename Tin>
__device__ __forceinline__ void ld_row16(const Tin* p, Row16<Tin>& r) {
#pragma unroll
  for (int k = 0; k < (int)sizeof(Tin); ++k) r.u[k] = __ldg(reinterpret_cast<const uint4*>(p) + k);
}
__device__ __forceinline__ void unpack16(const Row16<uint8_t>& r, float v[16]) {
  const uint32_t w[4] = {r.u[0].x, r.u[0].y, r.u[0].z, r.u[0].w};
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int k = 0; k < 4; ++k) v[4 * q + k] = u8_to_f32(w[q], k);
}
template <typename H2>
__device__ __forceinline__ float2 h2f(uint32_t w);
template <>
__device__ __forceinline__ float2 h2f<__nv_bfloat162>(uint32_t w) {
  return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w));
}
template <>
__device__ __forceinline__ float2 h2f<__half2>(uint32_t w) {
  return __half22float2(*reinterpret_cast<const __half2*>(&w));
}
template <typename T, typename H2>
__device__ __forceinline__ void unpack16_h(const Row16<T>& r, float v[16]) {
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const uint32_t w[4] = {r.u[k].x, r.u[k].y, r.u[k].z, r.u[k].w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float2 f = h2f<H2>(w[q]);
      v[8 * k + 2 * q] = f.x;
      v[8 * k + 2 * q + 1] = f.y;
    }
  }
}
__device__ __forceinline__ void unpack16(const Row16<__nv_bfloat16>& r, float v[16]) {
  unpack16_h<__nv_bfloat16, __nv_bfloat162>(r, v);
}
__device__ __forceinline__ void unpack16(const Row16<__half>& r, float v[16]) {
  unpack16_h<__half, __half2>(r, v);
}

// Analysis of one 32 x 64 block by one warp, levels 1..L (L <= 5).
template <typename Tin, typename Tout, int L>
__device__ __forceinline__ void dwt_block_w(const Img2& im, int64_t y0, int64_t x0, int lane) {
  static_assert(L >= 1 && L <= 5, "a 32-row warp block fuses at most 5 levels");
  using A = float;
  const int tx = lane & 3, ty = lane >> 2;
  const Bands<Tout> out{static_cast<Tout*>(im.dst), im.d_rs, im.h, im.w};
  const int64_t py = y0 + 4 * ty, px = x0 + 16 * tx;
  const Tin* src = static_cast<const Tin*>(im.src) + py * im.s_rs + px;
  Row16<Tin> raw[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) ld_row16(src + r * im.s_rs, raw[r]);

  // ---- level 1: two row pairs of eight 2x2 blocks ----
  A l1[2][8];
#pragma unroll
  for (int rp = 0; rp < 2; ++rp) {
    A top[16], bot[16];
    unpack16(raw[2 * rp], top);
    unpack16(raw[2 * rp + 1], bot);
    A hx[8], hy[8], hh[8];
#pragma unroll
    for (int c = 0; c < 8; ++c)
      fwd_quad(top[2 * c], top[2 * c + 1], bot[2 * c], bot[2 * c + 1], l1[rp][c], hx[c], hy[c],
               hh[c]);
    const int64_t row = (py >> 1) + rp, col = px >> 1;
    store8(out.hx(1, row, col), hx);
    store8(out.hy(1, row, col), hy);
    store8(out.hh(1, row, col), hh);
  }
  if constexpr (L == 1) {
#pragma unroll
    for (int rp = 0; rp < 2; ++rp)
      store8(static_cast<Tout*>(im.ll) + ((py >> 1) + rp) * im.l_rs + (px >> 1), l1[rp]);
    return;
  } else {
    // ---- level 2: four 2x2 blocks of LL1 ----
    A l2[4];
    {
      A hx[4], hy[4], hh[4];
#pragma unroll
      for (int c = 0; c < 4; ++c)
        fwd_quad(l1[0][2 * c], l1[0][2 * c + 1], l1[1][2 * c], l1[1][2 * c + 1], l2[c], hx[c],
                 hy[c], hh[c]);
      const int64_t row = py >> 2, col = px >> 2;
      store4(out.hx(2, row, col), hx);
      store4(out.hy(2, row, col), hy);
      store4(out.hh(2, row, col), hh);
    }
    if constexpr (L == 2) {
      store4(static_cast<Tout*>(im.ll) + (py >> 2) * im.l_rs + (px >> 2), l2);
      return;
    } else {
      // ---- level 3: column pairs in the lane, rows with lane ^ 4 ----
      A l3[2], x3[2], y3[2], z3[2];
      const bool bottom3 = (ty & 1) != 0;
#pragma unroll
      for (int c = 0; c < 2; ++c)
        vpair(l2[2 * c] + l2[2 * c + 1], l2[2 * c + 1] - l2[2 * c], bottom3, 4, l3[c], x3[c],
              y3[c], z3[c]);
      const int64_t r3 = py >> 3, c3 = px >> 3;
      if (!bottom3) {
        store2(out.hx(3, r3, c3), x3);
        store2(out.hy(3, r3, c3), y3);
        store2(out.hh(3, r3, c3), z3);
      }
      if constexpr (L == 3) {
        if (!bottom3) store2(static_cast<Tout*>(im.ll) + r3 * im.l_rs + c3, l3);
        return;
      } else {
        // ---- level 4: the two level-3 columns in the lane, rows with lane ^ 8 ----
        A l4, x4, y4, z4;
        const bool bottom4 = (ty & 2) != 0;
        vpair(l3[0] + l3[1], l3[1] - l3[0], bottom4, 8, l4, x4, y4, z4);
        const int64_t r4 = py >> 4, c4 = px >> 4;
        const bool own4 = (ty & 3) == 0;
        if (own4) {
          st_scalar(out.hx(4, r4, c4), x4);
          st_scalar(out.hy(4, r4, c4), y4);
          st_scalar(out.hh(4, r4, c4), z4);
        }
        if constexpr (L == 4) {
          if (own4) st_scalar(static_cast<Tout*>(im.ll) + r4 * im.l_rs + c4, l4);
          return;
        } else {
          // ---- level 5: columns with lane ^ 1, rows with lane ^ 16 ----
          A lo5, hi5, l5, x5, y5, z5;
          hpair(l4, (tx & 1) != 0, 1, lo5, hi5);
          vpair(lo5, hi5, (ty & 4) != 0, 16, l5, x5, y5, z5);
          if (ty == 0 && (tx & 1) == 0) {
            const int64_t r5 = py >> 5, c5 = px >> 5;
            st_scalar(out.hx(5, r5, c5), x5);
            st_scalar(out.hy(5, r5, c5), y5);
            st_scalar(out.hh(5, r5, c5), z5);
            st_scalar(static_cast<Tout*>(im.ll) + r5 * im.l_rs + c5, l5);
          }
        }
      }
    }
  }
}

// Blocks of WC warps side by side (WC x 64 columns); WARPS resident warps
// per SM set the register cap.  The input rows of a block are at least 128
// bytes, so the L2 warm-up asks for whole lines.
template <typename Tin, typename Tout, int L, int WC, int WARPS, int PF>
__global__ void __launch_bounds__(32 * WC, fast_min_blocks<1, WC, WARPS>())
    k_dwt2d_w(const Pass p) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t t = blockIdx.x;
  int64_t b, cy, cx;
  block_coords(p, b, cy, cx);
  const int64_t by0 = cy * 32, bx0 = cx * (64 * WC);
  if (PF == 1 || (PF == 2 && t < p.pf_blocks)) dwt_prefetch<Tin, 1, 2 * WC>(p, b, by0, bx0);
  pdl_wait();
  pdl_trigger();
  const int64_t x0 = bx0 + warp * 64;
  if (by0 < p.h && x0 < p.w)
    dwt_block_w<Tin, Tout, L>(pass_image<Tin, Tout>(p, b, true), by0, x0, lane);
}

// Whether a pass can take the wide kernel: width a multiple of 64, at most 5
// levels, the low band in the coefficient array, image rows and the
// coefficient rows 16-byte aligned (16-byte loads; 8 coefficients per
// store).
template <typename Tin, typename Tout>
inline bool wide_ok(const Pass& p) {
  const auto al16 = [](const void* q, int64_t bs, int64_t rs, int esz) {
    return ((uintptr_t)q % 16) == 0 && ((bs * esz) % 16) == 0 && ((rs * esz) % 16) == 0;
  };
  return p.w % 64 == 0 && p.levels <= 5 && !p.ll_acc &&
         al16(p.src, p.s_bs, p.s_rs, (int)sizeof(Tin)) &&
         al16(p.dst, p.d_bs, p.d_rs, (int)sizeof(Tout));
}

template <typename Tin, typename Tout, int WC, int WARPS, int PF>
cudaError_t dwt2d_w_cfg(Pass p, cudaStream_t s) {
  const int CW = 64 * WC;
  p.tiles_x = (p.w + CW - 1) / CW;
  p.tiles_y = (p.h + 31) / 32;
  p.ntiles = p.batch * p.tiles_x * p.tiles_y;
  if (p.ntiles == 0) return cudaSuccess;
  if (p.ntiles > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  p.pf_blocks = (int64_t)fast_sm_count() * (WARPS ? WARPS / WC : 1);
  const unsigned g = (unsigned)p.ntiles;
  const unsigned nt = 32 * WC;
  switch (p.levels) {
    case 1: return launch_pdl(k_dwt2d_w<Tin, Tout, 1, WC, WARPS, PF>, g, nt, s, p);
    case 2: return launch_pdl(k_dwt2d_w<Tin, Tout, 2, WC, WARPS, PF>, g, nt, s, p);
    case 3: return launch_pdl(k_dwt2d_w<Tin, Tout, 3, WC, WARPS, PF>, g, nt, s, p);
    case 4: return launch_pdl(k_dwt2d_w<Tin, Tout, 4, WC, WARPS, PF>, g, nt, s, p);
    case 5: return launch_pdl(k_dwt2d_w<Tin, Tout, 5, WC, WARPS, PF>, g, nt, s, p);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fh
