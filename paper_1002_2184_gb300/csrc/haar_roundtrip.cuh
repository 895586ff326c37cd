// haar_roundtrip.cuh -- a 32 x 32 block taken through the 2D analysis into
// the registers of one warp, mapped coefficient by coefficient, and taken
// back through the synthesis, with no memory traffic in between.
//
// After the analysis (levels 1-2 inside each lane, 3-5 through warp
// shuffles, exactly the operations of dwt_block32) every lane holds its own
// level-1 and level-2 details and a copy of every coarser coefficient on its
// path, so the synthesis needs no communication at all.
#pragma once

#include "haar_fast2d.cuh"

namespace fh {

template <typename T, int L>
struct WarpCoefs {
  T x1[2][4], y1[2][4], z1[2][4];  // level-1 details (Hx, Hy, HH) of the lane
  T x2[2], y2[2], z2[2];           // level-2 details
  T xl[6], yl[6], zl[6];           // levels 3..5 (shared with the lane's group)
  T ll1[2][4], ll2[2], ll;         // low band: LL1 (L = 1), LL2 (L = 2), LL_L (L >= 3)
};

// Analysis of the block into registers (same operations as dwt_block32).
template <typename T, int L>
__device__ __forceinline__ void warp_analysis(const T* src, int64_t rs, int lane, WarpCoefs<T, L>& k) {
  const int tx = lane & 3, ty = lane >> 2;
  T v[4][8];
#pragma unroll
  for (int r = 0; r < 4; ++r) load8(src + r * rs, v[r]);
#pragma unroll
  for (int rp = 0; rp < 2; ++rp)
#pragma unroll
    for (int c = 0; c < 4; ++c)
      fwd_quad(v[2 * rp][2 * c], v[2 * rp][2 * c + 1], v[2 * rp + 1][2 * c],
               v[2 * rp + 1][2 * c + 1], k.ll1[rp][c], k.x1[rp][c], k.y1[rp][c], k.z1[rp][c]);
  if constexpr (L >= 2) {
#pragma unroll
    for (int c = 0; c < 2; ++c)
      fwd_quad(k.ll1[0][2 * c], k.ll1[0][2 * c + 1], k.ll1[1][2 * c], k.ll1[1][2 * c + 1],
               k.ll2[c], k.x2[c], k.y2[c], k.z2[c]);
  }
  if constexpr (L >= 3) {
    T l3;
    vpair(k.ll2[0] + k.ll2[1], k.ll2[1] - k.ll2[0], (ty & 1) != 0, 4, l3, k.xl[3], k.yl[3],
          k.zl[3]);
    k.ll = l3;
  }
  if constexpr (L >= 4) {
    T lo, hi, l4;
    hpair(k.ll, (tx & 1) != 0, 1, lo, hi);
    vpair(lo, hi, ((ty >> 1) & 1) != 0, 8, l4, k.xl[4], k.yl[4], k.zl[4]);
    k.ll = l4;
  }
  if constexpr (L >= 5) {
    T lo, hi, l5;
    hpair(k.ll, (tx & 2) != 0, 2, lo, hi);
    vpair(lo, hi, (ty & 4) != 0, 16, l5, k.xl[5], k.yl[5], k.zl[5]);
    k.ll = l5;
  }
}

// Applies op(value, detail, owner) to every coefficient the lane holds;
// `owner` is true for exactly one copy of each coefficient in the warp (the
// coarse levels are duplicated across lane groups), so sums count each once.
template <typename T, int L, typename Op>
__device__ __forceinline__ void warp_map(int lane, WarpCoefs<T, L>& k, Op& op) {
  const int tx = lane & 3, ty = lane >> 2;
#pragma unroll
  for (int rp = 0; rp < 2; ++rp)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      k.x1[rp][c] = op(k.x1[rp][c], true, true);
      k.y1[rp][c] = op(k.y1[rp][c], true, true);
      k.z1[rp][c] = op(k.z1[rp][c], true, true);
      if constexpr (L == 1) k.ll1[rp][c] = op(k.ll1[rp][c], false, true);
    }
  if constexpr (L >= 2) {
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      k.x2[c] = op(k.x2[c], true, true);
      k.y2[c] = op(k.y2[c], true, true);
      k.z2[c] = op(k.z2[c], true, true);
      if constexpr (L == 2) k.ll2[c] = op(k.ll2[c], false, true);
    }
  }
  const bool own[6] = {false, false, false, (ty & 1) == 0, (ty & 3) == 0 && (tx & 1) == 0,
                       lane == 0};
#pragma unroll
  for (int l = 3; l <= L; ++l) {
    k.xl[l] = op(k.xl[l], true, own[l]);
    k.yl[l] = op(k.yl[l], true, own[l]);
    k.zl[l] = op(k.zl[l], true, own[l]);
  }
  if constexpr (L >= 3) k.ll = op(k.ll, false, own[L]);
}

// Synthesis of the (mapped) coefficients back to the lane's 4 x 8 pixels.
template <typename T, int L>
__device__ __forceinline__ void warp_synthesis(int lane, int64_t py, int64_t px,
                                               WarpCoefs<T, L>& k, T o[4][8]) {
  (void)lane;
  if constexpr (L >= 3) {
    T v = k.ll;
#pragma unroll
    for (int l = L; l >= 4; --l)
      v = inv_child(v, k.xl[l], k.yl[l], k.zl[l], (int)((py >> (l - 1)) & 1),
                    (int)((px >> (l - 1)) & 1));
    const int qy = (int)((py >> 2) & 1);
    k.ll2[0] = inv_child(v, k.xl[3], k.yl[3], k.zl[3], qy, 0);
    k.ll2[1] = inv_child(v, k.xl[3], k.yl[3], k.zl[3], qy, 1);
  }
  if constexpr (L >= 2) {
#pragma unroll
    for (int c = 0; c < 2; ++c)
      inv_quad(k.ll2[c], k.x2[c], k.y2[c], k.z2[c], k.ll1[0][2 * c], k.ll1[0][2 * c + 1],
               k.ll1[1][2 * c], k.ll1[1][2 * c + 1]);
  }
#pragma unroll
  for (int rp = 0; rp < 2; ++rp)
#pragma unroll
    for (int c = 0; c < 4; ++c)
      inv_quad(k.ll1[rp][c], k.x1[rp][c], k.y1[rp][c], k.z1[rp][c], o[2 * rp][2 * c],
               o[2 * rp][2 * c + 1], o[2 * rp + 1][2 * c], o[2 * rp + 1][2 * c + 1]);
}

}  // namespace fh
