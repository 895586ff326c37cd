// haar_kernels.cuh -- the fused multi-level Fast Haar kernels (1D and 2D,
// analysis and synthesis) as device templates.
//
// One thread block transforms one tile and fuses up to log2(tile height)
// levels (2D) or log2(chunk) levels (1D) on chip:
//   * level 1 runs straight from global memory: each thread loads two
//     8-wide row segments (a "quad" of four 2x2 blocks) with 16-byte loads,
//     forms the four bands with the polyphase butterfly (no decimated sample
//     is ever computed), stores the three level-1 detail bands with vector
//     stores and keeps LL_1 in shared memory;
//   * the remaining levels run in place in shared memory, which then holds
//     the tile's own Mallat layout of its LL_1 region;
//   * a final cooperative pass scatters that layout to the global Mallat
//     positions (coalesced along band rows).
// Synthesis mirrors this: level-1 detail loads are issued first, the deep
// coefficients are gathered into shared memory, the deep levels are undone
// in place, and level 1 writes the output rows with vector stores.
//
// Haar blocks never overlap, so tiles need no halo and are independent.
#pragma once

#include "haar_common.cuh"

namespace fh {

// Shared-memory row padding (in elements); keeps 16-byte row alignment.
constexpr int kPad = 4;

// ---------------------------------------------------------------------------
// Per-tile work descriptors (pointers already offset to the batch item).
// ---------------------------------------------------------------------------
struct Tile2 {
  const void* src;  // analysis: image (Tin); synthesis: coefficients (Tin)
  int64_t s_rs;
  void* dst;        // analysis: coefficients (Tout); synthesis: image (Tout)
  int64_t d_rs;
  void* ll;         // analysis: LL_L destination; synthesis: LL_L source
  int64_t l_rs;
  int ll_acc;       // 1: ll is an accumulator-typed workspace, 0: same type as coefficients
  int levels;
  int64_t h, w;     // full image extent of this pass
  int64_t y0, x0;   // tile origin
};

struct Tile1 {
  const void* src;
  void* dst;
  void* ll;
  int ll_acc;
  int levels;
  int64_t n;   // signal length of this pass
  int64_t x0;  // chunk origin
};

template <typename A>
__device__ __forceinline__ void sm_store4(A* p, const A v[4]);
template <>
__device__ __forceinline__ void sm_store4<float>(float* p, const float v[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
template <>
__device__ __forceinline__ void sm_store4<double>(double* p, const double v[4]) {
  reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
}
template <typename A>
__device__ __forceinline__ void sm_load4(const A* p, A v[4]) {
#pragma unroll
  for (int k = 0; k < 4; ++k) v[k] = p[k];
}

// Position of tile-local Mallat element (i, j) of the LL_1 region (valid
// extent H1 x W1) in the global layout.  Returns the global level g of the
// band (2..levels) and its row/column in the coefficient image, or g = 0 for
// an LL_levels element (row/column then relative to the LL destination).
struct GPos {
  int g;
  int64_t row, col;
};
__device__ __forceinline__ GPos mallat_pos2(int i, int j, int H1, int W1, int levels,
                                            int64_t h, int64_t w, int64_t y0, int64_t x0) {
  int hr = H1, wr = W1;
  for (int m = 1; m < levels; ++m) {
    const int h2 = hr >> 1, w2 = wr >> 1;
    if (i < h2 && j < w2) {
      hr = h2;
      wr = w2;
      continue;
    }
    const int g = m + 1;
    const int64_t oy = y0 >> g, ox = x0 >> g, Hg = h >> g, Wg = w >> g;
    GPos p;
    p.g = g;
    if (i < h2) {  // Hx
      p.row = oy + i;
      p.col = Wg + ox + (j - w2);
    } else if (j < w2) {  // Hy
      p.row = Hg + oy + (i - h2);
      p.col = ox + j;
    } else {  // HH
      p.row = Hg + oy + (i - h2);
      p.col = Wg + ox + (j - w2);
    }
    return p;
  }
  GPos p;
  p.g = 0;
  p.row = (y0 >> levels) + i;
  p.col = (x0 >> levels) + j;
  return p;
}

// ---------------------------------------------------------------------------
// 2D analysis of one tile.
// ---------------------------------------------------------------------------
template <typename Tin, typename Tout, int TH, int TW, int NT, bool VEC>
__device__ __forceinline__ void dwt2d_tile(const Tile2& t,
                                           typename AccT<Tin>::type (*S)[TW / 2 + kPad]) {
  using A = typename AccT<Tin>::type;
  const int tid = threadIdx.x;
  const int vh = (int)min((int64_t)TH, t.h - t.y0);
  const int vw = (int)min((int64_t)TW, t.w - t.x0);
  const Tin* __restrict__ src = static_cast<const Tin*>(t.src);
  Tout* __restrict__ dst = static_cast<Tout*>(t.dst);
  const int64_t hh1 = t.h >> 1, wh1 = t.w >> 1;
  const int64_t by = t.y0 >> 1, bx = t.x0 >> 1;

  // ---- level 1, straight from global memory ----
  if constexpr (VEC) {
    constexpr int QPR = TW / 8;             // quads per row pair
    constexpr int NQ = (TH / 2) * QPR;      // quads per tile
    static_assert(NQ % NT == 0, "tile must split evenly into quads");
    constexpr int QPT = NQ / NT;
    A r0[QPT][8], r1[QPT][8];
    bool ok[QPT];
#pragma unroll
    for (int k = 0; k < QPT; ++k) {
      const int q = tid + k * NT, rp = q / QPR, qc = q % QPR;
      ok[k] = (2 * rp < vh) && (8 * qc < vw);
      if (ok[k]) {
        const Tin* p0 = src + (t.y0 + 2 * rp) * t.s_rs + t.x0 + 8 * qc;
        load8(p0, r0[k]);
        load8(p0 + t.s_rs, r1[k]);
      }
    }
#pragma unroll
    for (int k = 0; k < QPT; ++k) {
      if (!ok[k]) continue;
      const int q = tid + k * NT, rp = q / QPR, qc = q % QPR;
      A ll[4], hx[4], hy[4], hh[4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        fwd_quad(r0[k][2 * u], r0[k][2 * u + 1], r1[k][2 * u], r1[k][2 * u + 1], ll[u], hx[u],
                 hy[u], hh[u]);
      const int64_t row = by + rp, col = bx + 4 * qc;
      store4(dst + row * t.d_rs + wh1 + col, hx);
      store4(dst + (hh1 + row) * t.d_rs + col, hy);
      store4(dst + (hh1 + row) * t.d_rs + wh1 + col, hh);
      sm_store4<A>(&S[rp][4 * qc], ll);
    }
  } else {
    constexpr int NB = (TH / 2) * (TW / 2);
    static_assert(NB % NT == 0, "tile must split evenly into 2x2 blocks");
    constexpr int BPT = NB / NT;
    A a[BPT], b[BPT], c[BPT], d[BPT];
    bool ok[BPT];
#pragma unroll
    for (int k = 0; k < BPT; ++k) {
      const int q = tid + k * NT, r = q / (TW / 2), cc = q % (TW / 2);
      ok[k] = (2 * r < vh) && (2 * cc < vw);
      if (ok[k]) {
        const Tin* p0 = src + (t.y0 + 2 * r) * t.s_rs + t.x0 + 2 * cc;
        a[k] = ld_scalar(p0);
        b[k] = ld_scalar(p0 + 1);
        c[k] = ld_scalar(p0 + t.s_rs);
        d[k] = ld_scalar(p0 + t.s_rs + 1);
      }
    }
#pragma unroll
    for (int k = 0; k < BPT; ++k) {
      if (!ok[k]) continue;
      const int q = tid + k * NT, r = q / (TW / 2), cc = q % (TW / 2);
      A ll, hx, hy, hh;
      fwd_quad(a[k], b[k], c[k], d[k], ll, hx, hy, hh);
      const int64_t row = by + r, col = bx + cc;
      st_scalar(dst + row * t.d_rs + wh1 + col, hx);
      st_scalar(dst + (hh1 + row) * t.d_rs + col, hy);
      st_scalar(dst + (hh1 + row) * t.d_rs + wh1 + col, hh);
      S[r][cc] = ll;
    }
  }
  __syncthreads();

  // ---- levels 2..L in place in shared memory ----
  const int H1 = vh >> 1, W1 = vw >> 1;
  constexpr int KD = ((TH / 4) * (TW / 4) + NT - 1) / NT;
  for (int m = 1; m < t.levels; ++m) {
    const int hr = H1 >> (m - 1), wr = W1 >> (m - 1);
    const int h2 = hr >> 1, w2 = wr >> 1, nb = h2 * w2;
    A vll[KD], vhx[KD], vhy[KD], vhh[KD];
#pragma unroll
    for (int k = 0; k < KD; ++k) {
      const int q = tid + k * NT;
      if (q < nb) {
        const int i = q / w2, j = q % w2;
        fwd_quad(S[2 * i][2 * j], S[2 * i][2 * j + 1], S[2 * i + 1][2 * j], S[2 * i + 1][2 * j + 1],
                 vll[k], vhx[k], vhy[k], vhh[k]);
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < KD; ++k) {
      const int q = tid + k * NT;
      if (q < nb) {
        const int i = q / w2, j = q % w2;
        S[i][j] = vll[k];
        S[i][w2 + j] = vhx[k];
        S[h2 + i][j] = vhy[k];
        S[h2 + i][w2 + j] = vhh[k];
      }
    }
    __syncthreads();
  }

  // ---- scatter the tile-local layout to the global Mallat positions ----
  const int n1 = H1 * W1;
  for (int idx = tid; idx < n1; idx += NT) {
    const int i = idx / W1, j = idx % W1;
    const GPos p = mallat_pos2(i, j, H1, W1, t.levels, t.h, t.w, t.y0, t.x0);
    const A v = S[i][j];
    if (p.g) {
      st_scalar(dst + p.row * t.d_rs + p.col, v);
    } else if (t.ll_acc) {
      static_cast<A*>(t.ll)[p.row * t.l_rs + p.col] = v;
    } else {
      st_scalar(static_cast<Tout*>(t.ll) + p.row * t.l_rs + p.col, v);
    }
  }
}

// ---------------------------------------------------------------------------
// 2D synthesis of one tile.
// ---------------------------------------------------------------------------
template <typename Tin, typename Tout, int TH, int TW, int NT, bool VEC>
__device__ __forceinline__ void idwt2d_tile(const Tile2& t,
                                            typename AccT<Tin>::type (*S)[TW / 2 + kPad]) {
  using A = typename AccT<Tin>::type;
  const int tid = threadIdx.x;
  const int vh = (int)min((int64_t)TH, t.h - t.y0);
  const int vw = (int)min((int64_t)TW, t.w - t.x0);
  const Tin* __restrict__ src = static_cast<const Tin*>(t.src);
  Tout* __restrict__ dst = static_cast<Tout*>(t.dst);
  const int64_t hh1 = t.h >> 1, wh1 = t.w >> 1;
  const int64_t by = t.y0 >> 1, bx = t.x0 >> 1;
  const int H1 = vh >> 1, W1 = vw >> 1;

  constexpr int QPR = TW / 8;
  constexpr int NQ = (TH / 2) * QPR;
  constexpr int QPT = VEC ? NQ / NT : 1;
  static_assert(!VEC || NQ % NT == 0, "tile must split evenly into quads");
  A hx[QPT][4], hy[QPT][4], hh[QPT][4];
  bool ok[QPT];

  // ---- issue the level-1 detail loads first (3/4 of all coefficients) ----
  if constexpr (VEC) {
#pragma unroll
    for (int k = 0; k < QPT; ++k) {
      const int q = tid + k * NT, rp = q / QPR, qc = q % QPR;
      ok[k] = (2 * rp < vh) && (8 * qc < vw);
      if (ok[k]) {
        const int64_t row = by + rp, col = bx + 4 * qc;
        load4(src + row * t.s_rs + wh1 + col, hx[k]);
        load4(src + (hh1 + row) * t.s_rs + col, hy[k]);
        load4(src + (hh1 + row) * t.s_rs + wh1 + col, hh[k]);
      }
    }
  }

  // ---- gather the deep coefficients (LL_1 region's layout) into smem ----
  const int n1 = H1 * W1;
  for (int idx = tid; idx < n1; idx += NT) {
    const int i = idx / W1, j = idx % W1;
    const GPos p = mallat_pos2(i, j, H1, W1, t.levels, t.h, t.w, t.y0, t.x0);
    A v;
    if (p.g) {
      v = ld_scalar(src + p.row * t.s_rs + p.col);
    } else if (t.ll_acc) {
      v = static_cast<const A*>(t.ll)[p.row * t.l_rs + p.col];
    } else {
      v = ld_scalar(static_cast<const Tin*>(t.ll) + p.row * t.l_rs + p.col);
    }
    S[i][j] = v;
  }
  __syncthreads();

  // ---- undo levels L..2 in place, coarsest first ----
  constexpr int KD = ((TH / 4) * (TW / 4) + NT - 1) / NT;
  for (int m = t.levels - 1; m >= 1; --m) {
    const int hr = H1 >> (m - 1), wr = W1 >> (m - 1);
    const int h2 = hr >> 1, w2 = wr >> 1, nb = h2 * w2;
    A va[KD], vb[KD], vc[KD], vd[KD];
#pragma unroll
    for (int k = 0; k < KD; ++k) {
      const int q = tid + k * NT;
      if (q < nb) {
        const int i = q / w2, j = q % w2;
        inv_quad(S[i][j], S[i][w2 + j], S[h2 + i][j], S[h2 + i][w2 + j], va[k], vb[k], vc[k],
                 vd[k]);
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < KD; ++k) {
      const int q = tid + k * NT;
      if (q < nb) {
        const int i = q / w2, j = q % w2;
        S[2 * i][2 * j] = va[k];
        S[2 * i][2 * j + 1] = vb[k];
        S[2 * i + 1][2 * j] = vc[k];
        S[2 * i + 1][2 * j + 1] = vd[k];
      }
    }
    __syncthreads();
  }

  // ---- level 1: write the output rows ----
  if constexpr (VEC) {
#pragma unroll
    for (int k = 0; k < QPT; ++k) {
      if (!ok[k]) continue;
      const int q = tid + k * NT, rp = q / QPR, qc = q % QPR;
      A ll[4];
      sm_load4<A>(&S[rp][4 * qc], ll);
      A o0[8], o1[8];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        inv_quad(ll[u], hx[k][u], hy[k][u], hh[k][u], o0[2 * u], o0[2 * u + 1], o1[2 * u],
                 o1[2 * u + 1]);
      Tout* p0 = dst + (t.y0 + 2 * rp) * t.d_rs + t.x0 + 8 * qc;
      store8(p0, o0);
      store8(p0 + t.d_rs, o1);
    }
  } else {
    constexpr int NB = (TH / 2) * (TW / 2);
    static_assert(NB % NT == 0, "tile must split evenly into 2x2 blocks");
    constexpr int BPT = NB / NT;
#pragma unroll
    for (int k = 0; k < BPT; ++k) {
      const int q = tid + k * NT, r = q / (TW / 2), cc = q % (TW / 2);
      if (!((2 * r < vh) && (2 * cc < vw))) continue;
      const int64_t row = by + r, col = bx + cc;
      const A ex = ld_scalar(src + row * t.s_rs + wh1 + col);
      const A ey = ld_scalar(src + (hh1 + row) * t.s_rs + col);
      const A ez = ld_scalar(src + (hh1 + row) * t.s_rs + wh1 + col);
      A a, b, c, d;
      inv_quad(S[r][cc], ex, ey, ez, a, b, c, d);
      Tout* p0 = dst + (t.y0 + 2 * r) * t.d_rs + t.x0 + 2 * cc;
      st_scalar(p0, a);
      st_scalar(p0 + 1, b);
      st_scalar(p0 + t.d_rs, c);
      st_scalar(p0 + t.d_rs + 1, d);
    }
  }
}

// ---------------------------------------------------------------------------
// 1D analysis / synthesis of one chunk of CH samples.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int64_t mallat_pos1(int idx, int V1, int levels, int64_t n, int64_t x0,
                                               int& g_out) {
  int r = V1;
  for (int m = 1; m < levels; ++m) {
    const int r2 = r >> 1;
    if (idx < r2) {
      r = r2;
      continue;
    }
    const int g = m + 1;
    g_out = g;
    return (n >> g) + (x0 >> g) + (idx - r2);
  }
  g_out = 0;
  return (x0 >> levels) + idx;
}

template <typename Tin, typename Tout, int CH, int NT, bool VEC>
__device__ __forceinline__ void dwt1d_chunk(const Tile1& t, typename AccT<Tin>::type* S) {
  using A = typename AccT<Tin>::type;
  const int tid = threadIdx.x;
  const int v = (int)min((int64_t)CH, t.n - t.x0);
  const Tin* __restrict__ src = static_cast<const Tin*>(t.src);
  Tout* __restrict__ dst = static_cast<Tout*>(t.dst);
  const int64_t nh = t.n >> 1, bx = t.x0 >> 1;

  if constexpr (VEC) {
    constexpr int NG = CH / 8;
    static_assert(NG % NT == 0, "chunk must split evenly into groups of 8");
    constexpr int GPT = NG / NT;
    A r[GPT][8];
    bool ok[GPT];
#pragma unroll
    for (int k = 0; k < GPT; ++k) {
      const int g = tid + k * NT;
      ok[k] = 8 * g < v;
      if (ok[k]) load8(src + t.x0 + 8 * g, r[k]);
    }
#pragma unroll
    for (int k = 0; k < GPT; ++k) {
      if (!ok[k]) continue;
      const int g = tid + k * NT;
      A lo[4], hi[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) fwd_pair(r[k][2 * u], r[k][2 * u + 1], lo[u], hi[u]);
      store4(dst + nh + bx + 4 * g, hi);
      sm_store4<A>(&S[4 * g], lo);
    }
  } else {
    constexpr int NP = CH / 2;
    static_assert(NP % NT == 0, "chunk must split evenly into pairs");
    constexpr int PPT = NP / NT;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
      const int q = tid + k * NT;
      if (2 * q >= v) continue;
      A lo, hi;
      fwd_pair(ld_scalar(src + t.x0 + 2 * q), ld_scalar(src + t.x0 + 2 * q + 1), lo, hi);
      st_scalar(dst + nh + bx + q, hi);
      S[q] = lo;
    }
  }
  __syncthreads();

  const int V1 = v >> 1;
  constexpr int KD = (CH / 4 + NT - 1) / NT;
  for (int m = 1; m < t.levels; ++m) {
    const int r = V1 >> (m - 1), r2 = r >> 1;
    A vlo[KD], vhi[KD];
#pragma unroll
    for (int k = 0; k < KD; ++k) {
      const int q = tid + k * NT;
      if (q < r2) fwd_pair(S[2 * q], S[2 * q + 1], vlo[k], vhi[k]);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < KD; ++k) {
      const int q = tid + k * NT;
      if (q < r2) {
        S[q] = vlo[k];
        S[r2 + q] = vhi[k];
      }
    }
    __syncthreads();
  }

  for (int idx = tid; idx < V1; idx += NT) {
    int g;
    const int64_t pos = mallat_pos1(idx, V1, t.levels, t.n, t.x0, g);
    const A val = S[idx];
    if (g) {
      st_scalar(dst + pos, val);
    } else if (t.ll_acc) {
      static_cast<A*>(t.ll)[pos] = val;
    } else {
      st_scalar(static_cast<Tout*>(t.ll) + pos, val);
    }
  }
}

template <typename Tin, typename Tout, int CH, int NT, bool VEC>
__device__ __forceinline__ void idwt1d_chunk(const Tile1& t, typename AccT<Tin>::type* S) {
  using A = typename AccT<Tin>::type;
  const int tid = threadIdx.x;
  const int v = (int)min((int64_t)CH, t.n - t.x0);
  const Tin* __restrict__ src = static_cast<const Tin*>(t.src);
  Tout* __restrict__ dst = static_cast<Tout*>(t.dst);
  const int64_t nh = t.n >> 1, bx = t.x0 >> 1;
  const int V1 = v >> 1;

  constexpr int NG = CH / 8;
  constexpr int GPT = VEC ? NG / NT : 1;
  static_assert(!VEC || NG % NT == 0, "chunk must split evenly into groups of 8");
  A hi[GPT][4];
  bool ok[GPT];
  if constexpr (VEC) {
#pragma unroll
    for (int k = 0; k < GPT; ++k) {
      const int g = tid + k * NT;
      ok[k] = 8 * g < v;
      if (ok[k]) load4(src + nh + bx + 4 * g, hi[k]);
    }
  }

  for (int idx = tid; idx < V1; idx += NT) {
    int g;
    const int64_t pos = mallat_pos1(idx, V1, t.levels, t.n, t.x0, g);
    A val;
    if (g) {
      val = ld_scalar(src + pos);
    } else if (t.ll_acc) {
      val = static_cast<const A*>(t.ll)[pos];
    } else {
      val = ld_scalar(static_cast<const Tin*>(t.ll) + pos);
    }
    S[idx] = val;
  }
  __syncthreads();

  constexpr int KD = (CH / 4 + NT - 1) / NT;
  for (int m = t.levels - 1; m >= 1; --m) {
    const int r = V1 >> (m - 1), r2 = r >> 1;
    A v0[KD], v1[KD];
#pragma unroll
    for (int k = 0; k < KD; ++k) {
      const int q = tid + k * NT;
      if (q < r2) inv_pair(S[q], S[r2 + q], v0[k], v1[k]);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < KD; ++k) {
      const int q = tid + k * NT;
      if (q < r2) {
        S[2 * q] = v0[k];
        S[2 * q + 1] = v1[k];
      }
    }
    __syncthreads();
  }

  if constexpr (VEC) {
#pragma unroll
    for (int k = 0; k < GPT; ++k) {
      if (!ok[k]) continue;
      const int g = tid + k * NT;
      A lo[4], o[8];
      sm_load4<A>(&S[4 * g], lo);
#pragma unroll
      for (int u = 0; u < 4; ++u) inv_pair(lo[u], hi[k][u], o[2 * u], o[2 * u + 1]);
      store8(dst + t.x0 + 8 * g, o);
    }
  } else {
    constexpr int NP = CH / 2;
    static_assert(NP % NT == 0, "chunk must split evenly into pairs");
    constexpr int PPT = NP / NT;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
      const int q = tid + k * NT;
      if (2 * q >= v) continue;
      A x0, x1;
      inv_pair(S[q], ld_scalar(src + nh + bx + q), x0, x1);
      st_scalar(dst + t.x0 + 2 * q, x0);
      st_scalar(dst + t.x0 + 2 * q + 1, x1);
    }
  }
}

}  // namespace fh
