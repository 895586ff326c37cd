// haar_3d.cu -- multi-level separable 3D Haar transform of volumes (octant
// Mallat layout), analysis and synthesis, with its C ABI.
//
// The 2x2x2 butterfly is the bank of Fig. 4 along x, then y, then z: on each
// z-slice the x and y stages collapse to fwd_quad (exact factor 1/2), then
// each of the four bands is split along z by fwd_pair (factor 1/sqrt 2).
// Octant (bz, by, bx) of level l (b = 0 low, 1 high on that axis) sits at
// (bz D_l/2, by H_l/2, bx W_l/2) inside the level's region D_l x H_l x W_l.
//
// A block of 128 threads transforms one 8 x 8 x 64 tile and fuses up to
// three levels: each thread owns a 2 (z) x 2 (y) x 8 (x) micro-block, runs
// level 1 straight from four pairs of 16-byte row loads and stores its seven
// detail octants with 16-byte stores; deeper levels run in shared memory on
// the tile's low band, which is then scattered to the global layout.
// Transforms deeper than three levels chain launches through a workspace.
// Volumes the tiles cannot take (width not a multiple of 8 at some pass,
// unaligned rows) run a generic kernel per level instead.
#include <cuda_runtime.h>

#include <type_traits>

#include "fasthaar.h"
#include "haar_internal.h"
#include "haar_kernels.cuh"

namespace fh {

constexpr int kTD = 8, kTH = 8, kTW = 64, kNT3 = 128, k3dFused = 3;
constexpr int kSD = kTD / 2, kSH = kTH / 2, kSW = kTW / 2 + 4;  // shared low band (+pad)

struct Pass3 {
  const void* src;
  int64_t s_bs, s_zs, s_rs;
  void* dst;
  int64_t d_bs, d_zs, d_rs;
  void* ll;  // LLL_L destination (analysis) / source (synthesis)
  int64_t l_bs, l_zs, l_rs;
  int ll_acc;
  int levels;
  int64_t batch, d, h, w;
  int64_t tz, ty, tx, ntiles;
  int vec4;  // fp32 throughout, 16-byte aligned bases and strides, w % 32 == 0
};

// 3D butterfly on v[z][y][x]; o[bz][by][bx].
template <typename A>
__device__ __forceinline__ void fwd_oct(const A v[2][2][2], A o[2][2][2]) {
  A q[2][4];
#pragma unroll
  for (int z = 0; z < 2; ++z)
    fwd_quad(v[z][0][0], v[z][0][1], v[z][1][0], v[z][1][1], q[z][0], q[z][1], q[z][2], q[z][3]);
  // q[z] = (LL, Hx, Hy, HH) = bands (by, bx) = (0,0), (0,1), (1,0), (1,1)
#pragma unroll
  for (int k = 0; k < 4; ++k) fwd_pair(q[0][k], q[1][k], o[0][k >> 1][k & 1], o[1][k >> 1][k & 1]);
}

template <typename A>
__device__ __forceinline__ void inv_oct(const A o[2][2][2], A v[2][2][2]) {
  A q[2][4];
#pragma unroll
  for (int k = 0; k < 4; ++k) inv_pair(o[0][k >> 1][k & 1], o[1][k >> 1][k & 1], q[0][k], q[1][k]);
#pragma unroll
  for (int z = 0; z < 2; ++z)
    inv_quad(q[z][0], q[z][1], q[z][2], q[z][3], v[z][0][0], v[z][0][1], v[z][1][0], v[z][1][1]);
}

// Global index of octant (bz, by, bx) position (z, y, x) at level g.
__device__ __forceinline__ int64_t oct_off(const Pass3& p, int64_t zs, int64_t rs, int g, int bz,
                                           int by, int bx, int64_t z, int64_t y, int64_t x) {
  return (bz * (p.d >> g) + z) * zs + (by * (p.h >> g) + y) * rs + (bx * (p.w >> g) + x);
}

// Tile-local low-band layout: relative level m of the shared region; for an
// element (i, j, k) returns the global level g (>= 2) and octant, or g = 0
// for LLL_L.
struct Oct {
  int g, bz, by, bx;
  int i, j, k;  // position inside the octant (tile-local)
};
__device__ __forceinline__ Oct classify3(int i, int j, int k, int D1, int H1, int W1, int L) {
  int dr = D1, hr = H1, wr = W1;
  for (int m = 1; m < L; ++m) {
    const int d2 = dr >> 1, h2 = hr >> 1, w2 = wr >> 1;
    if (i < d2 && j < h2 && k < w2) {
      dr = d2;
      hr = h2;
      wr = w2;
      continue;
    }
    Oct o;
    o.g = m + 1;
    o.bz = i >= d2;
    o.by = j >= h2;
    o.bx = k >= w2;
    o.i = i - o.bz * d2;
    o.j = j - o.by * h2;
    o.k = k - o.bx * w2;
    return o;
  }
  Oct o;
  o.g = 0;
  o.bz = o.by = o.bx = 0;
  o.i = i;
  o.j = j;
  o.k = k;
  return o;
}

// The coefficients of levels 2..L and LLL_L that a full 8 x 8 x 64 tile
// exchanges with its tile-local low-band layout are exactly 128 aligned runs
// of four values (L <= 3): for L = 1 the 4 x 4 x 32 LLL_1; else 7 octants x
// 2 x 2 rows x 4 runs of level 2, then 7 x 2 runs of level 3 and 2 of LLL_3
// (L = 3) or 2 x 2 x 4 runs of LLL_2 (L = 2).  Thread t moves run t.
struct Run4 {
  int g, bz, by, bx;  // level (0 = LLL_L) and octant
  int i, j, k;        // position inside the octant, k a multiple of 4
  int si, sj, sk;     // position in the tile-local layout
};
template <int L>
__device__ __forceinline__ Run4 run4(int t) {
  Run4 r{};
  if constexpr (L == 1) {
    r.i = t >> 5;
    r.j = (t >> 3) & 3;
    r.k = 4 * (t & 7);
  } else {
    if (t < 112) {
      const int o = (t >> 4) + 1, row = (t >> 2) & 3;
      r.g = 2;
      r.bz = o >> 2;
      r.by = (o >> 1) & 1;
      r.bx = o & 1;
      r.i = row >> 1;
      r.j = row & 1;
      r.k = 4 * (t & 3);
    } else if (L == 2) {
      const int u = t - 112, row = u >> 2;
      r.i = row >> 1;
      r.j = row & 1;
      r.k = 4 * (u & 3);
    } else if (t < 126) {
      const int u = t - 112, o = (u >> 1) + 1;
      r.g = 3;
      r.bz = o >> 2;
      r.by = (o >> 1) & 1;
      r.bx = o & 1;
      r.k = 4 * (u & 1);
    } else {
      r.k = 4 * (t - 126);
    }
  }
  // octant extents in the layout of a full tile: 2 x 2 x 16 at level 2, 1 x 1 x 8 at 3
  r.si = r.g == 2 ? 2 * r.bz + r.i : r.g == 3 ? r.bz + r.i : r.i;
  r.sj = r.g == 2 ? 2 * r.by + r.j : r.g == 3 ? r.by + r.j : r.j;
  r.sk = r.g == 2 ? 16 * r.bx + r.k : r.g == 3 ? 8 * r.bx + r.k : r.k;
  return r;
}

template <typename Tin, typename Tout, int L>
__global__ void __launch_bounds__(kNT3) k_dwt3d(const Pass3 p) {
  pdl_wait();
  pdl_trigger();
  using A = typename AccT<Tin>::type;
  __shared__ __align__(16) A S[kSD][kSH][kSW];
  const int tid = threadIdx.x;
  const int64_t per_b = p.tz * p.ty * p.tx;
  const int64_t t = blockIdx.x;
  const int64_t b = t / per_b;
  int64_t r = t - b * per_b;
  const int64_t tzi = r / (p.ty * p.tx);
  r -= tzi * p.ty * p.tx;
  const int64_t tyi = r / p.tx, txi = r - tyi * p.tx;
  const int64_t z0 = tzi * kTD, y0 = tyi * kTH, x0 = txi * kTW;
  const int vd = (int)min((int64_t)kTD, p.d - z0), vh = (int)min((int64_t)kTH, p.h - y0);
  const int vw = (int)min((int64_t)kTW, p.w - x0);
  const Tin* src = static_cast<const Tin*>(p.src) + b * p.s_bs;
  Tout* dst = static_cast<Tout*>(p.dst) + b * p.d_bs;

  // ---- level 1 from global memory: micro-block (mz, my, mx) ----
  const int mx = tid & 7, my = (tid >> 3) & 3, mz = tid >> 5;
  if (2 * mz < vd && 2 * my < vh && 8 * mx < vw) {
    A v[2][2][8];
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
      for (int dy = 0; dy < 2; ++dy)
        load8(src + (z0 + 2 * mz + dz) * p.s_zs + (y0 + 2 * my + dy) * p.s_rs + x0 + 8 * mx,
              v[dz][dy]);
    A o[8][4];  // octant index (bz*4 + by*2 + bx), four x positions
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      A blk[2][2][2], out[2][2][2];
#pragma unroll
      for (int dz = 0; dz < 2; ++dz)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
          blk[dz][dy][0] = v[dz][dy][2 * c];
          blk[dz][dy][1] = v[dz][dy][2 * c + 1];
        }
      fwd_oct(blk, out);
#pragma unroll
      for (int q = 0; q < 8; ++q) o[q][c] = out[q >> 2][(q >> 1) & 1][q & 1];
    }
    const int64_t zz = (z0 >> 1) + mz, yy = (y0 >> 1) + my, xx = (x0 >> 1) + 4 * mx;
#pragma unroll
    for (int q = 1; q < 8; ++q)
      store4(dst + oct_off(p, p.d_zs, p.d_rs, 1, q >> 2, (q >> 1) & 1, q & 1, zz, yy, xx), o[q]);
    sm_store4<A>(&S[mz][my][4 * mx], o[0]);
  }
  __syncthreads();

  // ---- levels 2..L in shared memory ----
  const int D1 = vd >> 1, H1 = vh >> 1, W1 = vw >> 1;
#pragma unroll
  for (int m = 1; m < L; ++m) {
    const int dr = D1 >> (m - 1), hr = H1 >> (m - 1), wr = W1 >> (m - 1);
    const int d2 = dr >> 1, h2 = hr >> 1, w2 = wr >> 1, nb = d2 * h2 * w2;
    A res[2][2][2];
    int bi = -1, bj = 0, bk = 0;
    if (tid < nb) {  // at most 2 x 2 x 16 = 64 blocks
      bi = tid / (h2 * w2);
      const int rem = tid - bi * h2 * w2;
      bj = rem / w2;
      bk = rem - bj * w2;
      A blk[2][2][2];
#pragma unroll
      for (int dz = 0; dz < 2; ++dz)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
          for (int dx = 0; dx < 2; ++dx)
            blk[dz][dy][dx] = S[2 * bi + dz][2 * bj + dy][2 * bk + dx];
      fwd_oct(blk, res);
    }
    __syncthreads();
    if (bi >= 0) {
#pragma unroll
      for (int bz = 0; bz < 2; ++bz)
#pragma unroll
        for (int by = 0; by < 2; ++by)
#pragma unroll
          for (int bx = 0; bx < 2; ++bx)
            S[bz * d2 + bi][by * h2 + bj][bx * w2 + bk] = res[bz][by][bx];
    }
    __syncthreads();
  }

  // ---- scatter the tile's low-band layout to the global octants ----
  if constexpr (std::is_same<Tout, float>::value && std::is_same<A, float>::value) {
    if (p.vec4 && vd == kTD && vh == kTH && vw == kTW) {
      const Run4 r = run4<L>(tid);
      const float4 v = *reinterpret_cast<const float4*>(&S[r.si][r.sj][r.sk]);
      float* g = r.g ? dst + oct_off(p, p.d_zs, p.d_rs, r.g, r.bz, r.by, r.bx, (z0 >> r.g) + r.i,
                                     (y0 >> r.g) + r.j, (x0 >> r.g) + r.k)
                     : static_cast<float*>(p.ll) + b * p.l_bs + ((z0 >> L) + r.i) * p.l_zs +
                           ((y0 >> L) + r.j) * p.l_rs + (x0 >> L) + r.k;
      *reinterpret_cast<float4*>(g) = v;
      return;
    }
  }
  const int n1 = D1 * H1 * W1;
  for (int idx = tid; idx < n1; idx += kNT3) {
    const int i = idx / (H1 * W1), rem = idx - i * H1 * W1, j = rem / W1, k = rem - j * W1;
    const Oct o = classify3(i, j, k, D1, H1, W1, L);
    const A val = S[i][j][k];
    if (o.g) {
      st_scalar(dst + oct_off(p, p.d_zs, p.d_rs, o.g, o.bz, o.by, o.bx, (z0 >> o.g) + o.i,
                              (y0 >> o.g) + o.j, (x0 >> o.g) + o.k),
                val);
    } else {
      const int64_t off = b * p.l_bs + ((z0 >> L) + i) * p.l_zs + ((y0 >> L) + j) * p.l_rs +
                          (x0 >> L) + k;
      if (p.ll_acc)
        static_cast<A*>(p.ll)[off] = val;
      else
        st_scalar(static_cast<Tout*>(p.ll) + off, val);
    }
  }
}

template <typename Tin, typename Tout, int L>
__global__ void __launch_bounds__(kNT3) k_idwt3d(const Pass3 p) {
  pdl_wait();
  pdl_trigger();
  using A = typename AccT<Tin>::type;
  __shared__ __align__(16) A S[kSD][kSH][kSW];
  const int tid = threadIdx.x;
  const int64_t per_b = p.tz * p.ty * p.tx;
  const int64_t t = blockIdx.x;
  const int64_t b = t / per_b;
  int64_t r = t - b * per_b;
  const int64_t tzi = r / (p.ty * p.tx);
  r -= tzi * p.ty * p.tx;
  const int64_t tyi = r / p.tx, txi = r - tyi * p.tx;
  const int64_t z0 = tzi * kTD, y0 = tyi * kTH, x0 = txi * kTW;
  const int vd = (int)min((int64_t)kTD, p.d - z0), vh = (int)min((int64_t)kTH, p.h - y0);
  const int vw = (int)min((int64_t)kTW, p.w - x0);
  const Tin* src = static_cast<const Tin*>(p.src) + b * p.s_bs;
  Tout* dst = static_cast<Tout*>(p.dst) + b * p.d_bs;
  const int mx = tid & 7, my = (tid >> 3) & 3, mz = tid >> 5;
  const bool act = 2 * mz < vd && 2 * my < vh && 8 * mx < vw;

  // ---- level-1 details of this thread first ----
  A o[8][4];
  const int64_t zz = (z0 >> 1) + mz, yy = (y0 >> 1) + my, xx = (x0 >> 1) + 4 * mx;
  if (act) {
#pragma unroll
    for (int q = 1; q < 8; ++q)
      load4(src + oct_off(p, p.s_zs, p.s_rs, 1, q >> 2, (q >> 1) & 1, q & 1, zz, yy, xx), o[q]);
  }
  // ---- gather the deeper coefficients of the tile into shared memory ----
  const int D1 = vd >> 1, H1 = vh >> 1, W1 = vw >> 1;
  bool gathered = false;
  if constexpr (std::is_same<Tin, float>::value && std::is_same<A, float>::value) {
    if (p.vec4 && vd == kTD && vh == kTH && vw == kTW) {
      const Run4 r = run4<L>(tid);
      const float* g = r.g ? src + oct_off(p, p.s_zs, p.s_rs, r.g, r.bz, r.by, r.bx,
                                           (z0 >> r.g) + r.i, (y0 >> r.g) + r.j, (x0 >> r.g) + r.k)
                           : static_cast<const float*>(p.ll) + b * p.l_bs +
                                 ((z0 >> L) + r.i) * p.l_zs + ((y0 >> L) + r.j) * p.l_rs +
                                 (x0 >> L) + r.k;
      *reinterpret_cast<float4*>(&S[r.si][r.sj][r.sk]) = __ldg(reinterpret_cast<const float4*>(g));
      gathered = true;
    }
  }
  const int n1 = gathered ? 0 : D1 * H1 * W1;
  for (int idx = tid; idx < n1; idx += kNT3) {
    const int i = idx / (H1 * W1), rem = idx - i * H1 * W1, j = rem / W1, k = rem - j * W1;
    const Oct oc = classify3(i, j, k, D1, H1, W1, L);
    A val;
    if (oc.g) {
      val = ld_scalar(src + oct_off(p, p.s_zs, p.s_rs, oc.g, oc.bz, oc.by, oc.bx,
                                    (z0 >> oc.g) + oc.i, (y0 >> oc.g) + oc.j,
                                    (x0 >> oc.g) + oc.k));
    } else {
      const int64_t off = b * p.l_bs + ((z0 >> L) + i) * p.l_zs + ((y0 >> L) + j) * p.l_rs +
                          (x0 >> L) + k;
      val = p.ll_acc ? static_cast<const A*>(p.ll)[off]
                     : ld_scalar(static_cast<const Tin*>(p.ll) + off);
    }
    S[i][j][k] = val;
  }
  __syncthreads();

  // ---- undo levels L..2 in shared memory ----
#pragma unroll
  for (int m = L - 1; m >= 1; --m) {
    const int dr = D1 >> (m - 1), hr = H1 >> (m - 1), wr = W1 >> (m - 1);
    const int d2 = dr >> 1, h2 = hr >> 1, w2 = wr >> 1, nb = d2 * h2 * w2;
    A res[2][2][2];
    int bi = -1, bj = 0, bk = 0;
    if (tid < nb) {
      bi = tid / (h2 * w2);
      const int rem = tid - bi * h2 * w2;
      bj = rem / w2;
      bk = rem - bj * w2;
      A oc[2][2][2];
#pragma unroll
      for (int bz = 0; bz < 2; ++bz)
#pragma unroll
        for (int by = 0; by < 2; ++by)
#pragma unroll
          for (int bx = 0; bx < 2; ++bx)
            oc[bz][by][bx] = S[bz * d2 + bi][by * h2 + bj][bx * w2 + bk];
      inv_oct(oc, res);
    }
    __syncthreads();
    if (bi >= 0) {
#pragma unroll
      for (int dz = 0; dz < 2; ++dz)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
          for (int dx = 0; dx < 2; ++dx) S[2 * bi + dz][2 * bj + dy][2 * bk + dx] = res[dz][dy][dx];
    }
    __syncthreads();
  }

  // ---- level 1: this thread's micro-block ----
  if (act) {
    sm_load4<A>(&S[mz][my][4 * mx], o[0]);
    A v[2][2][8];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      A oc[2][2][2], blk[2][2][2];
#pragma unroll
      for (int q = 0; q < 8; ++q) oc[q >> 2][(q >> 1) & 1][q & 1] = o[q][c];
      inv_oct(oc, blk);
#pragma unroll
      for (int dz = 0; dz < 2; ++dz)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
          v[dz][dy][2 * c] = blk[dz][dy][0];
          v[dz][dy][2 * c + 1] = blk[dz][dy][1];
        }
    }
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
      for (int dy = 0; dy < 2; ++dy)
        store8(dst + (z0 + 2 * mz + dz) * p.d_zs + (y0 + 2 * my + dy) * p.d_rs + x0 + 8 * mx,
               v[dz][dy]);
  }
}

template <typename Tin, typename Tout>
cudaError_t launch3d(bool fwd, Pass3 p, cudaStream_t s) {
  p.tz = (p.d + kTD - 1) / kTD;
  p.ty = (p.h + kTH - 1) / kTH;
  p.tx = (p.w + kTW - 1) / kTW;
  p.ntiles = p.batch * p.tz * p.ty * p.tx;
  if (p.ntiles == 0) return cudaSuccess;
  if (p.ntiles > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  const unsigned g = (unsigned)p.ntiles;
  switch (p.levels) {
    case 1: return fwd ? launch_pdl(k_dwt3d<Tin, Tout, 1>, g, kNT3, s, p)
                       : launch_pdl(k_idwt3d<Tin, Tout, 1>, g, kNT3, s, p);
    case 2: return fwd ? launch_pdl(k_dwt3d<Tin, Tout, 2>, g, kNT3, s, p)
                       : launch_pdl(k_idwt3d<Tin, Tout, 2>, g, kNT3, s, p);
    case 3: return fwd ? launch_pdl(k_dwt3d<Tin, Tout, 3>, g, kNT3, s, p)
                       : launch_pdl(k_idwt3d<Tin, Tout, 3>, g, kNT3, s, p);
  }
  return cudaErrorInvalidValue;
}

// dtype pair -> launcher (same storage in and out; fp32 accumulator passes)
cudaError_t dispatch3d(bool fwd, int tin, int tout, const Pass3& p, cudaStream_t s) {
  if (tin == HAAR_F64 || tout == HAAR_F64)
    return (tin == HAAR_F64 && tout == HAAR_F64) ? launch3d<double, double>(fwd, p, s)
                                                 : cudaErrorInvalidValue;
  if (tin == HAAR_F32 && tout == HAAR_F32) return launch3d<float, float>(fwd, p, s);
  if (tin == HAAR_BF16 && tout == HAAR_BF16) return launch3d<__nv_bfloat16, __nv_bfloat16>(fwd, p, s);
  if (tin == HAAR_F16 && tout == HAAR_F16) return launch3d<__half, __half>(fwd, p, s);
  // intermediate passes: accumulator (fp32) in or out
  if (tin == HAAR_F32 && tout == HAAR_BF16) return launch3d<float, __nv_bfloat16>(fwd, p, s);
  if (tin == HAAR_F32 && tout == HAAR_F16) return launch3d<float, __half>(fwd, p, s);
  if (tin == HAAR_BF16 && tout == HAAR_F32) return launch3d<__nv_bfloat16, float>(fwd, p, s);
  if (tin == HAAR_F16 && tout == HAAR_F32) return launch3d<__half, float>(fwd, p, s);
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// Generic path for the volumes the tiled kernels cannot take (a width that
// is not a multiple of 8, rows, planes or batch items that are not 16-byte
// aligned, or a deep pass on a region narrower than 8): one thread per
// 2 x 2 x 2 block, one launch per level, every element loaded and stored on
// its own, the low band of each level in the workspace.  The butterflies are
// fwd_oct / inv_oct, as in the tiled kernels.
// ---------------------------------------------------------------------------
struct Lvl3 {
  void* io;  // the level's full-resolution side: input (analysis) / output (synthesis)
  int64_t i_bs, i_zs, i_rs;
  void* coef;  // details of every level (octant layout)
  int64_t c_bs, c_zs, c_rs;
  void* low;  // this level's LLL: output (analysis) / input (synthesis)
  int64_t l_bs, l_zs, l_rs;
  int64_t batch, d, h, w;  // the level's full-resolution region
};

// Block index t -> batch item b and block (i, j, k) of the half-size region.
__device__ __forceinline__ void gen3_index(const Lvl3& q, int64_t t, int64_t& b, int64_t& i,
                                           int64_t& j, int64_t& k) {
  const int64_t h2 = q.h >> 1, w2 = q.w >> 1, per = (q.d >> 1) * h2 * w2;
  b = t / per;
  int64_t r = t - b * per;
  i = r / (h2 * w2);
  r -= i * h2 * w2;
  j = r / w2;
  k = r - j * w2;
}

template <typename TS, typename TC, typename TL>
__global__ void __launch_bounds__(256) k_dwt3d_gen(const Lvl3 q) {
  pdl_wait();
  pdl_trigger();
  using A = typename AccT<TS>::type;
  const int64_t d2 = q.d >> 1, h2 = q.h >> 1, w2 = q.w >> 1;
  const int64_t total = q.batch * d2 * h2 * w2;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    int64_t b, i, j, k;
    gen3_index(q, t, b, i, j, k);
    const TS* src = static_cast<const TS*>(q.io) + b * q.i_bs + 2 * i * q.i_zs + 2 * j * q.i_rs +
                    2 * k;
    A v[2][2][2], o[2][2][2];
#pragma unroll
    for (int z = 0; z < 2; ++z)
#pragma unroll
      for (int y = 0; y < 2; ++y)
#pragma unroll
        for (int x = 0; x < 2; ++x) v[z][y][x] = ld_scalar(src + z * q.i_zs + y * q.i_rs + x);
    fwd_oct(v, o);
    TC* c = static_cast<TC*>(q.coef) + b * q.c_bs;
#pragma unroll
    for (int oc = 1; oc < 8; ++oc) {
      const int bz = oc >> 2, by = (oc >> 1) & 1, bx = oc & 1;
      st_scalar(c + (bz * d2 + i) * q.c_zs + (by * h2 + j) * q.c_rs + bx * w2 + k, o[bz][by][bx]);
    }
    st_scalar(static_cast<TL*>(q.low) + b * q.l_bs + i * q.l_zs + j * q.l_rs + k, o[0][0][0]);
  }
}

template <typename TL, typename TC, typename TD>
__global__ void __launch_bounds__(256) k_idwt3d_gen(const Lvl3 q) {
  pdl_wait();
  pdl_trigger();
  using A = typename AccT<TC>::type;
  const int64_t d2 = q.d >> 1, h2 = q.h >> 1, w2 = q.w >> 1;
  const int64_t total = q.batch * d2 * h2 * w2;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    int64_t b, i, j, k;
    gen3_index(q, t, b, i, j, k);
    const TC* c = static_cast<const TC*>(q.coef) + b * q.c_bs;
    A o[2][2][2], v[2][2][2];
    o[0][0][0] = ld_scalar(static_cast<const TL*>(q.low) + b * q.l_bs + i * q.l_zs + j * q.l_rs + k);
#pragma unroll
    for (int oc = 1; oc < 8; ++oc) {
      const int bz = oc >> 2, by = (oc >> 1) & 1, bx = oc & 1;
      o[bz][by][bx] = ld_scalar(c + (bz * d2 + i) * q.c_zs + (by * h2 + j) * q.c_rs + bx * w2 + k);
    }
    inv_oct(o, v);
    TD* dst = static_cast<TD*>(q.io) + b * q.i_bs + 2 * i * q.i_zs + 2 * j * q.i_rs + 2 * k;
#pragma unroll
    for (int z = 0; z < 2; ++z)
#pragma unroll
      for (int y = 0; y < 2; ++y)
#pragma unroll
        for (int x = 0; x < 2; ++x) st_scalar(dst + z * q.i_zs + y * q.i_rs + x, v[z][y][x]);
  }
}

// One level of the generic path.  ta / tb / tc: dtypes of (analysis) the
// input, the coefficients and the low band, or (synthesis) the low band, the
// coefficients and the output.
template <typename X, typename Y, typename Z>
cudaError_t gen3_go(bool fwd, const Lvl3& q, unsigned grid, cudaStream_t s) {
  if (fwd) return launch_pdl(k_dwt3d_gen<X, Y, Z>, grid, 256, s, q);
  return launch_pdl(k_idwt3d_gen<X, Y, Z>, grid, 256, s, q);
}
template <typename X, typename Y>
cudaError_t gen3_z(bool fwd, int tc, const Lvl3& q, unsigned grid, cudaStream_t s) {
  switch (tc) {
    case HAAR_F32: return gen3_go<X, Y, float>(fwd, q, grid, s);
    case HAAR_BF16: return gen3_go<X, Y, __nv_bfloat16>(fwd, q, grid, s);
    case HAAR_F16: return gen3_go<X, Y, __half>(fwd, q, grid, s);
  }
  return cudaErrorInvalidValue;
}
template <typename X>
cudaError_t gen3_y(bool fwd, int tb, int tc, const Lvl3& q, unsigned grid, cudaStream_t s) {
  switch (tb) {
    case HAAR_F32: return gen3_z<X, float>(fwd, tc, q, grid, s);
    case HAAR_BF16: return gen3_z<X, __nv_bfloat16>(fwd, tc, q, grid, s);
    case HAAR_F16: return gen3_z<X, __half>(fwd, tc, q, grid, s);
  }
  return cudaErrorInvalidValue;
}
cudaError_t dispatch3d_gen(bool fwd, int ta, int tb, int tc, const Lvl3& q, cudaStream_t s) {
  const int64_t total = q.batch * (q.d >> 1) * (q.h >> 1) * (q.w >> 1);
  if (total == 0) return cudaSuccess;
  int64_t g = (total + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;  // grid-stride beyond 32 blocks per SM
  const unsigned grid = (unsigned)g;
  if (ta == HAAR_F64 || tb == HAAR_F64 || tc == HAAR_F64)
    return (ta == HAAR_F64 && tb == HAAR_F64 && tc == HAAR_F64)
               ? gen3_go<double, double, double>(fwd, q, grid, s)
               : cudaErrorInvalidValue;
  switch (ta) {
    case HAAR_F32: return gen3_y<float>(fwd, tb, tc, q, grid, s);
    case HAAR_BF16: return gen3_y<__nv_bfloat16>(fwd, tb, tc, q, grid, s);
    case HAAR_F16: return gen3_y<__half>(fwd, tb, tc, q, grid, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace fh

using namespace fh;

namespace {

bool same_storage(int a) { return a == HAAR_F32 || a == HAAR_BF16 || a == HAAR_F16 || a == HAAR_F64; }

int check3(const haar_desc3* d) {
  if (!d || d->reserved) return HAAR_EINVAL;
  if (!same_storage(d->dtype)) return HAAR_EDTYPE;
  if (d->batch < 0 || d->d < 0 || d->h < 0 || d->w < 0 || d->batch_stride < 0 ||
      d->plane_stride < 0 || d->row_stride < 0)
    return HAAR_EINVAL;
  if (d->batch == 0 || d->d == 0 || d->h == 0 || d->w == 0) return HAAR_OK;
  if (!d->ptr) return HAAR_EINVAL;
  if (d->h > 1 && d->row_stride < d->w) return HAAR_EINVAL;
  if (d->d > 1 && d->plane_stride < (d->h - 1) * d->row_stride + d->w) return HAAR_EINVAL;
  if (d->batch > 1 && d->batch_stride < (d->d - 1) * d->plane_stride + (d->h - 1) * d->row_stride + d->w)
    return HAAR_EINVAL;
  return HAAR_OK;
}

int64_t extent3(const haar_desc3* d) {
  return (d->batch - 1) * d->batch_stride + (d->d - 1) * d->plane_stride +
         (d->h - 1) * d->row_stride + d->w;
}

int plan_passes3(int levels, int lv[64], int cum[65]) {
  int n = 0, done = 0;
  cum[0] = 0;
  while (done < levels) {
    const int l = levels - done < k3dFused ? levels - done : k3dFused;
    lv[n] = l;
    done += l;
    cum[++n] = done;
  }
  return n;
}

size_t ws3(const haar_desc3* x, int levels, size_t off[64]) {
  int lv[64], cum[65];
  const int n = plan_passes3(levels, lv, cum);
  const size_t esz = x->dtype == HAAR_F64 ? 8 : 4;
  size_t tot = 0;
  for (int k = 1; k < n; ++k) {
    const int s = cum[k];
    off[k] = tot;
    const size_t bytes = (size_t)x->batch * (size_t)(x->d >> s) * (size_t)(x->h >> s) *
                         (size_t)(x->w >> s) * esz;
    tot += (bytes + 255) & ~(size_t)255;
  }
  return tot;
}

// Whether the tiled kernels take a transform: every pass's region at least
// 8 wide and a multiple of 8 (rows move 8 samples at a time), and the rows,
// planes and batch items of both arrays 16-byte aligned.
bool tiled3_ok(const haar_desc3* in, const haar_desc3* out, int levels) {
  auto al = [](const haar_desc3* d) {
    const int esz = dt_size(d->dtype);
    return ((uintptr_t)d->ptr % 16) == 0 && (d->row_stride * esz) % 16 == 0 &&
           (d->plane_stride * esz) % 16 == 0 && (d->batch_stride * esz) % 16 == 0;
  };
  if (!al(in) || !al(out)) return false;
  int lv[64], cum[65];
  const int np = plan_passes3(levels, lv, cum);
  for (int k = 0; k < np; ++k)
    if ((in->w >> cum[k]) % 8) return false;
  return true;
}

// Workspace of the generic path: the low band of every level but the last
// (accumulator type), one region each.
size_t ws_gen3(const haar_desc3* x, int levels, size_t off[64]) {
  const size_t esz = x->dtype == HAAR_F64 ? 8 : 4;
  size_t tot = 0;
  for (int l = 1; l < levels && l < 64; ++l) {
    off[l] = tot;
    const size_t bytes = (size_t)x->batch * (size_t)(x->d >> l) * (size_t)(x->h >> l) *
                         (size_t)(x->w >> l) * esz;
    tot += (bytes + 255) & ~(size_t)255;
  }
  return tot;
}

int run_gen3(const haar_desc3* in, const haar_desc3* out, int levels, void* ws, size_t ws_bytes,
             void* stream, bool fwd) {
  size_t off[64];
  const size_t need = ws_gen3(in, levels, off);
  if (need && (!ws || ws_bytes < need || ((uintptr_t)ws & 255))) return HAAR_EWORKSPACE;
  const int tin = in->dtype, tout = out->dtype;
  const int acc = tin == HAAR_F64 ? HAAR_F64 : HAAR_F32;
  char* wsb = static_cast<char*>(ws);
  const cudaStream_t st = (cudaStream_t)stream;
  const haar_desc3* coef = fwd ? out : in;
  const haar_desc3* img = fwd ? in : out;
  for (int kk = 0; kk < levels; ++kk) {
    const int l = fwd ? kk + 1 : levels - kk;  // level l: region (d, h, w) >> (l - 1)
    Lvl3 q{};
    q.batch = in->batch;
    q.d = in->d >> (l - 1);
    q.h = in->h >> (l - 1);
    q.w = in->w >> (l - 1);
    q.coef = coef->ptr;
    q.c_bs = coef->batch_stride;
    q.c_zs = coef->plane_stride;
    q.c_rs = coef->row_stride;
    int t_io, t_low;
    if (l == 1) {
      q.io = img->ptr;
      q.i_bs = img->batch_stride;
      q.i_zs = img->plane_stride;
      q.i_rs = img->row_stride;
      t_io = img->dtype;
    } else {
      q.io = wsb + off[l - 1];
      q.i_rs = q.w;
      q.i_zs = q.h * q.w;
      q.i_bs = q.d * q.h * q.w;
      t_io = acc;
    }
    if (l == levels) {
      q.low = coef->ptr;
      q.l_bs = coef->batch_stride;
      q.l_zs = coef->plane_stride;
      q.l_rs = coef->row_stride;
      t_low = coef->dtype;
    } else {
      q.low = wsb + off[l];
      q.l_rs = q.w >> 1;
      q.l_zs = (q.h >> 1) * (q.w >> 1);
      q.l_bs = (q.d >> 1) * (q.h >> 1) * (q.w >> 1);
      t_low = acc;
    }
    const cudaError_t e = fwd ? dispatch3d_gen(true, t_io, coef->dtype, t_low, q, st)
                              : dispatch3d_gen(false, t_low, coef->dtype, t_io, q, st);
    if (e != cudaSuccess) {
      set_last_cuda_error((int)e);
      return HAAR_ECUDA;
    }
  }
  return HAAR_OK;
}

int run3(const haar_desc3* in, const haar_desc3* out, int levels, void* ws, size_t ws_bytes,
         void* stream, bool fwd) {
  int rc = check3(in);
  if (!rc) rc = check3(out);
  if (rc) return rc;
  if (levels < 1 || levels > 30) return HAAR_EINVAL;
  if (in->batch != out->batch || in->d != out->d || in->h != out->h || in->w != out->w)
    return HAAR_EINVAL;
  const int64_t m = ((int64_t)1 << levels) - 1;
  if ((in->d & m) || (in->h & m) || (in->w & m)) return HAAR_ESHAPE;
  const int tin = in->dtype, tout = out->dtype;
  if ((tin == HAAR_F64) != (tout == HAAR_F64) || (tin != tout && tin != HAAR_F32 && tout != HAAR_F32))
    return HAAR_EDTYPE;
  if (in->batch == 0 || in->d == 0 || in->h == 0 || in->w == 0) return HAAR_OK;
  const int si = dt_size(tin), so = dt_size(tout);
  {
    const uintptr_t a0 = (uintptr_t)in->ptr, a1 = a0 + (uintptr_t)extent3(in) * si;
    const uintptr_t b0 = (uintptr_t)out->ptr, b1 = b0 + (uintptr_t)extent3(out) * so;
    if (a0 < b1 && b0 < a1) return HAAR_EALIAS;
  }
  if (!tiled3_ok(in, out, levels)) return run_gen3(in, out, levels, ws, ws_bytes, stream, fwd);
  int lv[64], cum[65];
  const int np = plan_passes3(levels, lv, cum);
  size_t off[64];
  const size_t need = ws3(in, levels, off);
  if (need && (!ws || ws_bytes < need || ((uintptr_t)ws & 255))) return HAAR_EWORKSPACE;
  const int acc = tin == HAAR_F64 ? HAAR_F64 : HAAR_F32;
  char* wsb = static_cast<char*>(ws);
  const cudaStream_t st = (cudaStream_t)stream;
  for (int kk = 0; kk < np; ++kk) {
    const int k = fwd ? kk : np - 1 - kk;
    const int s0 = cum[k], s1 = cum[k + 1];
    const int64_t dk = in->d >> s0, hk = in->h >> s0, wk = in->w >> s0;
    Pass3 p{};
    p.levels = lv[k];
    p.batch = in->batch;
    p.d = dk;
    p.h = hk;
    p.w = wk;
    int ptin, ptout;
    const haar_desc3* coef = fwd ? out : in;
    if (fwd) {
      if (k == 0) {
        p.src = in->ptr; p.s_bs = in->batch_stride; p.s_zs = in->plane_stride; p.s_rs = in->row_stride;
        ptin = tin;
      } else {
        p.src = wsb + off[k]; p.s_rs = wk; p.s_zs = hk * wk; p.s_bs = dk * hk * wk;
        ptin = acc;
      }
      p.dst = out->ptr; p.d_bs = out->batch_stride; p.d_zs = out->plane_stride; p.d_rs = out->row_stride;
      ptout = tout;
    } else {
      p.src = in->ptr; p.s_bs = in->batch_stride; p.s_zs = in->plane_stride; p.s_rs = in->row_stride;
      ptin = tin;
      if (k == 0) {
        p.dst = out->ptr; p.d_bs = out->batch_stride; p.d_zs = out->plane_stride; p.d_rs = out->row_stride;
        ptout = tout;
      } else {
        p.dst = wsb + off[k]; p.d_rs = wk; p.d_zs = hk * wk; p.d_bs = dk * hk * wk;
        ptout = acc;
      }
    }
    if (k == np - 1) {
      p.ll = coef->ptr; p.l_bs = coef->batch_stride; p.l_zs = coef->plane_stride; p.l_rs = coef->row_stride;
      p.ll_acc = 0;
    } else {
      const int64_t d1 = in->d >> s1, h1 = in->h >> s1, w1 = in->w >> s1;
      p.ll = wsb + off[k + 1]; p.l_rs = w1; p.l_zs = h1 * w1; p.l_bs = d1 * h1 * w1;
      p.ll_acc = 1;
    }
    {
      auto a16 = [](const void* ptr) { return (uintptr_t)ptr % 16 == 0; };
      p.vec4 = ptin == HAAR_F32 && ptout == HAAR_F32 && wk % 32 == 0 && a16(p.src) &&
               a16(p.dst) && a16(p.ll) && p.s_bs % 4 == 0 && p.s_zs % 4 == 0 &&
               p.s_rs % 4 == 0 && p.d_bs % 4 == 0 && p.d_zs % 4 == 0 && p.d_rs % 4 == 0 &&
               p.l_bs % 4 == 0 && p.l_zs % 4 == 0 && p.l_rs % 4 == 0;
    }
    const cudaError_t e = dispatch3d(fwd, ptin, ptout, p, st);
    if (e != cudaSuccess) {
      set_last_cuda_error((int)e);
      return HAAR_ECUDA;
    }
  }
  return HAAR_OK;
}

}  // namespace

extern "C" {

int haar_workspace_size_3d(const haar_desc3* x, int levels, size_t* bytes) {
  if (!bytes) return HAAR_EINVAL;
  *bytes = 0;
  const int rc = check3(x);
  if (rc) return rc;
  if (levels < 1 || levels > 30) return HAAR_EINVAL;
  size_t off[64];
  *bytes = tiled3_ok(x, x, levels) ? ws3(x, levels, off) : ws_gen3(x, levels, off);
  return HAAR_OK;
}

int haar_dwt_3d(const haar_desc3* x, const haar_desc3* coef, int levels, void* workspace,
                size_t workspace_bytes, void* cuda_stream) {
  return run3(x, coef, levels, workspace, workspace_bytes, cuda_stream, true);
}

int haar_idwt_3d(const haar_desc3* coef, const haar_desc3* x, int levels, void* workspace,
                 size_t workspace_bytes, void* cuda_stream) {
  return run3(coef, x, levels, workspace, workspace_bytes, cuda_stream, false);
}

}  // extern "C"
