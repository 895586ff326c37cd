/*
 * cpu_baseline.c -- TEST INFRASTRUCTURE ONLY: a CPU baseline, not the oracle.
 *
 * The Fast Haar method itself (the polyphase analysis and synthesis of
 * Section III, Fig. 4 and Section IV, Eq. 19, applied along rows and
 * columns) written as a plain single-threaded FP32 loop, for the
 * benchmark's CPU baseline: a fairer CPU reference than the FP64 oracle,
 * which computes the bank by its definition (full convolutions, then
 * decimation).  Only the benchmark's CPU-baseline leg and the tests load it;
 * the CUDA library never does and shares nothing with it.
 *
 * Per level, every 2 x 2 block [[a, b], [c, d]] of the current low band
 * gives its four coefficients directly:
 *     LL = (a+b+c+d)/2   Hx = (b-a+d-c)/2   Hy = (c+d-a-b)/2   HH = (a-b-c+d)/2
 * (the bank along the rows, then along the columns, with s*s = 1/2), in the
 * Mallat layout [LL | Hx] over [Hy | HH]; the synthesis inverts each block.
 * Arrays are contiguous row-major float; h and w divisible by 2^levels.
 * work must hold h*w/2 floats.  Returns 0, or -1 on a bad argument.
 */
#include <stddef.h>
#include <string.h>

static int check(long h, long w, int levels) {
  if (h <= 0 || w <= 0 || levels < 1 || levels > 30) return -1;
  if ((h % (1L << levels)) != 0 || (w % (1L << levels)) != 0) return -1;
  return 0;
}

int cpu_fast_haar_dwt2d_f32(const float* x, long h, long w, int levels, float* coef,
                            float* work) {
  if (check(h, w, levels)) return -1;
  /* the low band of level l lives in work (two halves, alternating) */
  float* buf[2] = {work, work + (h / 2) * (w / 2)};
  const float* src = x;
  long src_rs = w;
  for (int l = 0; l < levels; ++l) {
    const long hl = h >> l, wl = w >> l, h2 = hl / 2, w2 = wl / 2;
    float* low = buf[l & 1];
    for (long i = 0; i < h2; ++i) {
      const float* r0 = src + (2 * i) * src_rs;
      const float* r1 = r0 + src_rs;
      float* hx = coef + i * w + w2;
      float* hy = coef + (h2 + i) * w;
      float* hh = coef + (h2 + i) * w + w2;
      float* lo = low + i * w2;
      for (long j = 0; j < w2; ++j) {
        const float a = r0[2 * j], b = r0[2 * j + 1], c = r1[2 * j], d = r1[2 * j + 1];
        const float p = a + b, q = c + d, r = b - a, t = d - c;
        lo[j] = (p + q) * 0.5f;
        hy[j] = (q - p) * 0.5f;
        hx[j] = (r + t) * 0.5f;
        hh[j] = (t - r) * 0.5f;
      }
    }
    src = low;
    src_rs = w2;
  }
  const long hL = h >> levels, wL = w >> levels;
  for (long i = 0; i < hL; ++i) memcpy(coef + i * w, src + i * wL, (size_t)wL * sizeof(float));
  return 0;
}

int cpu_fast_haar_idwt2d_f32(const float* coef, long h, long w, int levels, float* x,
                             float* work) {
  if (check(h, w, levels)) return -1;
  float* buf[2] = {work, work + (h / 2) * (w / 2)};
  const long hL = h >> levels, wL = w >> levels;
  /* start from LL_L, copied out of the coefficient array */
  float* low = buf[levels & 1];
  for (long i = 0; i < hL; ++i) memcpy(low + i * wL, coef + i * w, (size_t)wL * sizeof(float));
  for (int l = levels - 1; l >= 0; --l) {
    const long hl = h >> l, wl = w >> l, h2 = hl / 2, w2 = wl / 2;
    float* out = l == 0 ? x : buf[l & 1];
    const long out_rs = l == 0 ? w : wl;
    for (long i = 0; i < h2; ++i) {
      const float* hx = coef + i * w + w2;
      const float* hy = coef + (h2 + i) * w;
      const float* hh = coef + (h2 + i) * w + w2;
      const float* lo = low + i * w2;
      float* r0 = out + (2 * i) * out_rs;
      float* r1 = r0 + out_rs;
      for (long j = 0; j < w2; ++j) {
        const float s1 = lo[j] - hy[j], s2 = hx[j] - hh[j];
        const float t1 = lo[j] + hy[j], t2 = hx[j] + hh[j];
        r0[2 * j] = (s1 - s2) * 0.5f;
        r0[2 * j + 1] = (s1 + s2) * 0.5f;
        r1[2 * j] = (t1 - t2) * 0.5f;
        r1[2 * j + 1] = (t1 + t2) * 0.5f;
      }
    }
    low = out;
  }
  return 0;
}
