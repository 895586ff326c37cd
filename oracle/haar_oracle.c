/*
 * haar_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow FP64 CPU oracle of the Haar two-channel filter bank of
 * "The Fast Haar Wavelet Transform for Signal & Image Processing"
 * (arXiv:1002.2184).  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load it; the CUDA library never does, and the
 * two share no source, header, table or helper.
 *
 * What it computes is the DEFINITION of the bank (Section II, Fig. 1):
 *   analysis  : full linear convolution of the input with b0 and b1, then
 *               keep every second output (decimation by 2);
 *   synthesis : upsample d0 and d1 by zero insertion, convolve with a0 and
 *               a1, add the two branches.
 * The polyphase "Fast Haar" form (Section III, Eq. 8-12, Fig. 4; Section IV,
 * Eq. 17-19, Fig. 7) is what the GPU computes.  Here it appears only as the
 * separate pair of routines oracle_polyphase_*, used to reproduce the
 * paper's "existing vs. fast" comparison (Section V) on synthetic data.
 *
 * Readings of the paper (it is ambiguous on these points):
 *  - Causal convolution y[k] = sum_j f[j] x[k-j].  Taps, with s = 1/sqrt(2):
 *        b0 = a0 = [ s,  s ]
 *        b1      = [ s, -s ]   (high pass of Eq. 9:  B00(z^2) - z^-1 B01(z^2))
 *        a1      = [-s,  s ]   (high pass of Eq. 18: -A00(z^2) + z^-1 A01(z^2))
 *    With these, d1[n] = (x[2n+1] - x[2n]) / sqrt(2).  detail_sign = -1
 *    negates b1 and a1, which is the Section II taps read as causal
 *    convolution taps; that is also a perfect-reconstruction bank.
 *  - Decimation keeps the odd-index convolution outputs, d_i[n] = y_i[2n+1],
 *    so each output pairs (x[2n], x[2n+1]) with zero delay.  Synthesis puts
 *    d_i[n] at even positions 2n and truncates the sum to the input length.
 *  - Orthonormal taps: no factor 1/2 (Eq. 1-4) or 2 (Eq. 14-15) is applied.
 *  - Multi-level (Mallat): the bank is re-applied to the low band.  1D
 *    layout [a_L | d_L | d_{L-1} | ... | d_1].  2D: at each level, every row
 *    of the current LL region is analysed (low half left, high half right),
 *    then every column (low half top, high half bottom), giving quadrants
 *        [ LL | Hx ]      Hx: high along width,  low along height
 *        [ Hy | HH ]      Hy: low along width,   high along height
 *    The paper only says wavelets decompose hierarchically (Section I) and
 *    shows a 2D low-pass image (Section V); the layout is this convention.
 *  - Sizes must be divisible by 2^levels; there is no boundary extension.
 *
 * All arrays are contiguous, row-major double.  Every function returns 0 on
 * success and -1 on a bad argument or a failed allocation.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

static const double S = 0.70710678118654752440; /* 1/sqrt(2) */

/* Filter taps of the bank (Section II, read as above). */
static void taps(int detail_sign, double b0[2], double b1[2], double a0[2],
                 double a1[2]) {
  double g = detail_sign < 0 ? -1.0 : 1.0;
  b0[0] = S;       b0[1] = S;
  b1[0] = g * S;   b1[1] = -g * S;
  a0[0] = S;       a0[1] = S;
  a1[0] = -g * S;  a1[1] = g * S;
}

/* Full linear convolution: y has n + nf - 1 samples. */
static void conv_full(const double *x, long n, const double *f, int nf,
                      double *y) {
  for (long k = 0; k < n + nf - 1; ++k) {
    double acc = 0.0;
    for (int j = 0; j < nf; ++j) {
      long i = k - j;
      if (i >= 0 && i < n) acc += f[j] * x[i];
    }
    y[k] = acc;
  }
}

static int is_pow2_divisible(long n, int levels) {
  if (levels < 0 || levels > 62 || n < 0) return 0;
  return (n % (1L << levels)) == 0;
}

/* One analysis stage (Fig. 1, left half): convolve with b0 and b1, then
 * decimate by 2.  x has n (even) samples; lo and hi get n/2 each. */
int oracle_analysis_1d(const double *x, long n, double *lo, double *hi,
                       int detail_sign) {
  if (n < 0 || n % 2 != 0) return -1;
  if (n == 0) return 0;
  double b0[2], b1[2], a0[2], a1[2];
  taps(detail_sign, b0, b1, a0, a1);
  double *y0 = malloc(sizeof(double) * (size_t)(n + 1));
  double *y1 = malloc(sizeof(double) * (size_t)(n + 1));
  if (!y0 || !y1) { free(y0); free(y1); return -1; }
  conv_full(x, n, b0, 2, y0);
  conv_full(x, n, b1, 2, y1);
  for (long m = 0; m < n / 2; ++m) {
    lo[m] = y0[2 * m + 1];
    hi[m] = y1[2 * m + 1];
  }
  free(y0);
  free(y1);
  return 0;
}

/* One synthesis stage (Fig. 1, right half, Eq. 13): upsample lo and hi by 2
 * (zero insertion), convolve with a0 and a1, add.  x gets 2m samples. */
int oracle_synthesis_1d(const double *lo, const double *hi, long m, double *x,
                        int detail_sign) {
  if (m < 0) return -1;
  if (m == 0) return 0;
  long n = 2 * m;
  double b0[2], b1[2], a0[2], a1[2];
  taps(detail_sign, b0, b1, a0, a1);
  double *u0 = calloc((size_t)n, sizeof(double));
  double *u1 = calloc((size_t)n, sizeof(double));
  double *y0 = malloc(sizeof(double) * (size_t)(n + 1));
  double *y1 = malloc(sizeof(double) * (size_t)(n + 1));
  if (!u0 || !u1 || !y0 || !y1) {
    free(u0); free(u1); free(y0); free(y1);
    return -1;
  }
  for (long k = 0; k < m; ++k) {
    u0[2 * k] = lo[k];
    u1[2 * k] = hi[k];
  }
  conv_full(u0, n, a0, 2, y0);
  conv_full(u1, n, a1, 2, y1);
  for (long k = 0; k < n; ++k) x[k] = y0[k] + y1[k];
  free(u0); free(u1); free(y0); free(y1);
  return 0;
}

/* The Fast Haar analysis bank (Fig. 4): the down-sampler sits at the input,
 * so the even and odd phases are taken first and combined with the single
 * polyphase tap b00 = 1/sqrt(2) (Eq. 11-12).  Used only for the
 * "existing vs. fast" comparison. */
int oracle_polyphase_analysis_1d(const double *x, long n, double *lo,
                                 double *hi, int detail_sign) {
  if (n < 0 || n % 2 != 0) return -1;
  double g = detail_sign < 0 ? -1.0 : 1.0;
  const double b00 = S;
  for (long m = 0; m < n / 2; ++m) {
    double even = x[2 * m], odd = x[2 * m + 1];
    lo[m] = b00 * (even + odd);
    hi[m] = g * b00 * (odd - even);
  }
  return 0;
}

/* The Fast Haar synthesis bank (Eq. 19, Fig. 7): difference and sum of the
 * two bands, scaled by a00 = a01 = 1/sqrt(2), interleaved at the output. */
int oracle_polyphase_synthesis_1d(const double *lo, const double *hi, long m,
                                  double *x, int detail_sign) {
  if (m < 0) return -1;
  double g = detail_sign < 0 ? -1.0 : 1.0;
  const double a00 = S, a01 = S;
  for (long k = 0; k < m; ++k) {
    double d0 = lo[k], d1 = g * hi[k];
    x[2 * k] = a00 * (d0 - d1);
    x[2 * k + 1] = a01 * (d0 + d1);
  }
  return 0;
}

/* Multi-level 1D analysis, Mallat layout [a_L | d_L | ... | d_1]. */
int oracle_dwt_1d(const double *x, long n, int levels, double *out,
                  int detail_sign) {
  if (!is_pow2_divisible(n, levels)) return -1;
  if (n == 0) return 0;
  double *a = malloc(sizeof(double) * (size_t)n);
  double *lo = malloc(sizeof(double) * (size_t)n);
  if (!a || !lo) { free(a); free(lo); return -1; }
  memcpy(a, x, sizeof(double) * (size_t)n);
  long len = n;
  for (int l = 1; l <= levels; ++l) {
    /* the detail of this level goes to out[len/2 : len] */
    if (oracle_analysis_1d(a, len, lo, out + len / 2, detail_sign) != 0) {
      free(a); free(lo);
      return -1;
    }
    len /= 2;
    memcpy(a, lo, sizeof(double) * (size_t)len);
  }
  memcpy(out, a, sizeof(double) * (size_t)len);
  free(a);
  free(lo);
  return 0;
}

/* Multi-level 1D synthesis: coarsest level first. */
int oracle_idwt_1d(const double *c, long n, int levels, double *out,
                   int detail_sign) {
  if (!is_pow2_divisible(n, levels)) return -1;
  if (n == 0) return 0;
  double *a = malloc(sizeof(double) * (size_t)n);
  double *next = malloc(sizeof(double) * (size_t)n);
  if (!a || !next) { free(a); free(next); return -1; }
  long len = n >> levels;
  memcpy(a, c, sizeof(double) * (size_t)len);
  for (int l = levels; l >= 1; --l) {
    /* a holds a_l (len samples); the detail d_l sits at c[len : 2 len] */
    if (oracle_synthesis_1d(a, c + len, len, next, detail_sign) != 0) {
      free(a); free(next);
      return -1;
    }
    len *= 2;
    memcpy(a, next, sizeof(double) * (size_t)len);
  }
  memcpy(out, a, sizeof(double) * (size_t)n);
  free(a);
  free(next);
  return 0;
}

/* Multi-level separable 2D analysis (rows, then columns, per level) of an
 * h x w image, Mallat quadrant layout. */
int oracle_dwt_2d(const double *x, long h, long w, int levels, double *out,
                  int detail_sign) {
  if (!is_pow2_divisible(h, levels) || !is_pow2_divisible(w, levels))
    return -1;
  if (h == 0 || w == 0) return 0;
  long big = h > w ? h : w;
  double *line = malloc(sizeof(double) * (size_t)big);
  double *lo = malloc(sizeof(double) * (size_t)big);
  double *hi = malloc(sizeof(double) * (size_t)big);
  if (!line || !lo || !hi) { free(line); free(lo); free(hi); return -1; }
  memcpy(out, x, sizeof(double) * (size_t)(h * w));
  for (int l = 1; l <= levels; ++l) {
    long hl = h >> (l - 1), wl = w >> (l - 1);
    for (long r = 0; r < hl; ++r) { /* every row of the current LL region */
      double *row = out + r * w;
      if (oracle_analysis_1d(row, wl, lo, hi, detail_sign) != 0) goto fail;
      memcpy(row, lo, sizeof(double) * (size_t)(wl / 2));
      memcpy(row + wl / 2, hi, sizeof(double) * (size_t)(wl / 2));
    }
    for (long c = 0; c < wl; ++c) { /* then every column */
      for (long r = 0; r < hl; ++r) line[r] = out[r * w + c];
      if (oracle_analysis_1d(line, hl, lo, hi, detail_sign) != 0) goto fail;
      for (long r = 0; r < hl / 2; ++r) {
        out[r * w + c] = lo[r];
        out[(r + hl / 2) * w + c] = hi[r];
      }
    }
  }
  free(line); free(lo); free(hi);
  return 0;
fail:
  free(line); free(lo); free(hi);
  return -1;
}

/* Multi-level separable 2D synthesis: coarsest level first; within a level
 * the column pass is undone before the row pass. */
int oracle_idwt_2d(const double *c, long h, long w, int levels, double *out,
                   int detail_sign) {
  if (!is_pow2_divisible(h, levels) || !is_pow2_divisible(w, levels))
    return -1;
  if (h == 0 || w == 0) return 0;
  long big = h > w ? h : w;
  double *line = malloc(sizeof(double) * (size_t)big);
  double *lo = malloc(sizeof(double) * (size_t)big);
  double *hi = malloc(sizeof(double) * (size_t)big);
  if (!line || !lo || !hi) { free(line); free(lo); free(hi); return -1; }
  memcpy(out, c, sizeof(double) * (size_t)(h * w));
  for (int l = levels; l >= 1; --l) {
    long hl = h >> (l - 1), wl = w >> (l - 1);
    for (long col = 0; col < wl; ++col) {
      for (long r = 0; r < hl / 2; ++r) {
        lo[r] = out[r * w + col];
        hi[r] = out[(r + hl / 2) * w + col];
      }
      if (oracle_synthesis_1d(lo, hi, hl / 2, line, detail_sign) != 0)
        goto fail;
      for (long r = 0; r < hl; ++r) out[r * w + col] = line[r];
    }
    for (long r = 0; r < hl; ++r) {
      double *row = out + r * w;
      memcpy(lo, row, sizeof(double) * (size_t)(wl / 2));
      memcpy(hi, row + wl / 2, sizeof(double) * (size_t)(wl / 2));
      if (oracle_synthesis_1d(lo, hi, wl / 2, row, detail_sign) != 0)
        goto fail;
    }
  }
  free(line); free(lo); free(hi);
  return 0;
fail:
  free(line); free(lo); free(hi);
  return -1;
}

/* Multi-level separable 3D analysis of a d x h x w volume (index
 * (z * h + y) * w + x): per level, on the current low-pass region, the
 * analysis stage along x for every (z, y) line, then along y for every
 * (z, x) line, then along z for every (y, x) line; each splits the region
 * into low (first half) and high (second half).  The same recursion as the
 * 2D transform, with a third axis; not in the paper. */
int oracle_dwt_3d(const double *x, long d, long h, long w, int levels, double *out,
                  int detail_sign) {
  if (!is_pow2_divisible(d, levels) || !is_pow2_divisible(h, levels) ||
      !is_pow2_divisible(w, levels))
    return -1;
  if (d == 0 || h == 0 || w == 0) return 0;
  long big = d > h ? d : h;
  big = big > w ? big : w;
  double *line = malloc(sizeof(double) * (size_t)big);
  double *lo = malloc(sizeof(double) * (size_t)big);
  double *hi = malloc(sizeof(double) * (size_t)big);
  if (!line || !lo || !hi) { free(line); free(lo); free(hi); return -1; }
  memcpy(out, x, sizeof(double) * (size_t)(d * h * w));
#define AT(z, y, xx) out[((z) * h + (y)) * w + (xx)]
  for (int l = 1; l <= levels; ++l) {
    long dl = d >> (l - 1), hl = h >> (l - 1), wl = w >> (l - 1);
    for (long z = 0; z < dl; ++z)
      for (long y = 0; y < hl; ++y) {
        for (long i = 0; i < wl; ++i) line[i] = AT(z, y, i);
        if (oracle_analysis_1d(line, wl, lo, hi, detail_sign) != 0) goto fail3;
        for (long i = 0; i < wl / 2; ++i) { AT(z, y, i) = lo[i]; AT(z, y, i + wl / 2) = hi[i]; }
      }
    for (long z = 0; z < dl; ++z)
      for (long xx = 0; xx < wl; ++xx) {
        for (long i = 0; i < hl; ++i) line[i] = AT(z, i, xx);
        if (oracle_analysis_1d(line, hl, lo, hi, detail_sign) != 0) goto fail3;
        for (long i = 0; i < hl / 2; ++i) { AT(z, i, xx) = lo[i]; AT(z, i + hl / 2, xx) = hi[i]; }
      }
    for (long y = 0; y < hl; ++y)
      for (long xx = 0; xx < wl; ++xx) {
        for (long i = 0; i < dl; ++i) line[i] = AT(i, y, xx);
        if (oracle_analysis_1d(line, dl, lo, hi, detail_sign) != 0) goto fail3;
        for (long i = 0; i < dl / 2; ++i) { AT(i, y, xx) = lo[i]; AT(i + dl / 2, y, xx) = hi[i]; }
      }
  }
  free(line); free(lo); free(hi);
  return 0;
fail3:
  free(line); free(lo); free(hi);
  return -1;
}

/* Multi-level 3D synthesis: coarsest level first; within a level the z, y
 * and x stages are undone in that order. */
int oracle_idwt_3d(const double *c, long d, long h, long w, int levels, double *out,
                   int detail_sign) {
  if (!is_pow2_divisible(d, levels) || !is_pow2_divisible(h, levels) ||
      !is_pow2_divisible(w, levels))
    return -1;
  if (d == 0 || h == 0 || w == 0) return 0;
  long big = d > h ? d : h;
  big = big > w ? big : w;
  double *line = malloc(sizeof(double) * (size_t)big);
  double *lo = malloc(sizeof(double) * (size_t)big);
  double *hi = malloc(sizeof(double) * (size_t)big);
  if (!line || !lo || !hi) { free(line); free(lo); free(hi); return -1; }
  memcpy(out, c, sizeof(double) * (size_t)(d * h * w));
  for (int l = levels; l >= 1; --l) {
    long dl = d >> (l - 1), hl = h >> (l - 1), wl = w >> (l - 1);
    for (long y = 0; y < hl; ++y)
      for (long xx = 0; xx < wl; ++xx) {
        for (long i = 0; i < dl / 2; ++i) { lo[i] = AT(i, y, xx); hi[i] = AT(i + dl / 2, y, xx); }
        if (oracle_synthesis_1d(lo, hi, dl / 2, line, detail_sign) != 0) goto fail4;
        for (long i = 0; i < dl; ++i) AT(i, y, xx) = line[i];
      }
    for (long z = 0; z < dl; ++z)
      for (long xx = 0; xx < wl; ++xx) {
        for (long i = 0; i < hl / 2; ++i) { lo[i] = AT(z, i, xx); hi[i] = AT(z, i + hl / 2, xx); }
        if (oracle_synthesis_1d(lo, hi, hl / 2, line, detail_sign) != 0) goto fail4;
        for (long i = 0; i < hl; ++i) AT(z, i, xx) = line[i];
      }
    for (long z = 0; z < dl; ++z)
      for (long y = 0; y < hl; ++y) {
        for (long i = 0; i < wl / 2; ++i) { lo[i] = AT(z, y, i); hi[i] = AT(z, y, i + wl / 2); }
        if (oracle_synthesis_1d(lo, hi, wl / 2, line, detail_sign) != 0) goto fail4;
        for (long i = 0; i < wl; ++i) AT(z, y, i) = line[i];
      }
  }
#undef AT
  free(line); free(lo); free(hi);
  return 0;
fail4:
  free(line); free(lo); free(hi);
  return -1;
}
