/*
 * fasthaar.h -- C ABI of the GB300 Fast Haar wavelet transform library
 * (libfasthaar.so).
 *
 * The transform is the two-channel Haar filter bank of arXiv:1002.2184 in
 * its polyphase ("Fast Haar") form: the down-sampler is moved in front of the
 * filters (Section III, Eq. 8-12, Fig. 4) and the up-sampler behind them
 * (Section IV, Eq. 17-19, Fig. 7), so each output pair is formed directly
 * from one input pair and no decimated sample is ever computed:
 *
 *   analysis   d0[n] = (x[2n] + x[2n+1]) / sqrt(2)
 *              d1[n] = (x[2n+1] - x[2n]) / sqrt(2)        (sign of Eq. 9)
 *   synthesis  x[2n]   = (d0[n] - d1[n]) / sqrt(2)
 *              x[2n+1] = (d0[n] + d1[n]) / sqrt(2)        (Eq. 19, Fig. 8)
 *
 * Multi-level transforms re-apply the bank to the low band (the paper's
 * hierarchical decomposition, Section I) and store the result in the Mallat
 * layout, with the same shape as the input:
 *   1D: [a_L | d_L | d_{L-1} | ... | d_1] along each row;
 *   2D: per level, rows then columns on the current LL region, quadrants
 *       [LL | Hx] over [Hy | HH] (Hx: high pass along the width, low pass
 *       along the height; Hy the reverse).  On one 2x2 block [[a, b], [c, d]]
 *       this is LL = (a+b+c+d)/2, Hx = (b-a+d-c)/2, Hy = (c+d-a-b)/2,
 *       HH = (a-b-c+d)/2.
 *
 * Conventions shared by every entry point:
 *  - All data pointers are DEVICE pointers owned by the caller; the library
 *    allocates no device memory.  Where a call needs scratch space it takes a
 *    caller-provided workspace (size from haar_workspace_size).
 *  - Calls are asynchronous on the given CUDA stream (NULL = legacy default
 *    stream); they never synchronise the device and may be captured into a
 *    CUDA graph.
 *  - Transforms are out of place.  Input and output ranges that overlap are
 *    rejected with HAAR_EALIAS.
 *  - Arithmetic is FP32 for fp32 / bf16 / fp16 / uint8 storage and FP64 for
 *    fp64 storage.  Outputs are rounded to nearest-even into the output type.
 *  - Extents must be divisible by 2^levels (no boundary extension): Haar
 *    pairs never overlap, so none is needed.
 *  - Errors are returned as negative status codes; nothing aborts, traps or
 *    prints.  A CUDA error is returned as HAAR_ECUDA and its code is kept for
 *    haar_last_cuda_error() (per host thread).
 */
#ifndef FASTHAAR_H
#define FASTHAAR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FASTHAAR_VERSION 1

/* Status codes. */
enum {
  HAAR_OK = 0,
  HAAR_EINVAL = -1,     /* null pointer, bad level count, negative extent or stride,
                           mismatched shapes, nonzero reserved field */
  HAAR_ESHAPE = -2,     /* a transformed extent is not divisible by 2^levels */
  HAAR_EDTYPE = -3,     /* dtype (or dtype pair) not supported by this entry point */
  HAAR_EALIAS = -4,     /* input and output memory ranges overlap */
  HAAR_ECUDA = -5,      /* a CUDA runtime call failed; see haar_last_cuda_error() */
  HAAR_ETIMEOUT = -6,   /* a bounded device-side wait gave up */
  HAAR_EWORKSPACE = -7, /* workspace missing or smaller than haar_workspace_size() */
  HAAR_EQUEUE = -8      /* a persistent launch found its work queue inconsistent */
};

/* Storage types.  uint8 is accepted as analysis input only (values 0..255
 * are transformed as they are, without scaling); fp64 pairs only with fp64
 * and exists for gradient checks. */
typedef enum {
  HAAR_F32 = 0,
  HAAR_BF16 = 1,
  HAAR_F16 = 2,
  HAAR_U8 = 3,
  HAAR_F64 = 4
} haar_dtype;

/* A strided batch of 2D arrays.  Element (b, y, x) lives at
 *   ptr + (b * batch_stride + y * row_stride + x) * sizeof(dtype).
 * Rows are contiguous (unit column stride).  Strides are in ELEMENTS, must be
 * non-negative, row_stride >= w when h > 1, and batch_stride must separate
 * the items (batch_stride >= (h - 1) * row_stride + w when batch > 1).
 * For 1D calls every row of every batch item is one independent signal of
 * length w.  Any of batch, h, w may be 0 (nothing is done). */
typedef struct {
  void *ptr;
  int32_t dtype;    /* haar_dtype */
  int32_t reserved; /* must be 0 */
  int64_t batch;
  int64_t h;
  int64_t w;
  int64_t batch_stride;
  int64_t row_stride;
} haar_desc;

/* Operation codes for haar_workspace_size. */
enum { HAAR_OP_DWT_1D = 0, HAAR_OP_IDWT_1D = 1, HAAR_OP_DWT_2D = 2, HAAR_OP_IDWT_2D = 3 };

/* Bytes of workspace the operation needs for this input descriptor and
 * level count (0 when every level fuses into one kernel launch: up to 6
 * levels in 2D, 12 in 1D).  Writes *bytes; returns a status. */
int haar_workspace_size(int op, const haar_desc *src, int levels, size_t *bytes);

/* 1D multi-level analysis (Fig. 4 per level) of every row of x into coef
 * (Mallat layout along the row).  x and coef must have equal batch, h, w;
 * w divisible by 2^levels; 1 <= levels <= 62.
 * dtypes: x in {F32, BF16, F16, U8}, coef in {F32, BF16, F16}; or both F64.
 * workspace: device memory of at least haar_workspace_size(HAAR_OP_DWT_1D)
 * bytes (may be NULL when that size is 0), 256-byte aligned. */
int haar_dwt_1d(const haar_desc *x, const haar_desc *coef, int levels, void *workspace,
                size_t workspace_bytes, void *cuda_stream);

/* 1D multi-level synthesis (Eq. 19 per level, coarsest first): inverse of
 * haar_dwt_1d.  dtypes: coef and x in {F32, BF16, F16}; or both F64. */
int haar_idwt_1d(const haar_desc *coef, const haar_desc *x, int levels, void *workspace,
                 size_t workspace_bytes, void *cuda_stream);

/* 2D multi-level separable analysis of every h x w image of x into coef
 * (Mallat quadrant layout).  h and w divisible by 2^levels.  Up to 6 levels
 * run fused in one launch; deeper transforms chain launches through the
 * workspace.  dtypes as haar_dwt_1d. */
int haar_dwt_2d(const haar_desc *x, const haar_desc *coef, int levels, void *workspace,
                size_t workspace_bytes, void *cuda_stream);

/* 2D multi-level synthesis, coarsest level first: inverse of haar_dwt_2d.
 * dtypes as haar_idwt_1d. */
int haar_idwt_2d(const haar_desc *coef, const haar_desc *x, int levels, void *workspace,
                 size_t workspace_bytes, void *cuda_stream);

/* Same as haar_dwt_2d, for callers that cannot allocate device memory (for
 * example code running inside a host application that owns every
 * allocation, or a loop where calling the allocator is not allowed): the
 * scratch space that transforms deeper than six levels need is taken from a
 * fixed 4 MiB array built into the library instead of from the caller, and
 * the call allocates nothing.  The paper has no counterpart; this is an
 * interface convenience.
 *  - Every GPU that loads the library holds the 4 MiB array until exit.
 *  - A transform whose scratch (haar_workspace_size(HAAR_OP_DWT_2D, ...))
 *    exceeds 4 MiB is rejected with HAAR_EWORKSPACE; use haar_dwt_2d.
 *  - The first call on each device looks the array's address up
 *    (cudaGetSymbolAddress, with that device current) and keeps it for the
 *    life of the process; make that first call before any stream capture.
 *    Call it with the stream's device current.  Not supported on a device
 *    that has been reset (cudaDeviceReset) after that first call: the kept
 *    address would point at freed memory.
 *  - Argument errors are reported as by haar_dwt_2d (both descriptors are
 *    checked first); HAAR_EWORKSPACE only for a valid call whose scratch is
 *    too large.
 *  - All calls on a device share the one array and it keeps the last call's
 *    contents (nothing in it needs to start at zero).  Calls whose kernels
 *    overlap in time on the GPU (different streams, not ordered) race on the
 *    array and give wrong results: keep them on one stream or order them. */
int haar_dwt_2d_noalloc(const haar_desc *x, const haar_desc *coef, int levels,
                        void *cuda_stream);

/* ------------------------------------------------------------------------
 * 3D (volumes, video): the bank along x, then y, then z at every level, on
 * the current low-pass region (the 2D recursion with a third axis; not in
 * the paper, which treats signals and images).  Octant (bz, by, bx) of level
 * l -- b = 0 low, 1 high along that axis -- sits at (bz D_l/2, by H_l/2,
 * bx W_l/2) inside the level's region (D_l, H_l, W_l) = (d, h, w) / 2^(l-1).
 * ---------------------------------------------------------------------- */
typedef struct {
  void *ptr;
  int32_t dtype;     /* haar_dtype: F32, BF16, F16 or F64 */
  int32_t reserved;  /* must be 0 */
  int64_t batch, d, h, w;
  int64_t batch_stride, plane_stride, row_stride; /* elements */
} haar_desc3;

/* Workspace of a 3D transform: the tiled kernels need one for more than 3
 * levels (3 fuse per launch); volumes they cannot take (below) need the low
 * band of every level but the last (about 1/7 of the volume, accumulator
 * type).  The answer is for x's layout; a transform between two arrays needs
 * the larger of the answers for both descriptors. */
int haar_workspace_size_3d(const haar_desc3 *x, int levels, size_t *bytes);

/* 3D analysis / synthesis.  d, h, w divisible by 2^levels.  The tiled
 * kernels take volumes whose width at every pass of 3 levels is a multiple
 * of 8 and whose rows, planes and batch items are 16-byte aligned in both
 * arrays; any other volume runs a generic kernel per level (element by
 * element, same results).  dtypes: equal storage types, or F32 with
 * BF16/F16 (either direction); F64 only with F64. */
int haar_dwt_3d(const haar_desc3 *x, const haar_desc3 *coef, int levels, void *workspace,
                size_t workspace_bytes, void *cuda_stream);
int haar_idwt_3d(const haar_desc3 *coef, const haar_desc3 *x, int levels, void *workspace,
                 size_t workspace_bytes, void *cuda_stream);

/* ------------------------------------------------------------------------
 * Ragged batches: many 2D images of different sizes and level counts in one
 * persistent launch.  Images live anywhere inside one input buffer and one
 * output buffer (element offsets from the two base pointers); the output of
 * each image is its Mallat layout (analysis) or the image (synthesis).
 * ---------------------------------------------------------------------- */
typedef struct {
  int64_t in_offset;      /* elements from the input base pointer to pixel (0, 0) */
  int64_t out_offset;     /* elements from the output base pointer */
  int64_t h, w;           /* multiples of 32, divisible by 2^levels */
  int64_t in_row_stride;  /* elements; >= w */
  int64_t out_row_stride; /* elements; >= w */
  int32_t levels;         /* 1..6 */
  int32_t reserved;       /* must be 0 */
} haar_ragged_item;

/* Work-unit shape of the persistent kernel: 64 x 128 pixels (any level count)
 * or 32 x 256 pixels (every image at most 5 levels). */
enum { HAAR_UNIT_64x128 = 0, HAAR_UNIT_32x256 = 1 };

typedef struct haar_ragged_plan haar_ragged_plan; /* opaque, host memory */

/* Builds a plan (host only, no device call): validates every item, cuts each
 * image into work units and prepares the device image table.
 * blocks_per_sm: blocks per SM of the persistent grid (1..32); the grid is
 * min(units, blocks_per_sm * SM count of the device current at launch).
 * Errors: HAAR_EINVAL (bad item or argument), HAAR_ESHAPE (side not a
 * multiple of 32 or not divisible by 2^levels, or 6 levels with the
 * 32 x 256 unit).  On success *plan must be released with
 * haar_ragged_plan_destroy. */
int haar_ragged_plan_create(const haar_ragged_item *items, int64_t count, int unit,
                            int blocks_per_sm, haar_ragged_plan **plan);

/* Device workspace the plan needs (header + image table), in bytes. */
int haar_ragged_workspace_size(const haar_ragged_plan *plan, size_t *bytes);

/* Work units, pixels and the persistent grid size of a plan on the current
 * device (queries its SM count). */
int haar_ragged_plan_info(const haar_ragged_plan *plan, int64_t *units, int64_t *pixels,
                          int64_t *grid);

/* Copies the image table into the workspace and zeroes its counters
 * (asynchronous on the stream; the plan must outlive the copy).  Call once
 * per workspace, before the first transform (and before any graph capture). */
int haar_ragged_upload(const haar_ragged_plan *plan, void *workspace, size_t workspace_bytes,
                       void *cuda_stream);

/* One persistent launch transforming every image of the plan.  dtypes as
 * haar_dwt_2d / haar_idwt_2d.  The workspace must have been uploaded; the
 * kernel leaves its counters zeroed again, so the call can be repeated or
 * replayed from a CUDA graph.  Two calls on one workspace must not overlap in
 * time (same stream, or ordered by events). */
int haar_dwt_2d_ragged(const haar_ragged_plan *plan, const void *in, int in_dtype, void *out,
                       int out_dtype, void *workspace, size_t workspace_bytes, void *cuda_stream);
int haar_idwt_2d_ragged(const haar_ragged_plan *plan, const void *in, int in_dtype, void *out,
                        int out_dtype, void *workspace, size_t workspace_bytes,
                        void *cuda_stream);

/* Reads (synchronously: it waits for the stream) the workspace's error word:
 * *status = HAAR_OK, or HAAR_EQUEUE if a launch found its work queue in an
 * inconsistent state (the word is then cleared). */
int haar_ragged_status(const haar_ragged_plan *plan, void *workspace, int *status,
                       void *cuda_stream);

int haar_ragged_plan_destroy(haar_ragged_plan *plan);

/* ------------------------------------------------------------------------
 * Longer orthogonal filters through the same down-sample-first polyphase
 * identity (Section III, Eq. 7 states the split for a general filter): the
 * two-channel bank for an even-length orthonormal low-pass h[0..K-1],
 * K in {2, 4, 6, 8} (e.g. Daubechies-4), 1D, periodic boundary, multi-level
 * Mallat layout [a_L | d_L | ... | d_1]:
 *   a[n] = sum_k h[k] x[(2n+k) mod N],   d[n] = sum_k g[k] x[(2n+k) mod N],
 *   g[k] = (-1)^(k+1) h[K-1-k]   (K = 2 gives the Haar detail sign of Eq. 9).
 * Only the decimated outputs are computed.  x, coef: device pointers owned
 * by the caller, rows x n contiguous elements of the one type `dtype` (F32 or
 * F64, else HAAR_EDTYPE), not overlapping (HAAR_EALIAS); n divisible by
 * 2^levels (HAAR_ESHAPE); 1 <= levels <= 10, ntaps in {2, 4, 6, 8}, non-null
 * pointers (HAAR_EINVAL); `lowpass` is a
 * host array of ntaps doubles, read before the call returns (orthonormality
 * is the caller's to ensure).  Asynchronous on the stream; a launch failure
 * returns HAAR_ECUDA.  rows == 0 or n == 0 is a no-op. */
int haar_filter_dwt_1d(const void *x, void *coef, int dtype, int64_t rows, int64_t n, int levels,
                       const double *lowpass, int ntaps, void *cuda_stream);
int haar_filter_idwt_1d(const void *coef, void *x, int dtype, int64_t rows, int64_t n,
                        int levels, const double *lowpass, int ntaps, void *cuda_stream);

/* ------------------------------------------------------------------------
 * The undecimated (stationary) Haar transform, 1D: the bank of Section II,
 * Fig. 1 with the down-sampler removed -- every convolution output is kept,
 * the filters dilated by 2^(l-1) at level l (a trous), boundaries periodic:
 *   a_l[k] = (a_{l-1}[k] + a_{l-1}[k+s]) / sqrt(2),
 *   d_l[k] = (a_{l-1}[k+s] - a_{l-1}[k]) / sqrt(2),   s = 2^(l-1)
 * It is the direct form whose decimated outputs the Fast Haar bank never
 * computes: d_l[2^l m] and a_L[2^L m] are the decimated transform's
 * coefficients.  x: rows x n contiguous; coef: rows x (levels + 1) x n
 * contiguous, row 0 = a_L, row l = d_l; both device pointers owned by the
 * caller, of the one type `dtype` (F32 or F64, else HAAR_EDTYPE), not
 * overlapping (HAAR_EALIAS); 1 <= levels <= 10 and non-null pointers
 * (HAAR_EINVAL); n >= 2^levels (HAAR_ESHAPE: a dilated tap would wrap more
 * than once); rows == 0 or n == 0 is a no-op; asynchronous on the stream,
 * HAAR_ECUDA if the launch fails.  The inverse averages the two reconstructions of each
 * sample: a_{l-1}[k] = ((a_l[k] - d_l[k]) + (a_l[k-s] + d_l[k-s])) / (2 sqrt 2). */
int haar_swt_1d(const void *x, void *coef, int dtype, int64_t rows, int64_t n, int levels,
                void *cuda_stream);
int haar_iswt_1d(const void *coef, void *x, int dtype, int64_t rows, int64_t n, int levels,
                 void *cuda_stream);

/* ------------------------------------------------------------------------
 * Wavelet shrinkage in one pass (the paper's denoising use case for
 * biosignals and medical images, Section VI; the shrinkage rule is the
 * standard one, not the paper's): y = W^T shrink(W x), where every detail
 * coefficient d becomes sign(d) max(|d| - t, 0) (soft) or d [|d| > t]
 * (hard) and the low band is kept.  The coefficients never leave the
 * registers of the warp that owns the block: 1D, 256 samples per warp and up
 * to 8 levels (length a multiple of 256); 2D, 32 x 32 pixels per warp and up
 * to 5 levels (sides multiples of 32).  x and y: same shape, F32 or F64,
 * 16-byte aligned rows, not overlapping.
 * ---------------------------------------------------------------------- */
enum { HAAR_THRESH_SOFT = 0, HAAR_THRESH_HARD = 1 };

int haar_denoise_1d(const haar_desc *x, const haar_desc *y, int levels, double threshold,
                    int mode, void *cuda_stream);
int haar_denoise_2d(const haar_desc *x, const haar_desc *y, int levels, double threshold,
                    int mode, void *cuda_stream);

/* ------------------------------------------------------------------------
 * Verification reductions and a differentiable denoising loss built on the
 * transform (the paper has neither: they serve checking and training).  The
 * loss, for a contiguous batch of h x w images with an L-level transform W:
 *   c = W x,  s = soft(c, t) = sign(c) max(|c| - t, 0),  xr = W^T s,
 *   loss = mean((xr - x)^2) + l1_weight * mean(|s| over detail coefficients)
 * Its gradient uses W^-1 = W^T (orthonormal bank, Section II): the adjoint
 * of the analysis is the synthesis and vice versa.
 * Arrays: contiguous batches (batch_stride = h*w, row_stride = w), all of
 * one dtype, F32 or F64.
 * ---------------------------------------------------------------------- */

/* FP64 sums over n contiguous elements of a (and b, which may be NULL),
 * accumulated into out3 (device, 3 doubles): out3[0] += sum a^2,
 * out3[1] += sum (a-b)^2, out3[2] = max(out3[2], max |a-b|).  Any dtype. */
int haar_norms_f64(const void *a, const void *b, int dtype, int64_t n, double *out3,
                   void *cuda_stream);

/* s = soft(c, threshold) elementwise (any layout of the Mallat coefficients
 * of `levels` levels); l1_acc (device double, may be NULL) += sum of |s| over
 * the detail positions. */
int haar_soft_threshold(const haar_desc *c, const haar_desc *s, int levels, double threshold,
                        double *l1_acc, void *cuda_stream);

/* Adjoint of haar_soft_threshold with the L1 term: g_c = (g_s + l1_scale *
 * g_l1 * sign(s) * [detail]) * [s != 0]; g_l1 is a device scalar of the
 * dtype (NULL: no L1 term).  The subgradient at |c| <= threshold is 0. */
int haar_soft_threshold_backward(const haar_desc *g_s, const haar_desc *s, const haar_desc *g_c,
                                 int levels, double l1_scale, const void *g_l1,
                                 void *cuda_stream);

/* g_a = scale * g * (a - b) and g_b = -g_a (either output may be NULL; g is
 * a device scalar of the dtype, NULL meaning 1). */
int haar_sq_diff_backward(const haar_desc *a, const haar_desc *b, const haar_desc *g_a,
                          const haar_desc *g_b, double scale, const void *g,
                          void *cuda_stream);

/* The loss, fused into one launch plus a one-thread finisher, reading x only.
 * W is orthonormal, so the residual is r = W^T s - x = -W^T clamp(c, -t, t):
 * each warp takes its 32 x 32 block through the analysis, maps the
 * coefficients, and runs the synthesis back in registers; nothing but the
 * loss is written (to `loss`, a device scalar of the dtype).  acc2: device
 * scratch of 2 doubles, zero on entry and left zero on return.  Sides
 * multiples of 32, 1 <= levels <= 5, arrays 16-byte aligned (else
 * HAAR_ESHAPE / HAAR_EINVAL). */
int haar_denoise_forward(const haar_desc *x, int levels, double threshold, double l1_weight,
                         double *acc2, void *loss, void *cuda_stream);

/* Gradient of that loss with respect to x, recomputed from x alone, times
 * the upstream gradient g (device scalar of the dtype, NULL meaning 1):
 *   g_x = W^T q,  q = [|c| > t] * (l1_weight g / n_d) * sign(c) * [detail]
 *                   + [|c| <= t] * (2 g / n) * c,         c = W x
 * (n pixels, n_d detail coefficients), in one launch reading x and writing
 * g_x.  Same shape rules as haar_denoise_forward; x and g_x must not overlap. */
int haar_denoise_backward(const haar_desc *x, const haar_desc *g_x, int levels, double threshold,
                          double l1_weight, const void *g_loss, void *cuda_stream);

/* Human-readable name of a status code (static string, never NULL). */
const char *haar_status_string(int status);

/* The cudaError_t of the last HAAR_ECUDA returned on this host thread. */
int haar_last_cuda_error(void);

/* FASTHAAR_VERSION of the loaded library. */
int haar_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FASTHAAR_H */
