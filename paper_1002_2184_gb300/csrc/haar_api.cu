// haar_api.cu -- the C ABI (include/fasthaar.h): argument validation, the
// plan of fused passes for deep transforms, and dispatch to the launchers.
// Host code only; every step of the transform itself runs in the kernels.
#include <cuda_runtime.h>

#include <atomic>

#include "fasthaar.h"
#include "haar_internal.h"

using namespace fh;

namespace {

thread_local int g_last_cuda = 0;

int cuda_fail(cudaError_t e) {
  g_last_cuda = (int)e;
  return HAAR_ECUDA;
}

}  // namespace

void fh::set_last_cuda_error(int e) { g_last_cuda = e; }

namespace {

bool dtype_known(int dt) { return dt >= HAAR_F32 && dt <= HAAR_F64; }

int acc_dtype(int dt) { return dt == HAAR_F64 ? HAAR_F64 : HAAR_F32; }

bool is_empty(const haar_desc* d) { return d->batch == 0 || d->h == 0 || d->w == 0; }

constexpr int64_t kMaxExtent = (int64_t)1 << 56;

int check_desc(const haar_desc* d) {
  if (!d) return HAAR_EINVAL;
  if (d->reserved != 0) return HAAR_EINVAL;
  if (!dtype_known(d->dtype)) return HAAR_EDTYPE;
  if (d->batch < 0 || d->h < 0 || d->w < 0 || d->batch_stride < 0 || d->row_stride < 0)
    return HAAR_EINVAL;
  if (d->batch > kMaxExtent || d->h > kMaxExtent || d->w > kMaxExtent ||
      d->batch_stride > kMaxExtent || d->row_stride > kMaxExtent)
    return HAAR_EINVAL;
  if (is_empty(d)) return HAAR_OK;
  if (!d->ptr) return HAAR_EINVAL;
  if (d->h > 1 && d->row_stride < d->w) return HAAR_EINVAL;
  if (d->batch > 1) {
    const __int128 need = (__int128)(d->h - 1) * d->row_stride + d->w;
    if ((__int128)d->batch_stride < need) return HAAR_EINVAL;
  }
  const __int128 extent = (__int128)(d->batch - 1) * d->batch_stride +
                          (__int128)(d->h - 1) * d->row_stride + d->w;
  if (extent > (__int128)kMaxExtent) return HAAR_EINVAL;
  return HAAR_OK;
}

// [lo, hi) byte range touched by a descriptor.
void byte_range(const haar_desc* d, uintptr_t* lo, uintptr_t* hi) {
  const int64_t ext = (d->batch - 1) * d->batch_stride + (d->h - 1) * d->row_stride + d->w;
  *lo = (uintptr_t)d->ptr;
  *hi = *lo + (uintptr_t)ext * (uintptr_t)dt_size(d->dtype);
}

bool overlaps(const haar_desc* a, const haar_desc* b) {
  uintptr_t alo, ahi, blo, bhi;
  byte_range(a, &alo, &ahi);
  byte_range(b, &blo, &bhi);
  return alo < bhi && blo < ahi;
}

bool divisible(int64_t n, int levels) { return (n & (((int64_t)1 << levels) - 1)) == 0; }

bool fwd_pair_ok(int tin, int tout) {
  if (tin == HAAR_F64 || tout == HAAR_F64) return tin == HAAR_F64 && tout == HAAR_F64;
  return tout != HAAR_U8;
}

bool inv_pair_ok(int tin, int tout) {
  if (tin == HAAR_F64 || tout == HAAR_F64) return tin == HAAR_F64 && tout == HAAR_F64;
  return tin != HAAR_U8 && tout != HAAR_U8;
}

// ---------------------------------------------------------------------------
// Plan: the level count split into fused passes.
// ---------------------------------------------------------------------------
constexpr int kMaxPasses = 64;
constexpr int kMax2dFused = 6;
constexpr int kMax1dFused = 12;

struct Plan {
  int n = 0;
  int lv[kMaxPasses];
  int cum[kMaxPasses + 1];  // levels done before pass k
};

Plan make_plan(int levels, int max_fused) {
  Plan p;
  int done = 0;
  p.cum[0] = 0;
  while (done < levels) {
    const int l = levels - done < max_fused ? levels - done : max_fused;
    p.lv[p.n] = l;
    done += l;
    p.cum[p.n + 1] = done;
    ++p.n;
  }
  return p;
}

// Workspace region k (1 <= k < n) holds the LL band after cum[k] levels as
// a dense accumulator-typed batch.
struct Workspace {
  size_t off[kMaxPasses];
  size_t total;
};

inline size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

Workspace ws_layout(const Plan& pl, const haar_desc* d, bool two_d) {
  Workspace ws;
  ws.total = 0;
  const size_t esz = (size_t)dt_size(acc_dtype(d->dtype));
  for (int k = 1; k < pl.n; ++k) {
    const int s = pl.cum[k];
    const int64_t hk = two_d ? (d->h >> s) : d->h;
    const int64_t wk = d->w >> s;
    ws.off[k] = ws.total;
    ws.total += align256((size_t)d->batch * (size_t)hk * (size_t)wk * esz);
  }
  return ws;
}

int tile_for_levels(int lv) { return lv <= tile_max_levels(kT32x128) ? kT32x128 : kT64x128; }
int chunk_for_levels(int lv) { return lv <= chunk_max_levels(kC1024) ? kC1024 : kC4096; }

bool aligned(const void* p, int64_t bs, int64_t rs, int esz, int a) {
  return ((uintptr_t)p % (uintptr_t)a) == 0 && ((bs * esz) % a) == 0 && ((rs * esz) % a) == 0;
}

// Alignment the vector path needs: rows read/written 8 elements at a time on
// the image side and 4 at a time on the coefficient side.
int vec_align_img(int dt) { return dt == HAAR_U8 ? 8 : 16; }
int vec_align_coef(int dt) {
  const int b = 4 * dt_size(dt);
  return b < 16 ? b : 16;
}

cudaError_t dispatch_dwt2d(int tin, int tout, Pass p, int cfg, bool vec, cudaStream_t s) {
  switch (tin) {
    case HAAR_F32: return launch_dwt2d_f32(tout, p, cfg, vec, 0, s);
    case HAAR_BF16: return launch_dwt2d_bf16(tout, p, cfg, vec, 0, s);
    case HAAR_F16: return launch_dwt2d_f16(tout, p, cfg, vec, 0, s);
    case HAAR_U8: return launch_dwt2d_u8(tout, p, cfg, vec, 0, s);
    case HAAR_F64: return launch_dwt2d_f64(tout, p, cfg, vec, 0, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t dispatch_idwt2d(int tin, int tout, Pass p, int cfg, bool vec, cudaStream_t s) {
  switch (tin) {
    case HAAR_F32: return launch_idwt2d_f32(tout, p, cfg, vec, 0, s);
    case HAAR_BF16: return launch_idwt2d_bf16(tout, p, cfg, vec, 0, s);
    case HAAR_F16: return launch_idwt2d_f16(tout, p, cfg, vec, 0, s);
    case HAAR_F64: return launch_idwt2d_f64(tout, p, cfg, vec, 0, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t dispatch_dwt1d(int tin, int tout, Pass p, int cfg, bool vec, cudaStream_t s) {
  switch (tin) {
    case HAAR_F32: return launch_dwt1d_f32(tout, p, cfg, vec, s);
    case HAAR_BF16: return launch_dwt1d_bf16(tout, p, cfg, vec, s);
    case HAAR_F16: return launch_dwt1d_f16(tout, p, cfg, vec, s);
    case HAAR_U8: return launch_dwt1d_u8(tout, p, cfg, vec, s);
    case HAAR_F64: return launch_dwt1d_f64(tout, p, cfg, vec, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t dispatch_idwt1d(int tin, int tout, Pass p, int cfg, bool vec, cudaStream_t s) {
  switch (tin) {
    case HAAR_F32: return launch_idwt1d_f32(tout, p, cfg, vec, s);
    case HAAR_BF16: return launch_idwt1d_bf16(tout, p, cfg, vec, s);
    case HAAR_F16: return launch_idwt1d_f16(tout, p, cfg, vec, s);
    case HAAR_F64: return launch_idwt1d_f64(tout, p, cfg, vec, s);
  }
  return cudaErrorInvalidValue;
}

// Common validation of (src, dst, levels); fills *empty.
int validate(const haar_desc* src, const haar_desc* dst, int levels, bool two_d, bool forward,
             bool* empty) {
  int rc = check_desc(src);
  if (rc) return rc;
  rc = check_desc(dst);
  if (rc) return rc;
  if (levels < 1 || levels > 62) return HAAR_EINVAL;
  if (src->batch != dst->batch || src->h != dst->h || src->w != dst->w) return HAAR_EINVAL;
  if (forward ? !fwd_pair_ok(src->dtype, dst->dtype) : !inv_pair_ok(src->dtype, dst->dtype))
    return HAAR_EDTYPE;
  if (!divisible(src->w, levels)) return HAAR_ESHAPE;
  if (two_d && !divisible(src->h, levels)) return HAAR_ESHAPE;
  *empty = is_empty(src);
  if (*empty) return HAAR_OK;
  if (overlaps(src, dst)) return HAAR_EALIAS;
  return HAAR_OK;
}

int check_workspace(const Workspace& ws, void* workspace, size_t bytes) {
  if (ws.total == 0) return HAAR_OK;
  if (!workspace || bytes < ws.total || ((uintptr_t)workspace & 255)) return HAAR_EWORKSPACE;
  return HAAR_OK;
}

}  // namespace

namespace fh {
// SM count of the current device, looked up once per device.
int fast_sm_count() {
  static std::atomic<int> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 1;
  if (dev < 64) {
    const int c = cache[dev].load(std::memory_order_relaxed);
    if (c > 0) return c;
  }
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
    return 1;
  if (dev < 64) cache[dev].store(n, std::memory_order_relaxed);
  return n;
}

// The argument checks of haar_dwt_2d alone, for the allocation-free variant
// (haar_noalloc.cu), which must report argument errors before it looks at
// the scratch size.
int validate_dwt_2d(const haar_desc* x, const haar_desc* coef, int levels, bool* empty) {
  return validate(x, coef, levels, true, true, empty);
}
}  // namespace fh

extern "C" {

int haar_version(void) { return FASTHAAR_VERSION; }

int haar_last_cuda_error(void) { return g_last_cuda; }

const char* haar_status_string(int status) {
  switch (status) {
    case HAAR_OK: return "ok";
    case HAAR_EINVAL: return "invalid argument";
    case HAAR_ESHAPE: return "extent not divisible by 2^levels";
    case HAAR_EDTYPE: return "unsupported dtype";
    case HAAR_EALIAS: return "input and output overlap";
    case HAAR_ECUDA: return "CUDA error";
    case HAAR_ETIMEOUT: return "device wait timed out";
    case HAAR_EWORKSPACE: return "workspace missing or too small";
    case HAAR_EQUEUE: return "work queue inconsistent";
  }
  return "unknown status";
}

int haar_workspace_size(int op, const haar_desc* src, int levels, size_t* bytes) {
  if (!bytes) return HAAR_EINVAL;
  *bytes = 0;
  const int rc = check_desc(src);
  if (rc) return rc;
  if (levels < 1 || levels > 62) return HAAR_EINVAL;
  const bool two_d = op == HAAR_OP_DWT_2D || op == HAAR_OP_IDWT_2D;
  if (op < HAAR_OP_DWT_1D || op > HAAR_OP_IDWT_2D) return HAAR_EINVAL;
  const Plan pl = make_plan(levels, two_d ? kMax2dFused : kMax1dFused);
  *bytes = ws_layout(pl, src, two_d).total;
  return HAAR_OK;
}

int haar_dwt_2d(const haar_desc* x, const haar_desc* coef, int levels, void* workspace,
                size_t workspace_bytes, void* cuda_stream) {
  bool empty = false;
  int rc = validate(x, coef, levels, true, true, &empty);
  if (rc || empty) return rc;
  const Plan pl = make_plan(levels, kMax2dFused);
  const Workspace ws = ws_layout(pl, x, true);
  rc = check_workspace(ws, workspace, workspace_bytes);
  if (rc) return rc;
  const cudaStream_t st = (cudaStream_t)cuda_stream;
  const int acc = acc_dtype(x->dtype);
  char* wsb = static_cast<char*>(workspace);

  for (int k = 0; k < pl.n; ++k) {
    const int s0 = pl.cum[k], s1 = pl.cum[k + 1];
    const int64_t hk = x->h >> s0, wk = x->w >> s0;
    Pass p{};
    int tin;
    if (k == 0) {
      p.src = x->ptr;
      p.s_bs = x->batch_stride;
      p.s_rs = x->row_stride;
      tin = x->dtype;
    } else {
      p.src = wsb + ws.off[k];
      p.s_bs = hk * wk;
      p.s_rs = wk;
      tin = acc;
    }
    p.dst = coef->ptr;
    p.d_bs = coef->batch_stride;
    p.d_rs = coef->row_stride;
    if (k == pl.n - 1) {
      p.ll = coef->ptr;
      p.l_bs = coef->batch_stride;
      p.l_rs = coef->row_stride;
      p.ll_acc = 0;
    } else {
      const int64_t h1 = x->h >> s1, w1 = x->w >> s1;
      p.ll = wsb + ws.off[k + 1];
      p.l_bs = h1 * w1;
      p.l_rs = w1;
      p.ll_acc = 1;
    }
    p.levels = pl.lv[k];
    p.batch = x->batch;
    p.h = hk;
    p.w = wk;
    const bool vec = (wk % 8 == 0) &&
                     aligned(p.src, p.s_bs, p.s_rs, dt_size(tin), vec_align_img(tin)) &&
                     aligned(p.dst, p.d_bs, p.d_rs, dt_size(coef->dtype),
                             vec_align_coef(coef->dtype));
    const int cfg = (vec && hk % 32 == 0 && wk % 32 == 0) ? kFast : tile_for_levels(pl.lv[k]);
    const cudaError_t e = dispatch_dwt2d(tin, coef->dtype, p, cfg, vec, st);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  return HAAR_OK;
}

int haar_idwt_2d(const haar_desc* coef, const haar_desc* x, int levels, void* workspace,
                 size_t workspace_bytes, void* cuda_stream) {
  bool empty = false;
  int rc = validate(coef, x, levels, true, false, &empty);
  if (rc || empty) return rc;
  const Plan pl = make_plan(levels, kMax2dFused);
  const Workspace ws = ws_layout(pl, coef, true);
  rc = check_workspace(ws, workspace, workspace_bytes);
  if (rc) return rc;
  const cudaStream_t st = (cudaStream_t)cuda_stream;
  const int acc = acc_dtype(coef->dtype);
  char* wsb = static_cast<char*>(workspace);

  for (int k = pl.n - 1; k >= 0; --k) {
    const int s0 = pl.cum[k], s1 = pl.cum[k + 1];
    const int64_t hk = coef->h >> s0, wk = coef->w >> s0;
    Pass p{};
    p.src = coef->ptr;
    p.s_bs = coef->batch_stride;
    p.s_rs = coef->row_stride;
    if (k == pl.n - 1) {
      p.ll = coef->ptr;
      p.l_bs = coef->batch_stride;
      p.l_rs = coef->row_stride;
      p.ll_acc = 0;
    } else {
      const int64_t h1 = coef->h >> s1, w1 = coef->w >> s1;
      p.ll = wsb + ws.off[k + 1];
      p.l_bs = h1 * w1;
      p.l_rs = w1;
      p.ll_acc = 1;
    }
    int tout;
    if (k == 0) {
      p.dst = x->ptr;
      p.d_bs = x->batch_stride;
      p.d_rs = x->row_stride;
      tout = x->dtype;
    } else {
      p.dst = wsb + ws.off[k];
      p.d_bs = hk * wk;
      p.d_rs = wk;
      tout = acc;
    }
    p.levels = pl.lv[k];
    p.batch = coef->batch;
    p.h = hk;
    p.w = wk;
    const bool vec = (wk % 8 == 0) &&
                     aligned(p.src, p.s_bs, p.s_rs, dt_size(coef->dtype),
                             vec_align_coef(coef->dtype)) &&
                     aligned(p.dst, p.d_bs, p.d_rs, dt_size(tout), vec_align_img(tout));
    const int cfg = (vec && hk % 32 == 0 && wk % 32 == 0) ? kFast : tile_for_levels(pl.lv[k]);
    const cudaError_t e = dispatch_idwt2d(coef->dtype, tout, p, cfg, vec, st);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  return HAAR_OK;
}

int haar_dwt_1d(const haar_desc* x, const haar_desc* coef, int levels, void* workspace,
                size_t workspace_bytes, void* cuda_stream) {
  bool empty = false;
  int rc = validate(x, coef, levels, false, true, &empty);
  if (rc || empty) return rc;
  const Plan pl = make_plan(levels, kMax1dFused);
  const Workspace ws = ws_layout(pl, x, false);
  rc = check_workspace(ws, workspace, workspace_bytes);
  if (rc) return rc;
  const cudaStream_t st = (cudaStream_t)cuda_stream;
  const int acc = acc_dtype(x->dtype);
  char* wsb = static_cast<char*>(workspace);

  for (int k = 0; k < pl.n; ++k) {
    const int s0 = pl.cum[k], s1 = pl.cum[k + 1];
    const int64_t wk = x->w >> s0;
    Pass p{};
    int tin;
    if (k == 0) {
      p.src = x->ptr;
      p.s_bs = x->batch_stride;
      p.s_rs = x->row_stride;
      tin = x->dtype;
    } else {
      p.src = wsb + ws.off[k];
      p.s_bs = x->h * wk;
      p.s_rs = wk;
      tin = acc;
    }
    p.dst = coef->ptr;
    p.d_bs = coef->batch_stride;
    p.d_rs = coef->row_stride;
    if (k == pl.n - 1) {
      p.ll = coef->ptr;
      p.l_bs = coef->batch_stride;
      p.l_rs = coef->row_stride;
      p.ll_acc = 0;
    } else {
      const int64_t w1 = x->w >> s1;
      p.ll = wsb + ws.off[k + 1];
      p.l_bs = x->h * w1;
      p.l_rs = w1;
      p.ll_acc = 1;
    }
    p.levels = pl.lv[k];
    p.batch = x->batch;
    p.h = x->h;
    p.w = wk;
    const bool vec = (wk % 8 == 0) &&
                     aligned(p.src, p.s_bs, p.s_rs, dt_size(tin), vec_align_img(tin)) &&
                     aligned(p.dst, p.d_bs, p.d_rs, dt_size(coef->dtype),
                             vec_align_coef(coef->dtype));
    const int cfg = (vec && wk % 256 == 0 && pl.lv[k] <= 8) ? kFast1 : chunk_for_levels(pl.lv[k]);
    const cudaError_t e = dispatch_dwt1d(tin, coef->dtype, p, cfg, vec, st);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  return HAAR_OK;
}

int haar_idwt_1d(const haar_desc* coef, const haar_desc* x, int levels, void* workspace,
                 size_t workspace_bytes, void* cuda_stream) {
  bool empty = false;
  int rc = validate(coef, x, levels, false, false, &empty);
  if (rc || empty) return rc;
  const Plan pl = make_plan(levels, kMax1dFused);
  const Workspace ws = ws_layout(pl, coef, false);
  rc = check_workspace(ws, workspace, workspace_bytes);
  if (rc) return rc;
  const cudaStream_t st = (cudaStream_t)cuda_stream;
  const int acc = acc_dtype(coef->dtype);
  char* wsb = static_cast<char*>(workspace);

  for (int k = pl.n - 1; k >= 0; --k) {
    const int s0 = pl.cum[k], s1 = pl.cum[k + 1];
    const int64_t wk = coef->w >> s0;
    Pass p{};
    p.src = coef->ptr;
    p.s_bs = coef->batch_stride;
    p.s_rs = coef->row_stride;
    if (k == pl.n - 1) {
      p.ll = coef->ptr;
      p.l_bs = coef->batch_stride;
      p.l_rs = coef->row_stride;
      p.ll_acc = 0;
    } else {
      const int64_t w1 = coef->w >> s1;
      p.ll = wsb + ws.off[k + 1];
      p.l_bs = coef->h * w1;
      p.l_rs = w1;
      p.ll_acc = 1;
    }
    int tout;
    if (k == 0) {
      p.dst = x->ptr;
      p.d_bs = x->batch_stride;
      p.d_rs = x->row_stride;
      tout = x->dtype;
    } else {
      p.dst = wsb + ws.off[k];
      p.d_bs = coef->h * wk;
      p.d_rs = wk;
      tout = acc;
    }
    p.levels = pl.lv[k];
    p.batch = coef->batch;
    p.h = coef->h;
    p.w = wk;
    const bool vec = (wk % 8 == 0) &&
                     aligned(p.src, p.s_bs, p.s_rs, dt_size(coef->dtype),
                             vec_align_coef(coef->dtype)) &&
                     aligned(p.dst, p.d_bs, p.d_rs, dt_size(tout), vec_align_img(tout));
    const int cfg = (vec && wk % 256 == 0 && pl.lv[k] <= 8) ? kFast1 : chunk_for_levels(pl.lv[k]);
    const cudaError_t e = dispatch_idwt1d(coef->dtype, tout, p, cfg, vec, st);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  return HAAR_OK;
}

}  // extern "C"
