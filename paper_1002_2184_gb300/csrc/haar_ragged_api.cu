// haar_ragged_api.cu -- C ABI of the ragged-batch launch: host-side plan
// (validation, work-unit table), workspace upload and dispatch.
#include <cuda_runtime.h>

#include <algorithm>
#include <new>
#include <numeric>
#include <vector>

#include "fasthaar.h"
#include "haar_internal.h"

using namespace fh;

struct haar_ragged_plan {
  std::vector<RaggedImg> imgs;
  std::vector<unsigned char> staging;  // header + table, as uploaded
  int64_t total_units = 0;
  int64_t pixels = 0;
  int unit = kUnit64x128;
  int blocks_per_sm = 4;
  int max_levels = 0;
  int64_t in_gcd = 0, out_gcd = 0;   // gcd of all offsets and strides (alignment)
  int64_t in_extent = 0, out_extent = 0;  // one past the largest element index
  size_t ws_bytes = 0;
};

namespace {

int64_t gcd64(int64_t a, int64_t b) {
  while (b) {
    const int64_t t = a % b;
    a = b;
    b = t;
  }
  return a < 0 ? -a : a;
}

bool fwd_ok(int tin, int tout) {
  if (tin == HAAR_F64 || tout == HAAR_F64) return tin == HAAR_F64 && tout == HAAR_F64;
  return tin >= HAAR_F32 && tin <= HAAR_U8 && tout >= HAAR_F32 && tout <= HAAR_F16;
}

bool inv_ok(int tin, int tout) {
  if (tin == HAAR_F64 || tout == HAAR_F64) return tin == HAAR_F64 && tout == HAAR_F64;
  return tin >= HAAR_F32 && tin <= HAAR_F16 && tout >= HAAR_F32 && tout <= HAAR_F16;
}

cudaError_t dispatch(int tin, int tout, bool fwd, const RaggedArgs& a, int unit, unsigned grid,
                     cudaStream_t s) {
  switch (tin) {
    case HAAR_F32: return launch_ragged_f32(tout, fwd, a, unit, grid, s);
    case HAAR_BF16: return launch_ragged_bf16(tout, fwd, a, unit, grid, s);
    case HAAR_F16: return launch_ragged_f16(tout, fwd, a, unit, grid, s);
    case HAAR_U8: return launch_ragged_u8(tout, fwd, a, unit, grid, s);
    case HAAR_F64: return launch_ragged_f64(tout, fwd, a, unit, grid, s);
  }
  return cudaErrorInvalidValue;
}

int sm_count(int* n) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(n, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    set_last_cuda_error((int)e);
    return HAAR_ECUDA;
  }
  return HAAR_OK;
}

int run(const haar_ragged_plan* plan, const void* in, int in_dtype, void* out, int out_dtype,
        void* workspace, size_t ws_bytes, void* stream, bool fwd) {
  if (!plan) return HAAR_EINVAL;
  if (in_dtype < HAAR_F32 || in_dtype > HAAR_F64 || out_dtype < HAAR_F32 || out_dtype > HAAR_F64)
    return HAAR_EDTYPE;
  if (fwd ? !fwd_ok(in_dtype, out_dtype) : !inv_ok(in_dtype, out_dtype)) return HAAR_EDTYPE;
  if (plan->total_units == 0) return HAAR_OK;
  if (!in || !out) return HAAR_EINVAL;
  if (!workspace || ws_bytes < plan->ws_bytes || ((uintptr_t)workspace & 255))
    return HAAR_EWORKSPACE;
  // vector alignment of every row start (16 B; 8 B for uint8 input)
  const int si = dt_size(in_dtype), so = dt_size(out_dtype);
  const int ai = (fwd && in_dtype == HAAR_U8) ? 8 : 16;
  const int ao = 16;
  if ((uintptr_t)in % ai || (uintptr_t)out % ao || (plan->in_gcd * si) % ai ||
      (plan->out_gcd * so) % ao)
    return HAAR_EINVAL;
  const uintptr_t ilo = (uintptr_t)in, ihi = ilo + (uintptr_t)plan->in_extent * si;
  const uintptr_t olo = (uintptr_t)out, ohi = olo + (uintptr_t)plan->out_extent * so;
  if (ilo < ohi && olo < ihi) return HAAR_EALIAS;
  int sms = 0;
  int rc = sm_count(&sms);
  if (rc) return rc;
  const int64_t g = std::min<int64_t>(plan->total_units, (int64_t)plan->blocks_per_sm * sms);
  RaggedArgs a;
  a.hdr = static_cast<RaggedHeader*>(workspace);
  a.imgs = reinterpret_cast<const RaggedImg*>(static_cast<char*>(workspace) + kRaggedTableOffset);
  a.n_imgs = (int64_t)plan->imgs.size();
  a.total_units = plan->total_units;
  a.in = in;
  a.out = out;
  const cudaError_t e = dispatch(in_dtype, out_dtype, fwd, a, plan->unit, (unsigned)g,
                                 (cudaStream_t)stream);
  if (e != cudaSuccess) {
    set_last_cuda_error((int)e);
    return HAAR_ECUDA;
  }
  return HAAR_OK;
}

}  // namespace

extern "C" {

int haar_ragged_plan_create(const haar_ragged_item* items, int64_t count, int unit,
                            int blocks_per_sm, haar_ragged_plan** plan) {
  if (!plan) return HAAR_EINVAL;
  *plan = nullptr;
  if (count < 0 || (count > 0 && !items)) return HAAR_EINVAL;
  if (count > ((int64_t)1 << 31)) return HAAR_EINVAL;
  if (!unit_valid(unit)) return HAAR_EINVAL;
  if (blocks_per_sm < 1 || blocks_per_sm > 32) return HAAR_EINVAL;
  haar_ragged_plan* p = new (std::nothrow) haar_ragged_plan;
  if (!p) return HAAR_EINVAL;
  p->unit = unit;
  p->blocks_per_sm = blocks_per_sm;
  const int uh = unit_h(unit), uw = unit_w(unit);
  p->imgs.reserve((size_t)count);
  for (int64_t i = 0; i < count; ++i) {
    const haar_ragged_item& it = items[i];
    int rc = HAAR_OK;
    if (it.reserved != 0 || it.h <= 0 || it.w <= 0 || it.in_offset < 0 || it.out_offset < 0 ||
        it.in_row_stride < it.w || it.out_row_stride < it.w || it.levels < 1 || it.levels > 6 ||
        it.h > ((int64_t)1 << 31) || it.w > ((int64_t)1 << 31) ||
        it.in_row_stride > ((int64_t)1 << 40) || it.out_row_stride > ((int64_t)1 << 40))
      rc = HAAR_EINVAL;
    else if (it.h % 32 || it.w % 32 || (it.h & ((1 << it.levels) - 1)) ||
             (it.w & ((1 << it.levels) - 1)) || (it.levels == 6 && unit_h(unit) < 64))
      rc = HAAR_ESHAPE;
    if (rc) {
      delete p;
      return rc;
    }
    RaggedImg r;
    r.in_off = it.in_offset;
    r.out_off = it.out_offset;
    r.h = it.h;
    r.w = it.w;
    r.in_rs = it.in_row_stride;
    r.out_rs = it.out_row_stride;
    r.levels = it.levels;
    r.units_x = (int32_t)((it.w + uw - 1) / uw);
    r.unit_begin = p->total_units;
    p->total_units += (int64_t)r.units_x * ((it.h + uh - 1) / uh);
    p->pixels += it.h * it.w;
    p->max_levels = std::max(p->max_levels, (int)it.levels);
    p->in_gcd = gcd64(gcd64(p->in_gcd, it.in_offset), it.in_row_stride);
    p->out_gcd = gcd64(gcd64(p->out_gcd, it.out_offset), it.out_row_stride);
    p->in_extent = std::max(p->in_extent, it.in_offset + (it.h - 1) * it.in_row_stride + it.w);
    p->out_extent =
        std::max(p->out_extent, it.out_offset + (it.h - 1) * it.out_row_stride + it.w);
    p->imgs.push_back(r);
  }
  p->ws_bytes = kRaggedTableOffset + sizeof(RaggedImg) * p->imgs.size();
  p->ws_bytes = (p->ws_bytes + 255) & ~(size_t)255;
  p->staging.assign(p->ws_bytes, 0);
  if (!p->imgs.empty())
    std::copy(reinterpret_cast<const unsigned char*>(p->imgs.data()),
              reinterpret_cast<const unsigned char*>(p->imgs.data() + p->imgs.size()),
              p->staging.begin() + kRaggedTableOffset);
  *plan = p;
  return HAAR_OK;
}

int haar_ragged_workspace_size(const haar_ragged_plan* plan, size_t* bytes) {
  if (!plan || !bytes) return HAAR_EINVAL;
  *bytes = plan->ws_bytes;
  return HAAR_OK;
}

int haar_ragged_plan_info(const haar_ragged_plan* plan, int64_t* units, int64_t* pixels,
                          int64_t* grid) {
  if (!plan) return HAAR_EINVAL;
  if (units) *units = plan->total_units;
  if (pixels) *pixels = plan->pixels;
  if (grid) {
    int sms = 0;
    const int rc = sm_count(&sms);
    if (rc) return rc;
    *grid = std::min<int64_t>(plan->total_units, (int64_t)plan->blocks_per_sm * sms);
  }
  return HAAR_OK;
}

int haar_ragged_upload(const haar_ragged_plan* plan, void* workspace, size_t workspace_bytes,
                       void* cuda_stream) {
  if (!plan) return HAAR_EINVAL;
  if (!workspace || workspace_bytes < plan->ws_bytes || ((uintptr_t)workspace & 255))
    return HAAR_EWORKSPACE;
  const cudaError_t e = cudaMemcpyAsync(workspace, plan->staging.data(), plan->ws_bytes,
                                        cudaMemcpyHostToDevice, (cudaStream_t)cuda_stream);
  if (e != cudaSuccess) {
    set_last_cuda_error((int)e);
    return HAAR_ECUDA;
  }
  return HAAR_OK;
}

int haar_dwt_2d_ragged(const haar_ragged_plan* plan, const void* in, int in_dtype, void* out,
                       int out_dtype, void* workspace, size_t workspace_bytes, void* cuda_stream) {
  return run(plan, in, in_dtype, out, out_dtype, workspace, workspace_bytes, cuda_stream, true);
}

int haar_idwt_2d_ragged(const haar_ragged_plan* plan, const void* in, int in_dtype, void* out,
                        int out_dtype, void* workspace, size_t workspace_bytes,
                        void* cuda_stream) {
  return run(plan, in, in_dtype, out, out_dtype, workspace, workspace_bytes, cuda_stream, false);
}

int haar_ragged_status(const haar_ragged_plan* plan, void* workspace, int* status,
                       void* cuda_stream) {
  if (!plan || !workspace || !status) return HAAR_EINVAL;
  RaggedHeader h;
  const cudaStream_t s = (cudaStream_t)cuda_stream;
  cudaError_t e = cudaMemcpyAsync(&h, workspace, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess && h.error) {
    const unsigned long long zero = 0;
    e = cudaMemcpyAsync(&static_cast<RaggedHeader*>(workspace)->error, &zero, sizeof(zero),
                        cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  if (e != cudaSuccess) {
    set_last_cuda_error((int)e);
    return HAAR_ECUDA;
  }
  *status = h.error ? HAAR_EQUEUE : HAAR_OK;
  return HAAR_OK;
}

int haar_ragged_plan_destroy(haar_ragged_plan* plan) {
  delete plan;
  return HAAR_OK;
}

}  // extern "C"
