// haar_noalloc.cu -- haar_dwt_2d_noalloc: the 2D analysis with its scratch
// space inside the library, for callers that cannot allocate device memory.
//
// A 2D analysis deeper than six levels chains launches through a scratch
// buffer that holds the intermediate low band; haar_dwt_2d takes that buffer
// from the caller.  Some callers have no way to provide it: code that runs
// where device allocation is forbidden or unavailable (a plugin inside a host
// application that owns every allocation, a real-time loop that must not call
// the allocator, a process whose memory pool is fixed up front).  For them
// this entry point keeps the scratch in one fixed array compiled into the
// library, so the call itself allocates nothing.
//
// The array is a file-scope __device__ variable: every GPU on which the
// library's device code is loaded holds kScratchBytes of it until the process
// exits.  Host code cannot use the symbol's name as a device address, so the
// first call on each device looks the address up with cudaGetSymbolAddress
// (with that device current) and remembers it for the life of the process.
// A device reset (cudaDeviceReset) unloads the module and frees the array;
// the remembered address would then be stale, so this entry point must not
// be used on a device after it has been reset.
#include <cuda_runtime.h>

#include <mutex>

#include "fasthaar.h"
#include "haar_internal.h"

namespace fh {
// The argument checks of haar_dwt_2d (descriptors, dtype pair, divisibility,
// aliasing) without any launch (haar_api.cu); *empty is set for an input
// with no pixels.
int validate_dwt_2d(const haar_desc* x, const haar_desc* coef, int levels, bool* empty);
}  // namespace fh

namespace {

constexpr size_t kScratchBytes = (size_t)4 << 20;  // 4 MiB per device
constexpr int kMaxDevices = 64;

std::mutex g_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

}  // namespace

// The scratch array itself (device memory, one copy per device).
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

extern "C" int haar_dwt_2d_noalloc(const haar_desc* x, const haar_desc* coef, int levels,
                                   void* cuda_stream) {
  // Both descriptors are checked before the scratch size, so a bad output
  // descriptor is reported as such whatever the input's size.
  bool empty = false;
  int rc = fh::validate_dwt_2d(x, coef, levels, &empty);
  if (rc != HAAR_OK || empty) return rc;
  size_t need = 0;
  rc = haar_workspace_size(HAAR_OP_DWT_2D, x, levels, &need);
  if (rc != HAAR_OK) return rc;
  if (need > kScratchBytes) return HAAR_EWORKSPACE;  // larger than the built-in array

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    fh::set_last_cuda_error((int)e);
    return HAAR_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return HAAR_EINVAL;

  void* ptr = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_scratch);
      if (e != cudaSuccess) {
        fh::set_last_cuda_error((int)e);
        return HAAR_ECUDA;
      }
      g_scratch_ptr[dev] = p;
    }
    ptr = g_scratch_ptr[dev];
  }
  // Every pass writes the whole scratch region the next pass reads, so no
  // part of the array has to start at zero.
  return haar_dwt_2d(x, coef, levels, ptr, kScratchBytes, cuda_stream);
}
