// haar_swt.cu -- the undecimated ("stationary") Haar transform in 1D: the
// bank of Section II, Fig. 1 WITHOUT the down-sampler, i.e. every output of
// the convolutions is kept, with the filters dilated by 2^(l-1) at level l
// (a trous).  It is the direct form whose decimated outputs the Fast Haar
// bank avoids computing: keeping every 2^l-th sample of level l gives the
// decimated transform exactly.  Boundaries wrap around (periodic).
//
//   a_l[k] = (a_{l-1}[k] + a_{l-1}[k + s]) / sqrt(2),   s = 2^(l-1)
//   d_l[k] = (a_{l-1}[k + s] - a_{l-1}[k]) / sqrt(2)
//   inverse: a_{l-1}[k] = ((a_l[k] - d_l[k]) + (a_l[k - s] + d_l[k - s])) / (2 sqrt(2))
//
// Layout: for every input row of n samples, L + 1 output rows of n samples:
// row 0 = a_L, row l = d_l.  A block produces 2048 consecutive positions of
// one row; the samples it needs (a halo of 2^L - 1 to the right for the
// analysis, to the left for the synthesis) are staged in shared memory and
// all levels are fused there (staged with cp.async 16-byte copies).
#include <cuda_runtime.h>

#include "fasthaar.h"
#include "haar_async.cuh"
#include "haar_internal.h"
#include "haar_kernels.cuh"

namespace fh {

constexpr int kSwtChunk = 2048;
constexpr int kSwtMaxLevels = 10;
constexpr int kSwtHalo = (1 << kSwtMaxLevels) - 1;

struct SwtArgs {
  const void* in;
  void* out;
  int64_t rows, n;
  int levels;
  int64_t chunks;
};

// one staged window: the chunk and its halo, plus the 16-byte copy slack
template <typename T>
__host__ __device__ constexpr int swt_cap() {
  return (kSwtChunk + kSwtHalo + 2 * fvec<T>() + fvec<T>() - 1) / fvec<T>() * fvec<T>();
}

template <typename T>
__global__ void __launch_bounds__(256) k_swt(const SwtArgs a) {
  const unsigned chunks = (unsigned)a.chunks;
  const int64_t row = blockIdx.x / chunks, k0 = (int64_t)(blockIdx.x % chunks) * kSwtChunk;
  const int64_t n = a.n;
  const int C = (int)min((int64_t)kSwtChunk, n - k0);
  const T* x = static_cast<const T*>(a.in) + row * n;
  // the chunk's input (1D, 64 x 2^20, one level: 98 -> 102 % of measured HBM)
  warm_l2<256>(x + k0, (int64_t)C * sizeof(T), threadIdx.x);
  pdl_wait();
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* A = reinterpret_cast<T*>(smem_raw);
  T* B = A + swt_cap<T>();
  const int H = (1 << a.levels) - 1;
  T* out = static_cast<T*>(a.out) + row * (a.levels + 1) * n;
  stage<256>(A, x, n, k0, C + H, threadIdx.x);  // k0 is 16-byte aligned: no shift
  cp_async_wait_all();
  __syncthreads();
  const T r = Consts<T>::s();
  for (int l = 1; l <= a.levels; ++l) {
    const int s = 1 << (l - 1);
    const int m = C + H - (2 * s - 1);  // positions of a_l still needed
    T* dl = out + (int64_t)l * n + k0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      const T u = A[i], v = A[i + s];
      B[i] = (u + v) * r;
      if (i < C) dl[i] = (v - u) * r;
    }
    __syncthreads();
    T* t = A;
    A = B;
    B = t;
  }
  for (int i = threadIdx.x; i < C; i += blockDim.x) out[k0 + i] = A[i];
}

template <typename T>
__global__ void __launch_bounds__(256) k_iswt(const SwtArgs a) {
  const unsigned chunks = (unsigned)a.chunks;
  const int64_t row = blockIdx.x / chunks, k0 = (int64_t)(blockIdx.x % chunks) * kSwtChunk;
  const int64_t n = a.n;
  const int C = (int)min((int64_t)kSwtChunk, n - k0);
  const T* c = static_cast<const T*>(a.in) + row * (a.levels + 1) * n;
  // the chunk's part of every coefficient row (one level: 90 -> 91 %)
  for (int l = 0; l <= a.levels; ++l)
    warm_l2<256>(c + (int64_t)l * n + k0, (int64_t)C * sizeof(T), threadIdx.x);
  pdl_wait();
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* bufA = reinterpret_cast<T*>(smem_raw);
  T* bufB = bufA + swt_cap<T>();
  T* bufD = bufB + swt_cap<T>();
  T* x = static_cast<T*>(a.out) + row * n;
  const int L = a.levels;
  int H = (1 << L) - 1;  // left halo of a_L
  const T* A = bufA + stage<256>(bufA, c, n, k0 - H, C + H, threadIdx.x);
  T* B = bufB;
  const T q = Consts<T>::s() * T(0.5);
  for (int l = L; l >= 1; --l) {
    const int s = 1 << (l - 1);
    const T* D = bufD + stage<256>(bufD, c + (int64_t)l * n, n, k0 - H, C + H, threadIdx.x);
    cp_async_wait_all();
    __syncthreads();
    const int Hn = H - s;  // left halo of a_{l-1}
    for (int j = threadIdx.x; j < C + Hn; j += blockDim.x) {
      const int i = j + s;  // index of position (k0 - Hn + j) in A and D
      B[j] = ((A[i] - D[i]) + (A[i - s] + D[i - s])) * q;
    }
    __syncthreads();
    T* next = B == bufB ? bufA : bufB;  // the buffer A came from
    A = B;
    B = next;
    H = Hn;
  }
  for (int i = threadIdx.x; i < C; i += blockDim.x) x[k0 + i] = A[i];
}

template <typename T>
cudaError_t swt_launch(bool fwd, SwtArgs a, cudaStream_t s) {
  a.chunks = (a.n + kSwtChunk - 1) / kSwtChunk;
  const int64_t g = a.rows * a.chunks;
  if (g == 0) return cudaSuccess;
  if (g > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  const size_t smem = (size_t)(fwd ? 2 : 3) * swt_cap<T>() * sizeof(T);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)g);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (fwd) {
    cudaError_t e = cudaFuncSetAttribute(k_swt<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    return cudaLaunchKernelEx(&cfg, k_swt<T>, a);
  }
  cudaError_t e = cudaFuncSetAttribute(k_iswt<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  return cudaLaunchKernelEx(&cfg, k_iswt<T>, a);
}

}  // namespace fh

using namespace fh;

namespace {

int swt_entry(const void* in, void* out, int dtype, int64_t rows, int64_t n, int levels,
              void* stream, bool fwd) {
  if (dtype != HAAR_F32 && dtype != HAAR_F64) return HAAR_EDTYPE;
  if (rows < 0 || n < 0 || levels < 1 || levels > kSwtMaxLevels) return HAAR_EINVAL;
  if (rows == 0 || n == 0) return HAAR_OK;
  if (!in || !out) return HAAR_EINVAL;
  if (n < ((int64_t)1 << levels)) return HAAR_ESHAPE;  // a dilated tap would wrap twice
  const size_t esz = dtype == HAAR_F64 ? 8 : 4;
  const uintptr_t big = (uintptr_t)rows * (uintptr_t)(levels + 1) * (uintptr_t)n * esz;
  const uintptr_t small = (uintptr_t)rows * (uintptr_t)n * esz;
  const uintptr_t il = (uintptr_t)in, ol = (uintptr_t)out;
  const uintptr_t ih = il + (fwd ? small : big), oh = ol + (fwd ? big : small);
  if (il < oh && ol < ih) return HAAR_EALIAS;
  SwtArgs a{};
  a.in = in;
  a.out = out;
  a.rows = rows;
  a.n = n;
  a.levels = levels;
  const cudaError_t e = dtype == HAAR_F64 ? swt_launch<double>(fwd, a, (cudaStream_t)stream)
                                          : swt_launch<float>(fwd, a, (cudaStream_t)stream);
  if (e != cudaSuccess) {
    set_last_cuda_error((int)e);
    return HAAR_ECUDA;
  }
  return HAAR_OK;
}

}  // namespace

extern "C" {

int haar_swt_1d(const void* x, void* coef, int dtype, int64_t rows, int64_t n, int levels,
                void* cuda_stream) {
  return swt_entry(x, coef, dtype, rows, n, levels, cuda_stream, true);
}

int haar_iswt_1d(const void* coef, void* x, int dtype, int64_t rows, int64_t n, int levels,
                 void* cuda_stream) {
  return swt_entry(coef, x, dtype, rows, n, levels, cuda_stream, false);
}

}  // extern "C"
