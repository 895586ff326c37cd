// haar_filter.cu -- the down-sample-first (polyphase) two-channel bank for
// any even-length orthogonal low-pass filter h[0..K-1], K in {2, 4, 6, 8}
// (Haar, Daubechies-4/6/8, ...), 1D, periodic boundary, multi-level Mallat
// layout [a_L | d_L | ... | d_1].
//
// The paper derives the polyphase split for the two-tap Haar filter and
// states the decomposition for a general filter (Section III, Eq. 7).  With
// the down-sampler moved in front, each output is formed from the K input
// samples it actually depends on and the decimated outputs are never
// computed:
//   a[n] = sum_k h[k] x[(2n + k) mod N],   d[n] = sum_k g[k] x[(2n + k) mod N],
//   g[k] = (-1)^(k+1) h[K-1-k]   (for K = 2 the detail sign of Eq. 9),
//   x[2n + p] = sum_i h[p + 2i] a[n - i] + g[p + 2i] d[n - i],  i < K/2.
//
// Analysis: a block produces 2048 level-0 positions' worth of coefficients
// (2048 / 2^l at level l); it stages the input samples it needs -- the chunk
// plus a right halo of (K - 2)(2^L - 1) samples, wrapped -- in shared memory
// and fuses every level there.  Synthesis: coarsest level first, each level
// needing K/2 - 1 extra coefficients on the left.
#include <cuda_runtime.h>

#include "fasthaar.h"
#include "haar_internal.h"
#include "haar_kernels.cuh"

namespace fh {

constexpr int kFChunk = 2048;
constexpr int kFMaxLevels = 10;
constexpr int kFMaxTaps = 8;
constexpr int kFHalo = (kFMaxTaps - 2) * ((1 << kFMaxLevels) - 1);  // analysis right halo
constexpr int kFBuf = kFChunk + kFHalo;

struct FilterArgs {
  const void* in;
  void* out;
  int64_t rows, n;
  int levels;
  int64_t chunks;
  double h[kFMaxTaps], g[kFMaxTaps];
};

__device__ __forceinline__ int64_t fwrap(int64_t k, int64_t n) {
  k %= n;
  return k < 0 ? k + n : k;
}

template <typename T, int K>
__global__ void __launch_bounds__(256) k_filter_dwt(const FilterArgs a) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* A = reinterpret_cast<T*>(smem_raw);
  T* B = A + kFBuf;
  T h[K], g[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    h[k] = (T)a.h[k];
    g[k] = (T)a.g[k];
  }
  const int64_t row = blockIdx.x / a.chunks, k0 = (blockIdx.x - row * a.chunks) * kFChunk;
  const int64_t n = a.n;
  const int L = a.levels;
  const int C = (int)min((int64_t)kFChunk, n - k0);
  const T* x = static_cast<const T*>(a.in) + row * n;
  T* out = static_cast<T*>(a.out) + row * n;
  int r = (K - 2) * ((1 << L) - 1);  // right halo of the current level
  for (int i = threadIdx.x; i < C + r; i += blockDim.x) A[i] = x[fwrap(k0 + i, n)];
  __syncthreads();
  int len = C;  // chunk length at the current level
  for (int l = 1; l <= L; ++l) {
    const int rn = (r - (K - 2)) / 2;  // halo of the next level
    const int m = len / 2 + rn;        // outputs of this level (chunk + halo)
    T* dl = out + (n >> l) + (k0 >> l);
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
      T lo = T(0), hi = T(0);
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const T v = A[2 * j + k];
        lo = fma(h[k], v, lo);
        hi = fma(g[k], v, hi);
      }
      B[j] = lo;
      if (j < len / 2) dl[j] = hi;
    }
    __syncthreads();
    T* t = A;
    A = B;
    B = t;
    len /= 2;
    r = rn;
  }
  for (int i = threadIdx.x; i < len; i += blockDim.x) out[(k0 >> L) + i] = A[i];
}

template <typename T, int K>
__global__ void __launch_bounds__(256) k_filter_idwt(const FilterArgs a) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int HL = K / 2 - 1;  // extra coefficients needed on the left
  T* A = reinterpret_cast<T*>(smem_raw);
  T* B = A + kFChunk + 64;
  T* D = B + kFChunk + 64;
  T h[K], g[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    h[k] = (T)a.h[k];
    g[k] = (T)a.g[k];
  }
  const int64_t row = blockIdx.x / a.chunks, m0 = (blockIdx.x - row * a.chunks) * kFChunk;
  const int64_t n = a.n;
  const int L = a.levels;
  const int C = (int)min((int64_t)kFChunk, n - m0);
  const T* c = static_cast<const T*>(a.in) + row * n;
  T* x = static_cast<T*>(a.out) + row * n;
  // lo_[l]: first index needed at level l (relative origin of the buffers)
  int64_t lo_[kFMaxLevels + 1];
  lo_[0] = m0;
  for (int l = 1; l <= L; ++l) {
    const int64_t p = lo_[l - 1];
    lo_[l] = (p >= 0 ? p / 2 : -((-p + 1) / 2)) - HL;  // floor(p / 2) - HL
  }
  const int64_t nL = n >> L;
  const int lenL = (int)(((m0 + C) >> L) - lo_[L]);
  for (int i = threadIdx.x; i < lenL; i += blockDim.x) A[i] = c[fwrap(lo_[L] + i, nL)];
  for (int l = L; l >= 1; --l) {
    const int64_t nl = n >> l;
    const int len_l = (int)(((m0 + C) >> l) - lo_[l]);
    const T* dl = c + nl;  // d_l occupies [n >> l, n >> (l - 1))
    for (int i = threadIdx.x; i < len_l; i += blockDim.x) D[i] = dl[fwrap(lo_[l] + i, nl)];
    __syncthreads();
    const int len_o = (int)(((m0 + C) >> (l - 1)) - lo_[l - 1]);
    for (int i = threadIdx.x; i < len_o; i += blockDim.x) {
      const int64_t j = lo_[l - 1] + i;
      const int64_t q = j >= 0 ? j / 2 : -((-j + 1) / 2);  // floor(j / 2)
      const int p = (int)(j - 2 * q);
      T v = T(0);
#pragma unroll
      for (int t = 0; t < K / 2; ++t) {
        const int s = (int)(q - t - lo_[l]);
        v = fma(h[p + 2 * t], A[s], v);
        v = fma(g[p + 2 * t], D[s], v);
      }
      B[i] = v;
    }
    __syncthreads();
    T* tt = A;
    A = B;
    B = tt;
  }
  for (int i = threadIdx.x; i < C; i += blockDim.x) x[m0 + i] = A[i];
}

template <typename T, int K>
cudaError_t filter_launch_k(bool fwd, const FilterArgs& a, unsigned grid, cudaStream_t s) {
  const size_t smem = fwd ? 2 * (size_t)kFBuf * sizeof(T) : 3 * (size_t)(kFChunk + 64) * sizeof(T);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (fwd) {
    cudaError_t e = cudaFuncSetAttribute(k_filter_dwt<T, K>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return e != cudaSuccess ? e : cudaLaunchKernelEx(&cfg, k_filter_dwt<T, K>, a);
  }
  cudaError_t e = cudaFuncSetAttribute(k_filter_idwt<T, K>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return e != cudaSuccess ? e : cudaLaunchKernelEx(&cfg, k_filter_idwt<T, K>, a);
}

template <typename T>
cudaError_t filter_launch(bool fwd, FilterArgs a, int K, cudaStream_t s) {
  a.chunks = (a.n + kFChunk - 1) / kFChunk;
  const int64_t g = a.rows * a.chunks;
  if (g == 0) return cudaSuccess;
  if (g > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  switch (K) {
    case 2: return filter_launch_k<T, 2>(fwd, a, (unsigned)g, s);
    case 4: return filter_launch_k<T, 4>(fwd, a, (unsigned)g, s);
    case 6: return filter_launch_k<T, 6>(fwd, a, (unsigned)g, s);
    case 8: return filter_launch_k<T, 8>(fwd, a, (unsigned)g, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace fh

using namespace fh;

namespace {

int filter_entry(const void* in, void* out, int dtype, int64_t rows, int64_t n, int levels,
                 const double* lowpass, int ntaps, void* stream, bool fwd) {
  if (dtype != HAAR_F32 && dtype != HAAR_F64) return HAAR_EDTYPE;
  if (rows < 0 || n < 0 || levels < 1 || levels > kFMaxLevels) return HAAR_EINVAL;
  if (!lowpass || (ntaps != 2 && ntaps != 4 && ntaps != 6 && ntaps != 8)) return HAAR_EINVAL;
  if (rows == 0 || n == 0) return HAAR_OK;
  if (!in || !out) return HAAR_EINVAL;
  if (n & (((int64_t)1 << levels) - 1)) return HAAR_ESHAPE;
  const size_t esz = dtype == HAAR_F64 ? 8 : 4;
  const uintptr_t bytes = (uintptr_t)rows * (uintptr_t)n * esz;
  const uintptr_t il = (uintptr_t)in, ol = (uintptr_t)out;
  if (il < ol + bytes && ol < il + bytes) return HAAR_EALIAS;
  FilterArgs a{};
  a.in = in;
  a.out = out;
  a.rows = rows;
  a.n = n;
  a.levels = levels;
  for (int k = 0; k < ntaps; ++k) {
    a.h[k] = lowpass[k];
    a.g[k] = ((k & 1) ? 1.0 : -1.0) * lowpass[ntaps - 1 - k];  // (-1)^(k+1) h[K-1-k]
  }
  const cudaError_t e = dtype == HAAR_F64 ? filter_launch<double>(fwd, a, ntaps, (cudaStream_t)stream)
                                          : filter_launch<float>(fwd, a, ntaps, (cudaStream_t)stream);
  if (e != cudaSuccess) {
    set_last_cuda_error((int)e);
    return HAAR_ECUDA;
  }
  return HAAR_OK;
}

}  // namespace

extern "C" {

int haar_filter_dwt_1d(const void* x, void* coef, int dtype, int64_t rows, int64_t n, int levels,
                       const double* lowpass, int ntaps, void* cuda_stream) {
  return filter_entry(x, coef, dtype, rows, n, levels, lowpass, ntaps, cuda_stream, true);
}

int haar_filter_idwt_1d(const void* coef, void* x, int dtype, int64_t rows, int64_t n,
                        int levels, const double* lowpass, int ntaps, void* cuda_stream) {
  return filter_entry(coef, x, dtype, rows, n, levels, lowpass, ntaps, cuda_stream, false);
}

}  // extern "C"
