// haar_internal.h -- host-side interface between the C-ABI layer and the
// kernel launchers.  Not installed; the public interface is include/fasthaar.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fh {

// Storage type codes (same values as haar_dtype in fasthaar.h).
enum Dt { kF32 = 0, kBF16 = 1, kF16 = 2, kU8 = 3, kF64 = 4 };

inline int dt_size(int dt) {
  switch (dt) {
    case kF32: return 4;
    case kBF16: return 2;
    case kF16: return 2;
    case kU8: return 1;
    case kF64: return 8;
    default: return 0;
  }
}

// One launch ("pass") of a fused kernel over a strided batch.  All strides
// are in elements of the buffer they describe.
//   analysis : src = image (Tin), dst = coefficients (Tout),
//              ll  = where LL_levels goes (dst itself, or an accumulator
//                    typed workspace when ll_acc = 1)
//   synthesis: src = coefficients (Tin), dst = image (Tout),
//              ll  = where LL_levels is read from (src itself, or workspace)
// For 2D passes `rows` is the image height h; for 1D passes every row of
// every batch item is an independent signal of length w.
struct Pass {
  const void* src;
  int64_t s_bs, s_rs;
  void* dst;
  int64_t d_bs, d_rs;
  void* ll;
  int64_t l_bs, l_rs;
  int ll_acc;
  int levels;
  int64_t batch, h, w;
  // filled in by the launcher
  int64_t tiles_x, tiles_y, ntiles;
  int64_t pf_blocks;  // blocks that warm L2 before their dependency wait
};

// Tile shapes of the generic 2D kernels (vector path); the scalar path always
// uses a 64 x 64 tile.  kFast selects the register/warp-shuffle kernels
// (haar_fast2d.cuh), valid when both sides are multiples of 32, the rows are
// vector aligned and the pass fuses at most 6 levels.
enum Tile2Cfg { kT32x128 = 0, kT64x128 = 1, kT64x64 = 2, kFast = 3, kTileCount = 4 };
inline int tile_h(int cfg) { return cfg == kT32x128 ? 32 : 64; }
inline int tile_w(int cfg) { return cfg == kT64x64 ? 64 : 128; }
inline int tile_max_levels(int cfg) { return cfg == kT32x128 ? 5 : 6; }
constexpr int kScalarTileLevels = 6;

// 1D chunk shapes: 1024 samples (up to 10 fused levels) or 4096 (12);
// kFast1 selects the register/warp-shuffle kernels (haar_fast1d.cuh), valid
// for lengths that are multiples of 256, aligned rows and at most 8 levels.
enum Chunk1Cfg { kC1024 = 0, kC4096 = 1, kFast1 = 2 };
inline int chunk_max_levels(int cfg) { return cfg == kC1024 ? 10 : 12; }

// ---------------------------------------------------------------------------
// Ragged batches (one persistent launch over images of different sizes).
// ---------------------------------------------------------------------------
struct RaggedImg {
  int64_t in_off, out_off;  // element offsets from the batch base pointers
  int64_t h, w;
  int64_t in_rs, out_rs;
  int64_t unit_begin;       // first work unit of this image
  int32_t levels, units_x;
};

// Workspace header (device): the unit counter, the count of finished blocks,
// the count of units transformed and an error word; the image table follows
// at kRaggedTableOffset.
struct RaggedHeader {
  unsigned long long next_unit;
  unsigned long long blocks_done;
  unsigned long long units_done;
  unsigned long long error;
};
constexpr size_t kRaggedTableOffset = 256;

struct RaggedArgs {
  RaggedHeader* hdr;
  const RaggedImg* imgs;
  int64_t n_imgs;
  int64_t total_units;
  const void* in;
  void* out;
};

// Work-unit shapes (32 x 32 warp blocks: 8, 8, 4 and 16 of them).  A sixth
// level needs units at least 64 rows high (two warp rows).
enum RaggedUnit { kUnit64x128 = 0, kUnit32x256 = 1, kUnit64x64 = 2, kUnit128x128 = 3 };
inline int unit_h(int u) { return u == kUnit32x256 ? 32 : u == kUnit128x128 ? 128 : 64; }
inline int unit_w(int u) {
  return u == kUnit32x256 ? 256 : u == kUnit64x64 ? 64 : 128;
}
inline bool unit_valid(int u) { return u >= kUnit64x128 && u <= kUnit128x128; }

// Records the cudaError_t reported by haar_last_cuda_error() (per host thread).
void set_last_cuda_error(int e);

// Launchers.  Return cudaErrorInvalidValue for an unsupported dtype pair.
// grid_cap <= 0 means one block per tile.
cudaError_t launch_dwt2d(int tin, int tout, Pass p, int tile_cfg, bool vec, int grid_cap,
                         cudaStream_t s);
cudaError_t launch_idwt2d(int tin, int tout, Pass p, int tile_cfg, bool vec, int grid_cap,
                          cudaStream_t s);
cudaError_t launch_dwt1d(int tin, int tout, Pass p, int chunk_cfg, bool vec, cudaStream_t s);
cudaError_t launch_idwt1d(int tin, int tout, Pass p, int chunk_cfg, bool vec, cudaStream_t s);

// Per-Tin entry points (one translation unit each, compiled in parallel).
#define FH_DECL_TIN(NAME)                                                                      \
  cudaError_t launch_dwt2d_##NAME(int tout, Pass p, int tile_cfg, bool vec, int grid_cap,     \
                                  cudaStream_t s);                                             \
  cudaError_t launch_idwt2d_##NAME(int tout, Pass p, int tile_cfg, bool vec, int grid_cap,    \
                                   cudaStream_t s);                                            \
  cudaError_t launch_dwt1d_##NAME(int tout, Pass p, int chunk_cfg, bool vec, cudaStream_t s); \
  cudaError_t launch_idwt1d_##NAME(int tout, Pass p, int chunk_cfg, bool vec, cudaStream_t s); \
  cudaError_t launch_ragged_##NAME(int tout, bool fwd, const RaggedArgs& a, int unit,        \
                                   unsigned grid, cudaStream_t s);
FH_DECL_TIN(f32)
FH_DECL_TIN(bf16)
FH_DECL_TIN(f16)
FH_DECL_TIN(u8)
FH_DECL_TIN(f64)
#undef FH_DECL_TIN

}  // namespace fh
