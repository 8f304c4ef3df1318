// Internal definitions shared by the host side (dfb_api.cu) and the kernels
// (dfb_kernels.cu) of the DFB compositing library.  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/dfb.h"

namespace dfb {

// Pixels (threads) per composite work item.  A work item is one chunk of
// one tile; a 64x64 tile is 16 work items.
constexpr int kItemPixels = 256;
// Per-pixel sort window of the depth mode: fragments are taken in rounds of
// at most kSortWindow, each round the kSortWindow nearest not yet blended.
constexpr int kSortWindow = 16;
// Fragment pointers staged in shared memory per work item.
constexpr int kRecSmem = 256;

// Device record of one submitted fragment tile (32 bytes).
struct FragRec {
  const void* rgba;     // T*T*4 values of the frame's dtype
  const float* depth;   // T*T floats
  uint32_t tile;        // global tile index (frame tile base + tile id)
  uint32_t key;         // order-preserving bits of the canonical order key
  float scale;          // FP8 dequantisation scale
  uint32_t frame;       // index of the frame in a batch (0 for one frame)
};
static_assert(sizeof(FragRec) == 32, "FragRec layout");

// Everything a composite work item needs about its frame.
struct FrameArgs {
  int W, H, T, logT;
  int tilesX, nTiles, chunks;  // chunks = work items per tile
  int tileBase;                // first global tile index of this frame
  int mode, dtype;
  unsigned flags;
  int frameN;                  // frames in the accumulation including this one
  int kahan;                   // 1: compensated running sum this frame
  int kahanFirst;              // 1: first compensated frame (comp reads as 0)
  float invN, invNm1;          // 1/n and 1/(n-1) (0 when n == 1)
  float bgR, bgG, bgB, bgA;    // premultiplied background colour and coverage
  const FragRec* recs;
  const uint32_t* sorted;      // record indices per global tile, (key, index) order
  const int* counts;           // per global tile
  const int* offsets;          // per global tile
  float4* color;
  float4* accum;
  float4* comp;
  float4* m2;
  uint32_t* rgba8;
  float* tileVar;
  float* varPartial;           // [nTiles * chunks] per-item partial sums
  unsigned* tileDone;          // [nTiles] items finished (self-resetting)
};

// Bucketing (K1): counts -> offsets -> scatter -> per-tile rank sort.
// `scratch` layouts are owned by the caller.
cudaError_t launch_bucket(const FragRec* recs, int nRec, int nTilesTotal, int* counts,
                          int* offsets, int* cursor, uint32_t* tmp, uint32_t* sorted,
                          cudaStream_t s);

// Composite + accumulate + variance + pack for one frame (K2/K3 + K4).
cudaError_t launch_composite(const FrameArgs& a, cudaStream_t s);

// Batched persistent form over many frames.  `frames` and `itemBase`
// (nFrames+1 prefix of work items) are device arrays; `queue` is a device
// counter that the kernel resets when the last CTA leaves.
cudaError_t launch_composite_batch(const FrameArgs* frames, const int* itemBase, int nFrames,
                                   int totalItems, int dtype, unsigned* queue, int ctasPerSm,
                                   cudaStream_t s);

// Normalised mean of the accumulation (sum * invN) into `out` (device).
cudaError_t launch_normalise(const float4* accum, const float4* comp, int kahan, float invN,
                             float4* out, int64_t n, cudaStream_t s);
// Per-pixel variance M2 * invNm1 into `out` (device).
cudaError_t launch_variance(const float4* m2, float invNm1, float4* out, int64_t n,
                            cudaStream_t s);

// FP32 -> storage dtype conversion of fragment tiles (producer side).
cudaError_t launch_convert(const float* src, void* dst, float* scales, int nTiles,
                           int tilePixels, int dtype, cudaStream_t s);

// Upload the sRGB threshold table to the current device (idempotent).
cudaError_t ensure_tables();

// Order-preserving 32-bit image of a float (NaN must be handled by caller).
inline uint32_t ordered_bits_host(float f) {
  union { float f; uint32_t u; } v;
  v.f = f;
  if (v.u == 0x80000000u) v.u = 0;  // -0 -> +0
  return (v.u & 0x80000000u) ? ~v.u : (v.u | 0x80000000u);
}

}  // namespace dfb
