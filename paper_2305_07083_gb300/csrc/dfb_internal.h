// Internal definitions shared by the host side (dfb_api.cu, dfb_noalloc.cu)
// and the kernels (dfb_kernels.cu, dfb_composite.cu).  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/dfb.h"

namespace dfb {

// Pixels per composite work item (= consumer threads of a CTA).  A work item
// is 256 consecutive pixels of one tile; a 64x64 tile is 16 items.  Tiles of
// fewer than 256 pixels are one item each.
constexpr int kItemPixels = 256;
// Fragments of a work item staged in shared memory by one fill of the
// composite's ring.  Items of tiles with more fragments are streamed through
// the ring in several fills of kFill fragments each.
constexpr int kStageFragments = 16;
constexpr int kFill = 8;
// Per-pixel sort window of the exact re-do path: fragments are taken in
// rounds of at most kSortWindow, each round the window's nearest not yet
// blended.
constexpr int kSortWindow = 16;

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

// Fixed-size per-tile block written by the bucketing: the tile's fragment
// count, its offset in the sorted records, and its first kStageFragments
// records.  The composite fetches one block per work item with a single bulk
// copy, so locating an item's fragments needs no dependent loads.
struct TileBlock {
  int n;
  int off;
  int pad[6];
  FragRec recs[kStageFragments];
};
static_assert(sizeof(TileBlock) == 32 + 32 * kStageFragments, "TileBlock layout");

// Tables of the sRGB encode (IEC 61966-2-1) used by the RGBA8 pack.  thr[c-1]
// is the linear value where code c begins (the inverse curve at (c-0.5)/255,
// evaluated in double and rounded to FP32), thr[255] = +inf, so the code of x
// is the number of entries <= x.  lut[i] is that number at the start of
// bucket i, the FP32 values whose top 16 bits are kSrgbLutBias + i (exponent
// and 7 mantissa bits; bucket 0 starts at 2^-13, below the first boundary,
// and bucket kSrgbLutEntries-1 is 1.0).  No bucket holds more than one
// boundary, so code(x) = lut[i] + (x >= thr[lut[i]]).
constexpr int kSrgbLutEntries = 13 * 128 + 1;
constexpr int kSrgbLutBias = (127 - 13) << 7;
struct SrgbTables {
  float thr[256];
  unsigned char lut[1792];
};
static_assert(sizeof(SrgbTables) % 128 == 0 && kSrgbLutEntries <= 1792, "sRGB tables");

// Everything a composite work item needs about its frame.
struct FrameArgs {
  int W, H, T, logT;
  int tilesX, nTiles;
  int P;                       // pixels per work item: min(kItemPixels, T*T)
  int chunks;                  // work items per tile: T*T / P (a power of two)
  int logChunks;
  float invTilesX;             // 1 / tilesX, for tile -> (tx, ty) without a division
  int slots;                   // per-tile variance partials: ceil(T*T / 32)
  int tileBase;                // first global tile index of this frame
  int mode, dtype;
  unsigned flags;
  int frameN;                  // frames in the accumulation including this one
  int kahan;                   // 1: compensated running sum this frame
  int kahanFirst;              // 1: first compensated frame (comp reads as 0)
  int stateInRing;             // 1: the accumulation state comes with the item's last
                               // fill; 0: the consumers load it themselves
  float invN, invNm1;          // 1/n and 1/(n-1) (0 when n == 1)
  float bgR, bgG, bgB, bgA;    // premultiplied background colour and coverage
  int pixelOp;                 // enum dfb_pixel_op applied before the RGBA8 pack
  float exposure;
  int curveN;                  // DFB_PIXELOP_CURVE: samples per channel (>= 2)
  float curveXMax;             // DFB_PIXELOP_CURVE: input range [0, curveXMax]
  float curveScale;            // (curveN - 1) / curveXMax
  const FragRec* srecs;        // records grouped by global tile, (key, index) order
  const TileBlock* blocks;     // per global tile
  float4* color;               // row-major image
  float4* accum;               // tile-major: tile * T*T + pixel of the tile
  float4* comp;                // tile-major
  float4* m2;                  // tile-major
  uint32_t* rgba8;
  float* tileVar;
  float* varPartial;           // [nTiles * slots] per-warp partial sums
  const float* curve;          // DFB_PIXELOP_CURVE: 3 * curveN samples, channel-major
};

// Samples per channel of a user tone curve (DFB_PIXELOP_CURVE), at most.
constexpr int kMaxCurve = 4096;

// Launch shape of the composite kernel, chosen by the autotuner.
struct TuneParams {
  int ringKB;     // shared-memory ring per CTA in KB (its depth: items in flight)
  int ctasPerSm;  // persistent CTAs per SM
  int groups;     // consumer groups per CTA (items composited at once)
};

// Tiles of a launch with more than kStageFragments fragments: their work
// items (the only ones that can need the exact re-do kernel) and the longest
// list among them.
struct LongList {
  int items = 0;
  int maxFragments = 0;
};

// Bits of a launch's device error word.
constexpr unsigned kErrTimeout = 1u;   // a wait ran out
constexpr unsigned kErrDrain = 2u;     // a copy in flight did not land while giving up
constexpr unsigned kErrCheck = 8u;     // a device-side check of the checked build failed

// Device-side checks, compiled in by -DDFB_CHECKED (libdfb_checked.so): a
// failed check sets kErrCheck in the error word and the guarded access is
// skipped.  In the normal build the condition is not evaluated.
#ifdef DFB_CHECKED
#define DFB_CHECK(cond, err) ((cond) || (atomicOr((err), ::dfb::kErrCheck), false))
#else
#define DFB_CHECK(cond, err) (true)
#endif

// Controls of one composite launch.
struct LaunchCtl {
  unsigned long long waitNs;  // bound on every barrier wait inside the kernel
  int stallItem;              // test fault injection: this item is never filled (-1: off)
  unsigned* err;              // device error word; bit 0 = a wait timed out
  int* redo;                  // [count, items...]: multi-fill items left to the re-do kernel
};

// Bucketing (K1), second half.  The host groups the records by global tile
// while it stages them (a stable counting sort: submission order kept within
// a tile) and uploads the tile offsets tileOff[0..nTiles] (tileOff[nTiles] =
// records).  One kernel then orders every tile's records by (order key,
// position) -- the (key, submit index) order -- into `srecs` and fills one
// TileBlock per tile.  It also clears the re-do count `redo[0]` (if given)
// of the composite launch that follows.
cudaError_t launch_bucket(const FragRec* grouped, const int* tileOff, int nTiles, FragRec* srecs,
                          TileBlock* blocks, int* redo, cudaStream_t s);

// Composite + accumulate + variance + pack (K2/K3 + K4) over the work items of
// `nFrames` frames (device arrays `frames` and `itemBase`, nFrames + 1 prefix
// of work items), all of storage dtype `dtype`, one persistent launch; then,
// if the launch has long tiles, the exact re-do of the multi-fill items the
// persistent kernel left (out-of-order depths); then, if `accumulate`, the
// per-tile variance of `totalTiles` global tiles.  `hostFrames` and
// `hostItemBase` are host copies of `frames` and `itemBase` (or null): for a
// launch of one frame, or of a few, the persistent kernel then takes them by
// value as a kernel parameter instead of reading the global tables.
// `afterMain`, if given, is recorded on `s` right after the persistent
// kernel (before the re-do and variance kernels), for tracing.
cudaError_t launch_composite(const FrameArgs* frames, const int* itemBase, int nFrames,
                             int totalItems, int totalTiles, bool accumulate, int dtype,
                             const TuneParams& tune, const LaunchCtl& ctl, const LongList& lng,
                             const FrameArgs* hostFrames, const int* hostItemBase,
                             cudaEvent_t afterMain, cudaStream_t s);

// Default launch shape for a dtype.
// Default launch shape for a launch whose frames have `fragmentsPerTile`
// fragment tiles per image tile on average.
TuneParams default_tune(int dtype, double fragmentsPerTile);

// Mean fragments per tile from which the composite's consumers load a
// frame's accumulation state themselves instead of receiving it through the
// shared-memory ring with the fragments.
constexpr double kStateLoadFragmentsPerTile = 2.0;

// Tile-major state -> row-major image `out` (device):
//   out = (a - b) * scale  when b is given, else a * scale.
cudaError_t launch_tiles_to_image(const float4* a, const float4* b, float scale, float4* out,
                                  int W, int H, int T, cudaStream_t s);
// Row-major image -> tile-major state (pixels outside the frame untouched).
cudaError_t launch_image_to_tiles(const float4* in, float4* out, int W, int H, int T,
                                  cudaStream_t s);

// FP32 -> storage dtype conversion of fragment tiles (producer side).
cudaError_t launch_convert(const float* src, void* dst, float* scales, int nTiles,
                           int tilePixels, int dtype, cudaStream_t s);

// Upload the sRGB threshold table to the current device (idempotent).
cudaError_t ensure_tables();

// Fill the geometry fields of FrameArgs that follow from W, H, T.
inline void frame_geometry(FrameArgs& a, int W, int H, int T) {
  a.W = W;
  a.H = H;
  a.T = T;
  int l = 0;
  while ((1 << l) < T) ++l;
  a.logT = l;
  a.tilesX = (W + T - 1) / T;
  a.nTiles = a.tilesX * ((H + T - 1) / T);
  a.P = T * T < kItemPixels ? T * T : kItemPixels;
  a.chunks = T * T / a.P;
  int lc = 0;
  while ((1 << lc) < a.chunks) ++lc;
  a.logChunks = lc;
  a.invTilesX = 1.0f / (float)a.tilesX;
  a.slots = (T * T + 31) / 32;
}

// Order-preserving 32-bit image of a float (NaN must be handled by caller).
inline uint32_t ordered_bits_host(float f) {
  union { float f; uint32_t u; } v;
  v.f = f;
  if (v.u == 0x80000000u) v.u = 0;  // -0 -> +0
  return (v.u & 0x80000000u) ? ~v.u : (v.u | 0x80000000u);
}

}  // namespace dfb
