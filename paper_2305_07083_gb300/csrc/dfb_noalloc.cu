// dfb_composite_noalloc: one frame composited without allocating memory.
//
// Who needs this: callers that are not allowed to call cudaMalloc.  Examples
// are an in-situ simulation or renderer that reserves the whole device up
// front and hands out memory only from its own pool; real-time code where a
// cudaMalloc / cudaFree may synchronise the device and break a frame
// deadline; and code running where the CUDA runtime forbids allocation.  The
// handle-based path (dfb_create ... dfb_end_frame) allocates its framebuffers
// and bucketing scratch, so those callers cannot use it.
//
// This entry point keeps all its scratch (fragment records and the per-tile
// bucketing arrays) in one file-scope device array of fixed size, g_scratch,
// and writes only to the caller's output buffers.  It reuses the bucketing and
// composite kernels of the handle path unchanged.
#include <math.h>
#include <stdint.h>

#include <atomic>
#include <mutex>
#include <vector>

#include "dfb_internal.h"

namespace {

// Failure-detection settings of the calls (process-wide): the bound on every
// device-side wait, and a work item that the next call leaves unfilled.
std::atomic<unsigned long long> g_waitNs{2000000000ull};
std::atomic<int> g_stallItem{-1};

using dfb::FragRec;
using dfb::FrameArgs;

constexpr int kMaxFragments = 65536;  // fragment tiles per call
constexpr int kMaxTiles = 16384;      // tiles per frame
constexpr int kMaxRedo = 1 << 19;     // re-do units (32-pixel units of long tiles' items)

// Layout of g_scratch (each region 256-byte aligned):
//   FrameArgs + item prefix + error word
//   FragRec  recs[kMaxFragments]      32 B each, grouped by tile
//   int      tileIn[kMaxFragments]    raw inputs copied from the caller
//   float    keyIn[kMaxFragments]
//   uint64   rgbaIn[kMaxFragments]
//   uint64   depthIn[kMaxFragments]
//   float    scaleIn[kMaxFragments]
//   int      posIn[kMaxFragments]     each record's place in the grouped list
//   FragRec  srecs[kMaxFragments]     records sorted per tile
//   int      tileOff[kMaxTiles + 1]   offsets of the tiles' lists
//   TileBlock blocks[kMaxTiles]       per-tile count/offset/first records
//   int      redo[kMaxRedo + 1]       the composite's re-do list
constexpr size_t align256(size_t v) { return (v + 255) & ~size_t(255); }
struct Header {
  FrameArgs fa;
  int itemBase[2];
  unsigned err;
};
constexpr size_t kOffRecs = align256(sizeof(Header));
constexpr size_t kOffTileIn = align256(kOffRecs + sizeof(FragRec) * kMaxFragments);
constexpr size_t kOffKeyIn = align256(kOffTileIn + sizeof(int) * kMaxFragments);
constexpr size_t kOffRgbaIn = align256(kOffKeyIn + sizeof(float) * kMaxFragments);
constexpr size_t kOffDepthIn = align256(kOffRgbaIn + sizeof(uint64_t) * kMaxFragments);
constexpr size_t kOffScaleIn = align256(kOffDepthIn + sizeof(uint64_t) * kMaxFragments);
constexpr size_t kOffPosIn = align256(kOffScaleIn + sizeof(float) * kMaxFragments);
constexpr size_t kOffSrecs = align256(kOffPosIn + sizeof(int) * kMaxFragments);
constexpr size_t kOffTileOff = align256(kOffSrecs + sizeof(FragRec) * kMaxFragments);
constexpr size_t kOffBlocks = align256(kOffTileOff + sizeof(int) * (kMaxTiles + 1));
constexpr size_t kOffRedo = align256(kOffBlocks + sizeof(dfb::TileBlock) * kMaxTiles);
constexpr size_t kScratchBytes = align256(kOffRedo + sizeof(int) * (kMaxRedo + 1));  // ~17 MB

// The scratch itself.  Every GPU that loads the library holds it until the
// process exits.  In host code `g_scratch` names a host-side stand-in, not the
// device memory, so host code must only use the address that
// cudaGetSymbolAddress returns for the current device.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch per device, looked up once with that device
// current (the first call on a device does it).
std::mutex g_mu;
void* g_addr[64] = {};

int scratch_for_current_device(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return DFB_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return DFB_ERR_CUDA;
    if (dfb::ensure_tables() != cudaSuccess) return DFB_ERR_CUDA;  // sRGB code boundaries
    g_addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_addr[dev]);
  return DFB_OK;
}

// Build the 32-byte fragment records from the raw per-fragment inputs, each
// at its place in the list grouped by tile.
__global__ void k_pack_records(const int* __restrict__ tileIn, const float* __restrict__ keyIn,
                               const uint64_t* __restrict__ rgbaIn,
                               const uint64_t* __restrict__ depthIn,
                               const float* __restrict__ scaleIn, const int* __restrict__ posIn,
                               int useScale, int n, FragRec* __restrict__ recs) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t u = __float_as_uint(keyIn[i]);
  if (u == 0x80000000u) u = 0u;
  FragRec r;
  r.rgba = reinterpret_cast<const void*>(rgbaIn[i]);
  r.depth = reinterpret_cast<const float*>(depthIn[i]);
  r.tile = (uint32_t)tileIn[i];
  r.key = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
  r.scale = useScale ? scaleIn[i] : 1.0f;
  r.frame = 0u;
  recs[posIn[i]] = r;
}

bool device_accessible(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Input tiles must be device (or managed) memory: the kernels read them with
// bulk copies.  Checking every pointer would cost one driver query per
// fragment tile, so only the first and the last tile of every run of
// back-to-back tiles (each starting `bytes` after the previous one, the
// layout of a pool) are checked.
template <class P>
bool tiles_accessible(const P* const* ptrs, int n, size_t bytes) {
  for (int i = 0; i < n;) {
    int j = i;
    while (j + 1 < n && reinterpret_cast<uintptr_t>(ptrs[j + 1]) ==
                            reinterpret_cast<uintptr_t>(ptrs[j]) + bytes)
      ++j;
    if (!device_accessible(ptrs[i]) || (j != i && !device_accessible(ptrs[j]))) return false;
    i = j + 1;
  }
  return true;
}

// The C entry point runs its body under this guard, so that no C++
// exception (a host vector that cannot grow) crosses the interface.
template <typename F>
int guarded_call(F&& body) noexcept {
  try {
    return body();
  } catch (const std::bad_alloc&) {
    return DFB_ERR_OOM;
  } catch (...) {
    return DFB_ERR_STATE;
  }
}

int composite_noalloc(int width, int height, int tile_size, int mode, int dtype, int n,
                      const int* tile_ids, const float* order_keys, const void* const* rgba,
                      const float* const* depth, const float* scales, const float* background,
                      float* color_out, uint32_t* rgba8_out, void* stream) {
  // ---- validation (host only) ----
  const int T = tile_size;
  if (width < 1 || height < 1 || T < 4 || T > 256 || (T & (T - 1))) return DFB_ERR_INVALID_ARG;
  if (mode < DFB_BLEND_DEPTH || mode > DFB_AVERAGE) return DFB_ERR_INVALID_ARG;
  if (dtype < DFB_F32 || dtype > DFB_FP8E4M3) return DFB_ERR_INVALID_ARG;
  if (n < 0 || (n > 0 && (!tile_ids || !order_keys || !rgba || !depth))) return DFB_ERR_INVALID_ARG;
  if (dtype == DFB_FP8E4M3 && n > 0 && !scales) return DFB_ERR_INVALID_ARG;
  if (!color_out && !rgba8_out) return DFB_ERR_INVALID_ARG;
  const int tilesX = (width + T - 1) / T, tilesY = (height + T - 1) / T;
  if ((int64_t)tilesX * tilesY > kMaxTiles || n > kMaxFragments) return DFB_ERR_CAPACITY;
  const int nTiles = tilesX * tilesY;
  std::vector<int> perTile((size_t)nTiles, 0);  // host memory only
  int nLong = 0, maxFrags = 0;
  for (int i = 0; i < n; ++i) {
    if (tile_ids[i] < 0 || tile_ids[i] >= nTiles) return DFB_ERR_TILE_RANGE;
    const int c = ++perTile[tile_ids[i]];
    if (c == dfb::kStageFragments + 1) ++nLong;
    if (c > maxFrags) maxFrags = c;
    if (isnan(order_keys[i]) || !rgba[i] || !depth[i]) return DFB_ERR_INVALID_ARG;
    if (((uintptr_t)rgba[i] % 16) || ((uintptr_t)depth[i] % 16)) return DFB_ERR_INVALID_ARG;
    if (dtype == DFB_FP8E4M3 && !(scales[i] > 0.0f && isfinite(scales[i])))
      return DFB_ERR_INVALID_ARG;
  }
  float bg[4] = {0.f, 0.f, 0.f, 0.f};
  if (background)
    for (int c = 0; c < 4; ++c) {
      if (!isfinite(background[c])) return DFB_ERR_INVALID_ARG;
      bg[c] = background[c];
    }
  cudaStream_t s = (cudaStream_t)stream;
  {
    // The call copies from pageable host memory and waits on the stream,
    // neither of which a capturing stream allows.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
      cudaGetLastError();
      return DFB_ERR_CUDA;
    }
    if (cap != cudaStreamCaptureStatusNone) return DFB_ERR_STATE;
  }
  if ((color_out && !device_accessible(color_out)) ||
      (rgba8_out && !device_accessible(rgba8_out)))
    return DFB_ERR_INVALID_ARG;
  const int chunksPerTile = T * T < dfb::kItemPixels ? 1 : T * T / dfb::kItemPixels;
  // only BLEND_DEPTH items of long tiles can need the re-do kernel
  const int64_t longItems = mode == DFB_BLEND_DEPTH ? (int64_t)nLong * chunksPerTile : 0;
  if (longItems * (dfb::kItemPixels / 32) > kMaxRedo) return DFB_ERR_CAPACITY;
  const size_t rgbaBytes = (size_t)T * T * 4 * (dtype == DFB_F32 ? 4 : (dtype == DFB_FP8E4M3 ? 1 : 2));
  if (!tiles_accessible(rgba, n, rgbaBytes) || !tiles_accessible(depth, n, (size_t)T * T * 4))
    return DFB_ERR_INVALID_ARG;

  unsigned char* base = nullptr;
  int st = scratch_for_current_device(&base);
  if (st != DFB_OK) return st;
  FragRec* recs = reinterpret_cast<FragRec*>(base + kOffRecs);
  int* tileIn = reinterpret_cast<int*>(base + kOffTileIn);
  float* keyIn = reinterpret_cast<float*>(base + kOffKeyIn);
  uint64_t* rgbaIn = reinterpret_cast<uint64_t*>(base + kOffRgbaIn);
  uint64_t* depthIn = reinterpret_cast<uint64_t*>(base + kOffDepthIn);
  float* scaleIn = reinterpret_cast<float*>(base + kOffScaleIn);
  int* posIn = reinterpret_cast<int*>(base + kOffPosIn);
  FragRec* srecs = reinterpret_cast<FragRec*>(base + kOffSrecs);
  int* tileOff = reinterpret_cast<int*>(base + kOffTileOff);
  dfb::TileBlock* blocks = reinterpret_cast<dfb::TileBlock*>(base + kOffBlocks);
  int* redo = reinterpret_cast<int*>(base + kOffRedo);
  Header* dHdr = reinterpret_cast<Header*>(base);
  // each record's place in the list grouped by tile (stable: submission order
  // kept within a tile) and the tiles' offsets -- host memory only
  std::vector<int> off((size_t)nTiles + 1), pos((size_t)n);
  {
    int acc = 0;
    for (int t = 0; t < nTiles; ++t) {
      off[t] = acc;
      acc += perTile[t];
    }
    off[nTiles] = acc;
    std::vector<int> cursor(off.begin(), off.end() - 1);
    for (int i = 0; i < n; ++i) pos[i] = cursor[tile_ids[i]]++;
  }
  dfb::LongList lng;
  lng.items = (int)longItems;
  lng.maxFragments = maxFrags;
  static_assert(sizeof(void*) == sizeof(uint64_t), "64-bit pointers");

  // ---- inputs into the scratch (plain copies; the host arrays may be pageable) ----
  cudaError_t e = cudaSuccess;
  const bool fp8 = dtype == DFB_FP8E4M3;
  if (n > 0) {
    e = cudaMemcpyAsync(tileIn, tile_ids, sizeof(int) * n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(keyIn, order_keys, sizeof(float) * n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(rgbaIn, rgba, sizeof(void*) * n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(depthIn, depth, sizeof(void*) * n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && fp8)
      e = cudaMemcpyAsync(scaleIn, scales, sizeof(float) * n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(posIn, pos.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(tileOff, off.data(), sizeof(int) * (nTiles + 1), cudaMemcpyHostToDevice, s);
  // the caller may reuse its host arrays once this call returns
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess && n > 0) {
    k_pack_records<<<(n + 255) / 256, 256, 0, s>>>(tileIn, keyIn, rgbaIn, depthIn, scaleIn, posIn,
                                                   fp8 ? 1 : 0, n, recs);
    e = cudaGetLastError();
  }
  // ---- bucketing (also clears the re-do count) and compositing ----
  if (e == cudaSuccess) e = dfb::launch_bucket(recs, tileOff, nTiles, srecs, blocks, redo, s);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? DFB_ERR_OOM : DFB_ERR_CUDA;

  Header hdr{};
  FrameArgs& a = hdr.fa;
  dfb::frame_geometry(a, width, height, T);
  a.tileBase = 0;
  a.mode = mode;
  a.dtype = dtype;
  // no accumulation: the per-tile variance scratch of the handle path is unused
  a.flags = (color_out ? DFB_FLAG_WRITE_COLOR : 0u) | (rgba8_out ? DFB_FLAG_PACK_RGBA8 : 0u);
  a.frameN = 1;
  a.stateInRing = 0;  // no accumulation state
  a.invN = 1.0f;
  a.invNm1 = 0.0f;
  a.bgR = bg[0] * bg[3];
  a.bgG = bg[1] * bg[3];
  a.bgB = bg[2] * bg[3];
  a.bgA = bg[3];
  a.pixelOp = DFB_PIXELOP_NONE;
  a.curve = nullptr;
  a.curveN = 0;
  a.curveXMax = 1.0f;
  a.curveScale = 0.0f;
  a.exposure = 1.0f;
  a.srecs = srecs;
  a.blocks = blocks;
  a.color = reinterpret_cast<float4*>(color_out);
  a.rgba8 = rgba8_out;
  hdr.itemBase[0] = 0;
  hdr.itemBase[1] = nTiles * a.chunks;
  hdr.err = 0u;
  // pageable source: the copy has consumed `hdr` when the call returns
  e = cudaMemcpyAsync(dHdr, &hdr, sizeof(Header), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return DFB_ERR_CUDA;
  const dfb::LaunchCtl ctl{g_waitNs.load(), g_stallItem.exchange(-1), &dHdr->err, redo};
  e = dfb::launch_composite(&dHdr->fa, dHdr->itemBase, 1, hdr.itemBase[1], nTiles, false, dtype,
                           dfb::default_tune(dtype, (double)n / (double)nTiles), ctl, lng,
                           &hdr.fa, hdr.itemBase, nullptr, s);
  if (e != cudaSuccess) return DFB_ERR_CUDA;
  // The launch's error word: a wait that ran out (the frame is then
  // incomplete) or, in the checked build, a failed device-side check.  The
  // next call clears it, so it is read here, once the frame is done.
  unsigned err = 0u;
  e = cudaMemcpyAsync(&err, &dHdr->err, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return DFB_ERR_CUDA;
  if (err & dfb::kErrCheck) return DFB_ERR_CHECK;
  if (err) return DFB_ERR_TIMEOUT;
  return DFB_OK;
}

}  // namespace

extern "C" int dfb_noalloc_set_wait_limit(double seconds) {
  if (!(seconds > 0.0) || seconds > 3600.0) return DFB_ERR_INVALID_ARG;
  g_waitNs.store((unsigned long long)(seconds * 1e9));
  return DFB_OK;
}

extern "C" int dfb_noalloc_inject_stall(int item) {
  if (item < -1) return DFB_ERR_INVALID_ARG;
  g_stallItem.store(item);
  return DFB_OK;
}

extern "C" int dfb_composite_noalloc(int width, int height, int tile_size, int mode, int dtype,
                                     int n, const int* tile_ids, const float* order_keys,
                                     const void* const* rgba, const float* const* depth,
                                     const float* scales, const float* background,
                                     float* color_out, uint32_t* rgba8_out, void* stream) {
  return guarded_call([&]() -> int {
    return composite_noalloc(width, height, tile_size, mode, dtype, n, tile_ids, order_keys, rgba,
                             depth, scales, background, color_out, rgba8_out, stream);
  });
}
