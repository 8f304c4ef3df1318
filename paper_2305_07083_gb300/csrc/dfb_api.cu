// Host side of the DFB C ABI (include/dfb.h): validation, per-tile dependency
// trees, resident framebuffers, record upload and kernel launches.
//
// The paper's DFB runs setTile on every rank and routes tiles to their owners
// through an MPI messaging layer (Sec. 3, 3.2).  Here every tile is owned by
// this process: setTile appends a 32-byte record to the frame's list, and at
// end-of-frame the list is uploaded once and bucketed by tile on the GPU.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <stdexcept>
#include <vector>

#include "dfb_internal.h"

namespace dfb {
cudaError_t upload_srgb_tables(const SrgbTables& host);
}

using dfb::FragRec;
using dfb::FrameArgs;

// What one frame uploads ahead of its records: the frame's arguments and the
// work-item prefix of a one-frame launch.  A multiple of 32 bytes so the
// records that follow stay aligned.
struct FrameHeader {
  FrameArgs fa;
  int itemBase[2];
};
constexpr size_t kHdrBytes = (sizeof(FrameHeader) + 31) / 32 * 32;

namespace {

constexpr int kVersion = 10000;  // 1.0.0

struct GenCount {
  int received = 0;
  int children = 0;
};

struct Arena {
  // Device memory that receives tiles submitted from host pointers.  Chunks
  // are never moved, so earlier pointers of a frame stay valid when it grows.
  std::vector<char*> chunks;
  std::vector<size_t> sizes;
  size_t cur = 0;   // chunk in use
  size_t used = 0;  // bytes used in chunk `cur`
  void reset() { cur = 0; used = 0; }
  char* take(size_t bytes) {
    bytes = (bytes + 255) & ~size_t(255);
    while (cur < chunks.size()) {
      if (used + bytes <= sizes[cur]) {
        char* p = chunks[cur] + used;
        used += bytes;
        return p;
      }
      ++cur;
      used = 0;
    }
    size_t sz = bytes > (size_t(256) << 20) ? bytes : (size_t(256) << 20);
    char* p = nullptr;
    if (cudaMalloc(&p, sz) != cudaSuccess) return nullptr;
    chunks.push_back(p);
    sizes.push_back(sz);
    cur = chunks.size() - 1;
    used = bytes;
    return p;
  }
  void release() {
    for (char* p : chunks) cudaFree(p);
    chunks.clear();
    sizes.clear();
    reset();
  }
};

int elt_bytes(int dtype) {
  switch (dtype) {
    case DFB_F32: return 4;
    case DFB_F16: case DFB_BF16: return 2;
    default: return 1;
  }
}

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

int ilog2(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

std::mutex g_table_mu;
unsigned long long g_table_devices = 0;  // bit d: table uploaded on device d

}  // namespace

// Device buffers of one frame's bucketing (K1) and its launch header.
struct BucketSet {
  // [FrameHeader][FragRec x records, grouped by tile][tile offsets x nTiles+1],
  // uploaded per frame
  unsigned char* dStage = nullptr;
  FragRec* dRecs = nullptr;         // = dStage + kHdrBytes
  FragRec* srecs = nullptr;         // records sorted per tile (bucketing output)
  dfb::TileBlock* blocks = nullptr; // per-tile count/offset/first records
  int* redo = nullptr;              // re-do list of the composite: [count, units...]
  cudaEvent_t ready = nullptr;      // the bucketing that filled this set has finished
  cudaEvent_t released = nullptr;   // the composite that read this set has finished
  bool used = false;
};

struct dfb_ctx {
  dfb_config cfg{};
  int tilesX = 0, tilesY = 0, nTiles = 0, logT = 0, chunks = 0, tilePixels = 0;
  size_t rgbaBytes = 0, depthBytes = 0;
  int device = 0;
  bool allocated = false;

  // frame state
  bool inFrame = false;
  bool haveFrame = false;  // a frame has been composited
  int accumN = 0;          // frames in the accumulation after the last frame
  int pendingN = 0;        // frames in the accumulation after the open frame
  float bg[4] = {0, 0, 0, 0};
  int pixelOp = DFB_PIXELOP_NONE;
  float exposure = 1.0f;
  float* curve = nullptr;  // 3 * kMaxCurve floats once a tone curve is loaded
  int curveDevice = -1;    // device of `curve`
  int curveN = 0;
  float curveXMax = 1.0f;
  std::vector<FragRec> recs;
  std::vector<int> declared;             // gen-0 children per tile, -1 = none
  std::vector<int> recvGen1, childGen1;  // generation-1 arrivals per tile
  std::vector<std::vector<GenCount>> deeper;  // generations >= 2, per tile (lazy)
  std::vector<int> touchedDeeper;
  std::vector<int> fragCount;  // records per tile in the open frame (all generations)
  std::vector<int> longTiles;  // tiles with more than kStageFragments records
  std::vector<int> tileCursor; // host scratch of the grouping by tile
  bool hostCopies = false;
  int64_t launches = 0;  // kernels launched by this handle
  dfb_frame_stats stats{};
  dfb_frame_stats pendingStats{};

  // device buffers
  float4 *color = nullptr, *accum = nullptr, *comp = nullptr, *m2 = nullptr;
  uint32_t* rgba8 = nullptr;
  float *tileVar = nullptr, *varPartial = nullptr;
  // Two bucketing sets, used by alternate frames: the bucketing of frame f+1
  // runs on `bucketStream` while frame f composites from the other set.
  BucketSet sets[2];
  int setIdx = 0;
  size_t recCap = 0;
  cudaStream_t bucketStream = nullptr;
  unsigned* errFlag = nullptr;      // device error word of this handle's launches
  unsigned* lastErr = nullptr;      // error word the last launch touching this handle used
  dfb::TuneParams tune{0, 0, 0};    // {0,0,0}: the library default
  unsigned long long waitNs = 2000000000ull;  // bound on every device-side wait
  int stallItem = -1;               // fault injection for tests (next launch only)
  float4* readTmp = nullptr;  // normalise / variance output for host reads
  unsigned char* hRecs[2] = {nullptr, nullptr};  // pinned staging (double buffered)
  size_t hRecCap[2] = {0, 0};
  cudaEvent_t hRecDone[2] = {nullptr, nullptr};
  int hRecBuf = 0;
  Arena arenas[2];           // alternate per frame so copies overlap compositing
  cudaEvent_t arenaFree[2] = {nullptr, nullptr};  // last frame that read arena k done
  bool arenaUsed[2] = {false, false};
  int arenaIdx = 0;
  cudaStream_t copyStream = nullptr;
  cudaEvent_t copyDone = nullptr;
  cudaEvent_t frameDone = nullptr;
  cudaStream_t lastStream = nullptr;
  bool lastStreamSet = false;

  // tracing: ring of (bucket start, bucket end, composite start, composite end) events
  bool timing = false;
  std::vector<cudaEvent_t> tev;  // 4 per slot
  size_t tHead = 0, tCount = 0;
  dfb_timing tSum{};
};

namespace {

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return DFB_OK;
  if (e == cudaErrorMemoryAllocation) return DFB_ERR_OOM;
  return DFB_ERR_CUDA;
}

int ensure_table(int dev) {
  std::lock_guard<std::mutex> lk(g_table_mu);
  if (dev < 64 && (g_table_devices >> dev) & 1ull) return DFB_OK;
  dfb::SrgbTables tb{};
  float* thr = tb.thr;
  for (int c = 1; c <= 255; ++c) {
    // linear value where code c begins: the inverse sRGB curve at (c-0.5)/255
    const double v = (c - 0.5) / 255.0;
    const double lin = v <= 0.04045 ? v / 12.92 : pow((v + 0.055) / 1.055, 2.4);
    thr[c - 1] = (float)lin;
  }
  thr[255] = INFINITY;
  // bucket table: boundaries <= the first value of each bucket, and a check
  // that no bucket holds a second boundary
  for (int i = 0; i < dfb::kSrgbLutEntries; ++i) {
    auto bucket_start = [](int j) {
      const uint32_t bits = (uint32_t)(j + dfb::kSrgbLutBias) << 16;
      float f;
      memcpy(&f, &bits, sizeof f);
      return f;
    };
    const float x0 = bucket_start(i);
    int c = 0;
    while (c < 255 && thr[c] <= x0) ++c;
    tb.lut[i] = (unsigned char)c;
    if (i + 1 < dfb::kSrgbLutEntries && c + 1 < 255 && thr[c + 1] < bucket_start(i + 1))
      return DFB_ERR_CUDA;  // cannot happen for this curve and bucket width
  }
  const int st = cuda_status(dfb::upload_srgb_tables(tb));
  if (st == DFB_OK && dev < 64) g_table_devices |= (1ull << dev);
  return st;
}

}  // namespace

// Uploads the sRGB code boundaries to the current device once (no allocation).
cudaError_t dfb::ensure_tables() {
  int dev = 0;
  const cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  return ensure_table(dev) == DFB_OK ? cudaSuccess : cudaErrorUnknown;
}

namespace {

template <class T>
cudaError_t dalloc(T** p, size_t count) {
  return cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * (count ? count : 1));
}

// Upload buffer of one frame:
//   [FrameHeader][FragRec x records, grouped by tile][tile offsets x nTiles+1]
size_t stage_bytes(const dfb_ctx* h, size_t records) {
  return kHdrBytes + sizeof(FragRec) * records + sizeof(int) * ((size_t)h->nTiles + 1);
}

// Stable counting sort of records by tile: dst[off[t] ..] holds the records of
// tile t in submission order; off[t] is the exclusive prefix of counts[t] over
// the tiles and off[nTiles] the number of records.  `tileBase` is added to
// each record's tile.  This is the routing half of the bucketing: each record
// lands in its tile's list, as a setTile message lands at the tile's owner.
void group_by_tile(const FragRec* src, size_t n, const int* counts, int nTiles, int tileBase,
                   FragRec* dst, int* off, std::vector<int>& cursor) {
  cursor.resize((size_t)nTiles);
  int acc = 0;
  for (int t = 0; t < nTiles; ++t) {
    off[t] = acc;
    cursor[t] = acc;
    acc += counts[t];
  }
  off[nTiles] = acc;
  for (size_t i = 0; i < n; ++i) {
    FragRec r = src[i];
    const int t = (int)r.tile;
    r.tile += (uint32_t)tileBase;
    dst[cursor[t]++] = r;
  }
}

int grow_records(dfb_ctx* h, size_t need) {
  if (need <= h->recCap && h->sets[0].dStage) return DFB_OK;
  size_t cap = h->recCap ? h->recCap : 4096;
  while (cap < need) cap *= 2;
  // Earlier frames may still read the old arrays (the last frame's
  // composite is ordered after every earlier bucketing and composite).
  if (h->lastStreamSet) cudaEventSynchronize(h->frameDone);
  h->recCap = 0;
  for (BucketSet& b : h->sets) {
    cudaFree(b.dStage);
    cudaFree(b.srecs);
    b.dStage = nullptr;
    b.dRecs = nullptr;
    b.srecs = nullptr;
  }
  for (BucketSet& b : h->sets) {
    cudaError_t e =
        cudaMalloc(reinterpret_cast<void**>(&b.dStage), stage_bytes(h, cap));
    if (e == cudaSuccess) e = dalloc(&b.srecs, cap);
    if (e != cudaSuccess) return cuda_status(e);
    b.dRecs = reinterpret_cast<FragRec*>(b.dStage + kHdrBytes);
  }
  h->recCap = cap;
  return DFB_OK;
}

int grow_staging(dfb_ctx* h, int buf, size_t need) {
  if (need <= h->hRecCap[buf]) return DFB_OK;
  size_t cap = h->hRecCap[buf] ? h->hRecCap[buf] : 4096;
  while (cap < need) cap *= 2;
  if (h->hRecs[buf]) cudaFreeHost(h->hRecs[buf]);
  h->hRecs[buf] = nullptr;
  h->hRecCap[buf] = 0;
  cudaError_t e =
      cudaMallocHost(reinterpret_cast<void**>(&h->hRecs[buf]), stage_bytes(h, cap));
  if (e != cudaSuccess) return DFB_ERR_OOM;
  h->hRecCap[buf] = cap;
  return DFB_OK;
}

void free_device(dfb_ctx* h) {
  // Frees everything and leaves the pointers null, so a second call is a no-op.
  auto fr = [](auto*& p) {
    if (p) cudaFree((void*)p);
    p = nullptr;
  };
  fr(h->color); fr(h->accum); fr(h->comp); fr(h->m2); fr(h->rgba8);
  fr(h->tileVar); fr(h->varPartial);
  fr(h->readTmp); fr(h->errFlag);
  for (BucketSet& b : h->sets) {
    fr(b.redo);
    fr(b.dStage); fr(b.srecs); fr(b.blocks);
    b.dRecs = nullptr;
    if (b.ready) cudaEventDestroy(b.ready);
    if (b.released) cudaEventDestroy(b.released);
    b.ready = b.released = nullptr;
    b.used = false;
  }
  h->recCap = 0;
  if (h->bucketStream) cudaStreamDestroy(h->bucketStream);
  h->bucketStream = nullptr;
  for (int b = 0; b < 2; ++b) {
    if (h->hRecs[b]) cudaFreeHost(h->hRecs[b]);
    h->hRecs[b] = nullptr;
    h->hRecCap[b] = 0;
    if (h->hRecDone[b]) cudaEventDestroy(h->hRecDone[b]);
    h->hRecDone[b] = nullptr;
  }
  for (int k = 0; k < 2; ++k) {
    h->arenas[k].release();
    if (h->arenaFree[k]) cudaEventDestroy(h->arenaFree[k]);
    h->arenaFree[k] = nullptr;
    h->arenaUsed[k] = false;
  }
  for (auto& e : h->tev)
    if (e) cudaEventDestroy(e);
  h->tev.clear();
  h->tHead = h->tCount = 0;
  if (h->copyStream) cudaStreamDestroy(h->copyStream);
  if (h->copyDone) cudaEventDestroy(h->copyDone);
  if (h->frameDone) cudaEventDestroy(h->frameDone);
  h->copyStream = nullptr;
  h->copyDone = h->frameDone = nullptr;
  h->allocated = false;
}

int allocate(dfb_ctx* h) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return DFB_ERR_CUDA;
  // device work of a handle stays on its device (its buffers live there)
  if (h->allocated) return dev == h->device ? DFB_OK : DFB_ERR_STATE;
  if (h->curve && dev != h->curveDevice) return DFB_ERR_STATE;
  h->device = dev;
  int st = ensure_table(dev);
  if (st != DFB_OK) return st;
  const size_t px = (size_t)h->cfg.width * h->cfg.height;
  const size_t tpx = (size_t)h->nTiles * h->tilePixels;  // tile-major state covers whole tiles
  const unsigned f = h->cfg.flags;
  if (f & DFB_FLAG_WRITE_COLOR) e = dalloc(&h->color, px);
  if (e == cudaSuccess && (f & DFB_FLAG_ACCUMULATE)) {
    e = dalloc(&h->accum, tpx);
    if (e == cudaSuccess) e = dalloc(&h->comp, tpx);
    if (e == cudaSuccess) e = dalloc(&h->m2, tpx);
  }
  if (e == cudaSuccess && (f & DFB_FLAG_PACK_RGBA8)) e = dalloc(&h->rgba8, px);
  if (e == cudaSuccess) e = dalloc(&h->tileVar, h->nTiles);
  if (e == cudaSuccess) e = dalloc(&h->varPartial, (size_t)h->nTiles * ((h->tilePixels + 31) / 32));
  if (e == cudaSuccess) e = dalloc(&h->errFlag, 1);
  if (e == cudaSuccess) e = cudaMemset(h->errFlag, 0, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemset(h->tileVar, 0, sizeof(float) * h->nTiles);
  for (BucketSet& b : h->sets) {
    if (e == cudaSuccess) e = dalloc(&b.blocks, h->nTiles);
    // one re-do unit per warp of every work item at most
    if (e == cudaSuccess) e = dalloc(&b.redo, (size_t)h->nTiles * h->chunks * (dfb::kItemPixels / 32) + 1);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b.ready, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b.released, cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->bucketStream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->copyStream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->copyDone, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->frameDone, cudaEventDisableTiming);
  for (int b = 0; b < 2 && e == cudaSuccess; ++b)
    e = cudaEventCreateWithFlags(&h->hRecDone[b], cudaEventDisableTiming);
  for (int b = 0; b < 2 && e == cudaSuccess; ++b)
    e = cudaEventCreateWithFlags(&h->arenaFree[b], cudaEventDisableTiming);
  if (e != cudaSuccess) {
    free_device(h);
    return cuda_status(e);
  }
  h->allocated = true;
  size_t cap = h->cfg.max_fragments > 0 ? (size_t)h->cfg.max_fragments : 4096;
  st = grow_records(h, cap);
  if (st == DFB_OK) st = grow_staging(h, 0, cap);
  if (st == DFB_OK) st = grow_staging(h, 1, cap);
  return st;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int validate_tile(const dfb_ctx* h, const dfb_tile_desc* t) {
  if (!t) return DFB_ERR_INVALID_ARG;
  if (t->tile_id < 0 || t->tile_id >= h->nTiles) return DFB_ERR_TILE_RANGE;
  if (isnan(t->order_key)) return DFB_ERR_INVALID_ARG;
  if (!t->rgba || !t->depth) return DFB_ERR_INVALID_ARG;
  // tiles are streamed with bulk copies, which need 16-byte aligned sources
  if (((uintptr_t)t->rgba % 16) || ((uintptr_t)t->depth % 16)) return DFB_ERR_INVALID_ARG;
  if (t->generation < 1 || t->children < 0) return DFB_ERR_INVALID_ARG;
  if (h->cfg.dtype == DFB_FP8E4M3 && !(t->scale > 0.0f && isfinite(t->scale)))
    return DFB_ERR_INVALID_ARG;
  return DFB_OK;
}

int64_t in_frame_pixels(const dfb_ctx* h, int tile) {
  const int tx = tile % h->tilesX, ty = tile / h->tilesX;
  const int64_t w = h->cfg.width - (int64_t)tx * h->cfg.tile_size;
  const int64_t hh = h->cfg.height - (int64_t)ty * h->cfg.tile_size;
  const int64_t T = h->cfg.tile_size;
  return (w < T ? w : T) * (hh < T ? hh : T);
}

// Count `c` more records of `tile`; list the tile once it has more than the
// composite kernel stages.
inline void count_frags(dfb_ctx* h, int tile, int c) {
  int& v = h->fragCount[tile];
  if (v <= dfb::kStageFragments && v + c > dfb::kStageFragments) h->longTiles.push_back(tile);
  v += c;
}

void note_tree(dfb_ctx* h, int tile, int gen, int children) {
  if (gen == 1) {
    h->recvGen1[tile] += 1;
    h->childGen1[tile] += children;
    return;
  }
  if (h->deeper.empty()) h->deeper.resize(h->nTiles);
  auto& v = h->deeper[tile];
  if (v.empty()) h->touchedDeeper.push_back(tile);
  if ((int)v.size() < gen - 1) v.resize(gen - 1);
  v[gen - 2].received += 1;
  v[gen - 2].children += children;
}

// Copy host data of one or more tiles into the arena; returns device pointers.
int append_records(dfb_ctx* h, int n, const dfb_tile_desc* tiles, int where) {
  // Decide where each pointer lives and copy host tiles into the arena.
  std::vector<const void*> dr(n), dd(n);
  bool anyHost = false;
  for (int i = 0; i < n; ++i) {
    bool devR, devD;
    if (where == DFB_PTR_DEVICE) devR = devD = true;
    else if (where == DFB_PTR_HOST || where == DFB_PTR_HOST_BORROWED) devR = devD = false;
    else {
      devR = is_device_ptr(tiles[i].rgba);
      devD = is_device_ptr(tiles[i].depth);
    }
    dr[i] = devR ? tiles[i].rgba : nullptr;
    dd[i] = devD ? (const void*)tiles[i].depth : nullptr;
    anyHost |= !devR || !devD;
  }
  if (anyHost) {
    int st = allocate(h);
    if (st != DFB_OK) return st;
    Arena& arena = h->arenas[h->arenaIdx];
    if (!h->hostCopies && h->arenaUsed[h->arenaIdx])
      cudaStreamWaitEvent(h->copyStream, h->arenaFree[h->arenaIdx], 0);
    // copy runs of source-contiguous tiles with one call each
    for (int pass = 0; pass < 2; ++pass) {
      const size_t bytes = pass == 0 ? h->rgbaBytes : h->depthBytes;
      int i = 0;
      while (i < n) {
        const void* src0 = pass == 0 ? tiles[i].rgba : (const void*)tiles[i].depth;
        const void* have = pass == 0 ? dr[i] : dd[i];
        if (have) { ++i; continue; }
        int j = i + 1;
        while (j < n) {
          const void* sj = pass == 0 ? tiles[j].rgba : (const void*)tiles[j].depth;
          const void* hj = pass == 0 ? dr[j] : dd[j];
          if (hj || (const char*)sj != (const char*)src0 + (size_t)(j - i) * bytes) break;
          ++j;
        }
        char* dst = arena.take(bytes * (size_t)(j - i));
        if (!dst) return DFB_ERR_OOM;
        cudaError_t e = cudaMemcpyAsync(dst, src0, bytes * (size_t)(j - i),
                                        cudaMemcpyHostToDevice, h->copyStream);
        if (e != cudaSuccess) return cuda_status(e);
        for (int k = i; k < j; ++k) {
          if (pass == 0) dr[k] = dst + (size_t)(k - i) * bytes;
          else dd[k] = dst + (size_t)(k - i) * bytes;
        }
        i = j;
      }
    }
    cudaError_t e = cudaEventRecord(h->copyDone, h->copyStream);
    // DFB_PTR_HOST: the sources are reusable when the call returns;
    // DFB_PTR_HOST_BORROWED: the caller keeps them until the frame is done
    if (e == cudaSuccess && where != DFB_PTR_HOST_BORROWED) e = cudaEventSynchronize(h->copyDone);
    if (e != cudaSuccess) return cuda_status(e);
    h->hostCopies = true;
  }
  for (int i = 0; i < n; ++i) {
    const dfb_tile_desc& t = tiles[i];
    FragRec r;
    r.rgba = dr[i];
    r.depth = (const float*)dd[i];
    r.tile = (uint32_t)t.tile_id;
    r.key = dfb::ordered_bits_host(t.order_key);
    r.scale = h->cfg.dtype == DFB_FP8E4M3 ? t.scale : 1.0f;
    r.frame = 0;
    h->recs.push_back(r);
    note_tree(h, t.tile_id, t.generation, t.children);
    count_frags(h, t.tile_id, 1);
    const int64_t fpx = in_frame_pixels(h, t.tile_id);
    h->pendingStats.fragments += 1;
    h->pendingStats.fragment_pixels += fpx;
  }
  return DFB_OK;
}

int check_trees(const dfb_ctx* h) {
  for (int t = 0; t < h->nTiles; ++t) {
    if (h->declared[t] < 0) continue;
    int expected = h->declared[t];
    if (h->recvGen1[t] != expected) return DFB_ERR_INCOMPLETE;
    int next = h->childGen1[t];
    const std::vector<GenCount>* deeper = h->deeper.empty() ? nullptr : &h->deeper[t];
    int g = 2;
    while (true) {
      const int have = (deeper && (int)deeper->size() >= g - 1) ? (*deeper)[g - 2].received : 0;
      if (next == 0) {
        // nothing more expected: no tile may sit in a deeper generation
        if (deeper)
          for (size_t k = g - 2; k < deeper->size(); ++k)
            if ((*deeper)[k].received) return DFB_ERR_INCOMPLETE;
        break;
      }
      if (have != next) return DFB_ERR_INCOMPLETE;
      next = (*deeper)[g - 2].children;
      ++g;
    }
  }
  return DFB_OK;
}

void fill_frame_args(const dfb_ctx* h, FrameArgs& a, int tileBase, const FragRec* srecs,
                     const dfb::TileBlock* blocks) {
  dfb::frame_geometry(a, h->cfg.width, h->cfg.height, h->cfg.tile_size);
  a.tileBase = tileBase;
  a.mode = h->cfg.mode;
  a.dtype = h->cfg.dtype;
  a.flags = h->cfg.flags & (DFB_FLAG_ACCUMULATE | DFB_FLAG_WRITE_COLOR | DFB_FLAG_PACK_RGBA8);
  const int n = h->pendingN;
  a.frameN = n;
  const int ka = h->cfg.kahan_after;
  a.kahan = n > ka ? 1 : 0;
  a.kahanFirst = n == ka + 1 ? 1 : 0;
  a.invN = 1.0f / (float)n;
  a.invNm1 = n > 1 ? 1.0f / (float)(n - 1) : 0.0f;
  a.bgR = h->bg[0] * h->bg[3];
  a.bgG = h->bg[1] * h->bg[3];
  a.bgB = h->bg[2] * h->bg[3];
  a.bgA = h->bg[3];
  a.pixelOp = h->pixelOp;
  a.exposure = h->exposure;
  a.curve = h->curve;
  a.curveN = h->curveN;
  a.curveXMax = h->curveXMax;
  a.curveScale = h->curveN > 1 ? (float)(h->curveN - 1) / h->curveXMax : 0.0f;
  // The accumulation state travels through the composite's shared-memory
  // ring with the fragments in frames of few fragments per tile (there it
  // is most of an item's bytes, and the ring's prefetch hides its latency);
  // in the others the consumers load it, leaving the ring to the fragments
  // (FP32 at 5.5 fragments per tile: 0.1279 ms against 0.1302 ms).
  a.stateInRing =
      (double)h->recs.size() < dfb::kStateLoadFragmentsPerTile * (double)h->nTiles ? 1 : 0;
  a.srecs = srecs;
  a.blocks = blocks;
  a.color = h->color;
  a.accum = h->accum;
  a.comp = h->comp;
  a.m2 = h->m2;
  a.rgba8 = h->rgba8;
  a.tileVar = h->tileVar;
  a.varPartial = h->varPartial;
}

// Launch shapes the composite is built for (groups per CTA, CTAs per SM).
bool valid_tuning(int ring_kb, int ctas_per_sm, int groups) {
  if (ring_kb == 0 && ctas_per_sm == 0 && groups == 0) return true;
  if (ring_kb < 1 || ring_kb > 227) return false;
  static const int shapes[][2] = {{1, 2}, {2, 2}, {1, 3}, {2, 1}, {3, 1}};
  for (const auto& sh : shapes)
    if (sh[0] == groups && sh[1] == ctas_per_sm) return true;
  return false;
}

// Launch shape for a launch of `nRec` fragment tiles over `nTiles` tiles.
dfb::TuneParams tune_of(const dfb_ctx* h, size_t nRec, size_t nTiles) {
  return h->tune.ringKB ? h->tune
                        : dfb::default_tune(h->cfg.dtype,
                                            (double)nRec / (double)(nTiles ? nTiles : 1));
}

dfb::LaunchCtl ctl_of(const dfb_ctx* h, int* redo) {
  return dfb::LaunchCtl{h->waitNs, h->stallItem, h->errFlag, redo};
}

void finish_stats(dfb_ctx* h) {
  dfb_frame_stats& s = h->pendingStats;
  const int64_t px = (int64_t)h->cfg.width * h->cfg.height;
  s.frame_pixels = px;
  s.tiles = h->nTiles;
  s.accumulated = h->pendingN;
  const int eb = elt_bytes(h->cfg.dtype);
  const int64_t rgbaPx = 4 * eb;
  if (h->cfg.mode == DFB_BLEND_ORDERED || h->cfg.mode == DFB_AVERAGE)
    s.fragment_bytes = s.fragment_pixels * rgbaPx;  // no depth read
  else if (h->cfg.mode == DFB_BLEND_DEPTH) s.fragment_bytes = s.fragment_pixels * (rgbaPx + 4);
  else s.fragment_bytes = s.fragment_pixels * 4 + px * rgbaPx;  // depth + one winner
  int64_t st = 0;
  const unsigned f = h->cfg.flags;
  if (f & DFB_FLAG_WRITE_COLOR) st += 16;
  if (f & DFB_FLAG_ACCUMULATE) {
    const int n = h->pendingN;
    st += n == 1 ? 32 : 64;  // sum and M2: write only on a reset, else read + write
    if (n > h->cfg.kahan_after) st += (n == h->cfg.kahan_after + 1) ? 16 : 32;
  }
  if (f & DFB_FLAG_PACK_RGBA8) st += 4;
  s.state_bytes = st * px;
  s.kernel_launches = h->launches;
}

// Argument checks of a bulk setTile with device or host pointers.
int validate_arrays(const dfb_ctx* h, int n, const int* tile_ids, const float* order_keys,
                    const void* const* rgba, const float* const* depth, const float* scales) {
  if (n > 0 && (!tile_ids || !order_keys || !rgba || !depth)) return DFB_ERR_INVALID_ARG;
  const bool fp8 = h->cfg.dtype == DFB_FP8E4M3;
  if (n > 0 && fp8 && !scales) return DFB_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i) {
    if (tile_ids[i] < 0 || tile_ids[i] >= h->nTiles) return DFB_ERR_TILE_RANGE;
    if (isnan(order_keys[i]) || !rgba[i] || !depth[i]) return DFB_ERR_INVALID_ARG;
    if (((uintptr_t)rgba[i] % 16) || ((uintptr_t)depth[i] % 16)) return DFB_ERR_INVALID_ARG;
    if (fp8 && !(scales[i] > 0.0f && isfinite(scales[i]))) return DFB_ERR_INVALID_ARG;
  }
  return DFB_OK;
}

// Records of n validated generation-1 tiles with device pointers; counts the
// arrivals per tile into `gen1` (if given).  Returns their in-frame pixels.
int64_t build_records(const dfb_ctx* h, int n, const int* tile_ids, const float* order_keys,
                      const void* const* rgba, const float* const* depth, const float* scales,
                      FragRec* out, int* gen1) {
  const bool fp8 = h->cfg.dtype == DFB_FP8E4M3;
  int64_t fpx = 0;
  const int T = h->cfg.tile_size;
  const int fullX = h->cfg.width / T, fullY = h->cfg.height / T;
  for (int i = 0; i < n; ++i) {
    const int t = tile_ids[i];
    out[i].rgba = rgba[i];
    out[i].depth = depth[i];
    out[i].tile = (uint32_t)t;
    out[i].key = dfb::ordered_bits_host(order_keys[i]);
    out[i].scale = fp8 ? scales[i] : 1.0f;
    out[i].frame = 0;
    if (gen1) gen1[t] += 1;
    const int tx = t % h->tilesX, ty = t / h->tilesX;
    fpx += (tx < fullX && ty < fullY) ? (int64_t)T * T : in_frame_pixels(h, t);
  }
  return fpx;
}

// Group the open frame's records by tile behind the header slot of a pinned
// staging buffer, followed by the tile offsets; returns the slot index and
// the buffer start.
int stage_records(dfb_ctx* h, FragRec** out) {
  const int buf = h->hRecBuf;
  h->hRecBuf ^= 1;
  cudaEventSynchronize(h->hRecDone[buf]);  // its previous upload has finished
  int st = grow_staging(h, buf, h->recs.size());
  if (st != DFB_OK) return st;
  const size_t n = h->recs.size();
  FragRec* dst = reinterpret_cast<FragRec*>(h->hRecs[buf] + kHdrBytes);
  int* off = reinterpret_cast<int*>(h->hRecs[buf] + kHdrBytes + sizeof(FragRec) * n);
  group_by_tile(h->recs.data(), n, h->fragCount.data(), h->nTiles, 0, dst, off, h->tileCursor);
  *out = reinterpret_cast<FragRec*>(h->hRecs[buf]);
  return buf;
}

// Every entry point of the C ABI runs its body under this guard, so that no
// C++ exception crosses the interface: a failed host allocation (a growing
// record list, tree or staging vector) returns DFB_ERR_OOM; no other
// exception is thrown by this library, and one from elsewhere returns
// DFB_ERR_STATE.
template <typename F>
int guarded(F&& body) noexcept {
  try {
    return body();
  } catch (const std::bad_alloc&) {
    return DFB_ERR_OOM;
  } catch (const std::length_error&) {
    return DFB_ERR_OOM;
  } catch (...) {
    return DFB_ERR_STATE;
  }
}

}  // namespace

// ============================================================================
// C ABI
// ============================================================================
extern "C" {

const char* dfb_error_string(int s) {
  switch (s) {
    case DFB_OK: return "ok";
    case DFB_ERR_INVALID_ARG: return "invalid argument";
    case DFB_ERR_TILE_RANGE: return "tile id out of range";
    case DFB_ERR_STATE: return "call not allowed in the current state";
    case DFB_ERR_INCOMPLETE: return "tile dependency tree incomplete";
    case DFB_ERR_OOM: return "out of memory";
    case DFB_ERR_TIMEOUT: return "device wait timed out";
    case DFB_ERR_CUDA: return "CUDA error";
    case DFB_ERR_CAPACITY: return "request exceeds the fixed scratch of dfb_composite_noalloc";
    case DFB_ERR_CHECK: return "device-side check failed (checked build)";
    default: return "unknown status";
  }
}

int dfb_version(void) { return kVersion; }

int dfb_create_ex(const dfb_config* cfg, dfb_handle* out) {
  return guarded([&]() -> int {
    if (!cfg || !out) return DFB_ERR_INVALID_ARG;
    *out = nullptr;
    const int T = cfg->tile_size;
    if (cfg->width < 1 || cfg->height < 1 || !is_pow2(T) || T < 4 || T > 256)
      return DFB_ERR_INVALID_ARG;
    if ((int64_t)cfg->width * cfg->height > (int64_t)1 << 31) return DFB_ERR_INVALID_ARG;
    // the kernels index the tile-major state (whole tiles) with 32 bits
    if ((int64_t)((cfg->width + T - 1) / T) * ((cfg->height + T - 1) / T) * T * T > (int64_t)1 << 32)
      return DFB_ERR_INVALID_ARG;
    if (cfg->mode < DFB_BLEND_DEPTH || cfg->mode > DFB_AVERAGE) return DFB_ERR_INVALID_ARG;
    if (cfg->dtype < DFB_F32 || cfg->dtype > DFB_FP8E4M3) return DFB_ERR_INVALID_ARG;
    if (cfg->flags & ~(DFB_FLAG_ACCUMULATE | DFB_FLAG_WRITE_COLOR | DFB_FLAG_PACK_RGBA8 |
                       DFB_FLAG_DEFER_ALLOC))
      return DFB_ERR_INVALID_ARG;
    dfb_ctx* h = new (std::nothrow) dfb_ctx();
    if (!h) return DFB_ERR_OOM;
    h->cfg = *cfg;
    if (h->cfg.kahan_after <= 0) h->cfg.kahan_after = 256;
    h->tilesX = (cfg->width + T - 1) / T;
    h->tilesY = (cfg->height + T - 1) / T;
    h->nTiles = h->tilesX * h->tilesY;
    h->logT = ilog2(T);
    h->tilePixels = T * T;
    h->chunks = h->tilePixels < dfb::kItemPixels ? 1 : h->tilePixels / dfb::kItemPixels;
    h->rgbaBytes = (size_t)h->tilePixels * 4 * elt_bytes(cfg->dtype);
    h->depthBytes = (size_t)h->tilePixels * 4;
    try {
      h->declared.assign(h->nTiles, -1);
      h->recvGen1.assign(h->nTiles, 0);
      h->childGen1.assign(h->nTiles, 0);
      h->fragCount.assign(h->nTiles, 0);
    } catch (...) {
      delete h;
      throw;
    }
    if (!(cfg->flags & DFB_FLAG_DEFER_ALLOC)) {
      const int st = allocate(h);
      if (st != DFB_OK) {
        free_device(h);
        delete h;
        return st;
      }
    }
    *out = h;
    return DFB_OK;
  });
}

int dfb_create(int width, int height, int tile_size, int mode, dfb_handle* out) {
  return guarded([&]() -> int {
    dfb_config c{};
    c.width = width;
    c.height = height;
    c.tile_size = tile_size;
    c.mode = mode;
    c.dtype = DFB_F32;
    c.flags = DFB_FLAGS_DEFAULT;
    return dfb_create_ex(&c, out);
  });
}

int dfb_destroy(dfb_handle h) {
  return guarded([&]() -> int {
    if (!h) return DFB_OK;
    if (h->allocated && h->lastStreamSet) cudaEventSynchronize(h->frameDone);
    free_device(h);
    if (h->curve) cudaFree(h->curve);
    delete h;
    return DFB_OK;
  });
}

int dfb_set_background(dfb_handle h, float r, float g, float b, float a) {
  return guarded([&]() -> int {
    if (!h) return DFB_ERR_INVALID_ARG;
    if (!isfinite(r) || !isfinite(g) || !isfinite(b) || !isfinite(a)) return DFB_ERR_INVALID_ARG;
    h->bg[0] = r; h->bg[1] = g; h->bg[2] = b; h->bg[3] = a;
    return DFB_OK;
  });
}

int dfb_set_pixel_op(dfb_handle h, int op, float exposure) {
  return guarded([&]() -> int {
    if (!h) return DFB_ERR_INVALID_ARG;
    if (op < DFB_PIXELOP_NONE || op > DFB_PIXELOP_CURVE) return DFB_ERR_INVALID_ARG;
    if (!isfinite(exposure) || exposure < 0.0f) return DFB_ERR_INVALID_ARG;
    if (op == DFB_PIXELOP_CURVE && !h->curve) return DFB_ERR_STATE;
    h->pixelOp = op;
    h->exposure = exposure;
    return DFB_OK;
  });
}

int dfb_set_pixel_curve(dfb_handle h, const float* curves, int n, float x_max) {
  return guarded([&]() -> int {
    if (!h || !curves || n < 2 || n > dfb::kMaxCurve) return DFB_ERR_INVALID_ARG;
    if (!isfinite(x_max) || x_max <= 0.0f) return DFB_ERR_INVALID_ARG;
    for (int i = 0; i < 3 * n; ++i)
      if (!isfinite(curves[i])) return DFB_ERR_INVALID_ARG;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return DFB_ERR_CUDA;
    if ((h->allocated && dev != h->device) || (h->curve && dev != h->curveDevice))
      return DFB_ERR_STATE;
    if (!h->curve) {
      e = cudaMalloc(&h->curve, sizeof(float) * 3 * (size_t)dfb::kMaxCurve);
      if (e != cudaSuccess) {
        h->curve = nullptr;
        return e == cudaErrorMemoryAllocation ? DFB_ERR_OOM : DFB_ERR_CUDA;
      }
      h->curveDevice = dev;
    } else if (h->allocated && h->lastStreamSet) {
      // frames in flight may still read the previous samples
      e = cudaEventSynchronize(h->frameDone);
      if (e != cudaSuccess) return DFB_ERR_CUDA;
    }
    // the legacy stream, waited for: the DMA of a pageable source has landed
    // when the call returns
    e = cudaMemcpyAsync(h->curve, curves, sizeof(float) * 3 * (size_t)n, cudaMemcpyHostToDevice, 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(0);
    if (e != cudaSuccess) return DFB_ERR_CUDA;
    h->curveN = n;
    h->curveXMax = x_max;
    h->pixelOp = DFB_PIXELOP_CURVE;
    return DFB_OK;
  });
}

int dfb_begin_frame(dfb_handle h, int accumulate) {
  return guarded([&]() -> int {
    if (!h) return DFB_ERR_INVALID_ARG;
    if (h->inFrame) return DFB_ERR_STATE;
    h->inFrame = true;
    h->recs.clear();
    std::fill(h->declared.begin(), h->declared.end(), -1);
    std::fill(h->recvGen1.begin(), h->recvGen1.end(), 0);
    std::fill(h->childGen1.begin(), h->childGen1.end(), 0);
    for (int t : h->touchedDeeper) h->deeper[t].clear();
    h->touchedDeeper.clear();
    std::fill(h->fragCount.begin(), h->fragCount.end(), 0);
    h->longTiles.clear();
    h->hostCopies = false;
    h->arenaIdx ^= 1;
    h->arenas[h->arenaIdx].reset();
    const bool acc = (h->cfg.flags & DFB_FLAG_ACCUMULATE) && accumulate && h->accumN > 0;
    h->pendingN = acc ? h->accumN + 1 : 1;
    h->pendingStats = dfb_frame_stats{};
    return DFB_OK;
  });
}

int dfb_set_tile_children(dfb_handle h, int tile_id, int n_children) {
  return guarded([&]() -> int {
    if (!h) return DFB_ERR_INVALID_ARG;
    if (!h->inFrame) return DFB_ERR_STATE;
    if (tile_id < 0 || tile_id >= h->nTiles) return DFB_ERR_TILE_RANGE;
    if (n_children < 0) return DFB_ERR_INVALID_ARG;
    if (h->declared[tile_id] >= 0) return DFB_ERR_STATE;
    h->declared[tile_id] = n_children;
    return DFB_OK;
  });
}

int dfb_submit_tile_ex(dfb_handle h, const dfb_tile_desc* tile) {
  return guarded([&]() -> int {
    if (!h) return DFB_ERR_INVALID_ARG;
    if (!h->inFrame) return DFB_ERR_STATE;
    const int st = validate_tile(h, tile);
    if (st != DFB_OK) return st;
    return append_records(h, 1, tile, DFB_PTR_AUTO);
  });
}

int dfb_submit_tile(dfb_handle h, int tile_id, float order_key, const void* rgba,
                    const float* depth) {
  return guarded([&]() -> int {
    dfb_tile_desc t;
    t.tile_id = tile_id;
    t.order_key = order_key;
    t.rgba = rgba;
    t.depth = depth;
    t.scale = 1.0f;
    t.generation = 1;
    t.children = 0;
    if (h && h->cfg.dtype == DFB_FP8E4M3) return DFB_ERR_INVALID_ARG;  // needs a scale
    return dfb_submit_tile_ex(h, &t);
  });
}

int dfb_submit_tiles(dfb_handle h, int n, const int* tile_ids, const float* order_keys,
                     const void* const* rgba, const float* const* depth, const float* scales,
                     int where) {
  return guarded([&]() -> int {
    if (!h || n < 0) return DFB_ERR_INVALID_ARG;
    if (!h->inFrame) return DFB_ERR_STATE;
    if (n == 0) return DFB_OK;
    if (where < DFB_PTR_AUTO || where > DFB_PTR_HOST_BORROWED) return DFB_ERR_INVALID_ARG;
    // validate everything first: nothing is submitted if an entry is bad
    const int st = validate_arrays(h, n, tile_ids, order_keys, rgba, depth, scales);
    if (st != DFB_OK) return st;
    if (where != DFB_PTR_DEVICE) {
      std::vector<dfb_tile_desc> ts((size_t)n);
      for (int i = 0; i < n; ++i)
        ts[i] = dfb_tile_desc{tile_ids[i], order_keys[i], rgba[i], depth[i],
                              scales ? scales[i] : 1.0f, 1, 0};
      return append_records(h, n, ts.data(), where);
    }
    // device pointers: append directly
    const size_t base = h->recs.size();
    h->recs.resize(base + (size_t)n);
    const int64_t fpx = build_records(h, n, tile_ids, order_keys, rgba, depth, scales,
                                      h->recs.data() + base, h->recvGen1.data());
    for (int i = 0; i < n; ++i) count_frags(h, tile_ids[i], 1);
    h->pendingStats.fragments += n;
    h->pendingStats.fragment_pixels += fpx;
    return DFB_OK;
  });
}

int dfb_submit_tiles_ex(dfb_handle h, int n, const dfb_tile_desc* tiles, int where) {
  return guarded([&]() -> int {
    if (!h || n < 0) return DFB_ERR_INVALID_ARG;
    if (!h->inFrame) return DFB_ERR_STATE;
    if (n == 0) return DFB_OK;
    if (!tiles || where < DFB_PTR_AUTO || where > DFB_PTR_HOST_BORROWED) return DFB_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i) {
      const int st = validate_tile(h, &tiles[i]);
      if (st != DFB_OK) return st;
    }
    return append_records(h, n, tiles, where);
  });
}

int dfb_end_frame(dfb_handle h, void* stream) {
  return guarded([&]() -> int {
    if (!h) return DFB_ERR_INVALID_ARG;
    return dfb_end_frames(&h, 1, stream);
  });
}

}  // extern "C"

// ---- batched end-of-frame: shared by dfb_end_frame (n = 1) -----------------
namespace {

struct BatchRes {
  // Resources of one multi-frame launch; each device has two, used by
  // alternate launches, so the bucketing of the next batch (on a side
  // stream) overlaps the composite of the current one.
  FragRec* dRecs = nullptr;       // records grouped by global tile
  FragRec* srecs = nullptr;
  size_t recCap = 0;
  dfb::TileBlock* blocks = nullptr;
  int* dOff = nullptr;            // tile offsets of dRecs (tiles + 1)
  int* hOff = nullptr;
  size_t tileCap = 0;
  int* redo = nullptr;            // re-do list of the composite: [count, units...]
  size_t redoCap = 0;
  std::vector<int> counts;        // records per global tile (host)
  std::vector<int> cursor;        // host scratch of the grouping
  FrameArgs* dFrames = nullptr;
  int* dItemBase = nullptr;
  size_t frameCap = 0;
  FragRec* hRecs = nullptr;
  FrameArgs* hFrames = nullptr;
  int* hItemBase = nullptr;
  cudaEvent_t ready = nullptr;     // the bucketing into this set has finished
  cudaEvent_t released = nullptr;  // the composite that read this set has finished
  bool used = false;
};

struct BatchDev {
  BatchRes sets[2];
  int idx = 0;
  cudaStream_t side = nullptr;
};

std::mutex g_batch_mu;
BatchDev g_batch[64];

int batch_reserve(BatchRes& b, size_t nRec, size_t nTiles, size_t nFrames, size_t redoUnits) {
  cudaError_t e = cudaSuccess;
  if (!b.ready) {
    e = cudaEventCreateWithFlags(&b.ready, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b.released, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_status(e);
  }
  // The launch that last used this set has finished with its host and device
  // arrays (its uploads and bucketing precede its composite).
  if (b.used) cudaEventSynchronize(b.released);
  if (nRec > b.recCap) {
    size_t cap = b.recCap ? b.recCap : 4096;
    while (cap < nRec) cap *= 2;
    cudaFree(b.dRecs); cudaFree(b.srecs); cudaFreeHost(b.hRecs);
    b.dRecs = nullptr; b.srecs = nullptr; b.hRecs = nullptr; b.recCap = 0;
    e = dalloc(&b.dRecs, cap);
    if (e == cudaSuccess) e = dalloc(&b.srecs, cap);
    if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&b.hRecs), sizeof(FragRec) * cap);
    if (e != cudaSuccess) return cuda_status(e);
    b.recCap = cap;
  }
  if (nTiles > b.tileCap) {
    size_t cap = b.tileCap ? b.tileCap : 4096;
    while (cap < nTiles) cap *= 2;
    cudaFree(b.blocks); cudaFree(b.dOff); cudaFreeHost(b.hOff);
    b.blocks = nullptr; b.dOff = b.hOff = nullptr; b.tileCap = 0;
    e = dalloc(&b.blocks, cap);
    if (e == cudaSuccess) e = dalloc(&b.dOff, cap + 1);
    if (e == cudaSuccess)
      e = cudaMallocHost(reinterpret_cast<void**>(&b.hOff), sizeof(int) * (cap + 1));
    if (e != cudaSuccess) return cuda_status(e);
    b.tileCap = cap;
  }
  if (redoUnits + 1 > b.redoCap) {
    size_t cap = b.redoCap ? b.redoCap : 4096;
    while (cap < redoUnits + 1) cap *= 2;
    cudaFree(b.redo);
    b.redo = nullptr;
    b.redoCap = 0;
    e = dalloc(&b.redo, cap);
    if (e != cudaSuccess) return cuda_status(e);
    b.redoCap = cap;
  }
  if (nFrames > b.frameCap) {
    size_t cap = b.frameCap ? b.frameCap : 64;
    while (cap < nFrames) cap *= 2;
    cudaFree(b.dFrames); cudaFree(b.dItemBase); cudaFreeHost(b.hFrames); cudaFreeHost(b.hItemBase);
    b.dFrames = nullptr; b.dItemBase = nullptr; b.hFrames = nullptr; b.hItemBase = nullptr;
    b.frameCap = 0;
    e = dalloc(&b.dFrames, cap);
    if (e == cudaSuccess) e = dalloc(&b.dItemBase, cap + 1);
    if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&b.hFrames), sizeof(FrameArgs) * cap);
    if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&b.hItemBase), sizeof(int) * (cap + 1));
    if (e != cudaSuccess) return cuda_status(e);
    b.frameCap = cap;
  }
  return DFB_OK;
}

constexpr size_t kTimingSlots = 128;

// Fold the oldest recorded slot into the running sums (waits for it).
int harvest_one(dfb_ctx* h) {
  const size_t slot = (h->tHead + kTimingSlots - h->tCount) % kTimingSlots;
  cudaEvent_t* e = &h->tev[4 * slot];
  cudaError_t r = cudaEventSynchronize(e[3]);
  float b = 0.f, c = 0.f;
  if (r == cudaSuccess) r = cudaEventSynchronize(e[1]);
  if (r == cudaSuccess) r = cudaEventElapsedTime(&b, e[0], e[1]);
  if (r == cudaSuccess) r = cudaEventElapsedTime(&c, e[2], e[3]);
  if (r != cudaSuccess) return cuda_status(r);
  h->tSum.launches += 1;
  h->tSum.bucket_ms += b;
  h->tSum.composite_ms += c;
  h->tCount -= 1;
  return DFB_OK;
}

// Events of the next timing slot, or null when timing is off.
cudaEvent_t* timing_slot(dfb_ctx* h) {
  if (!h->timing) return nullptr;
  if (h->tev.empty()) {
    h->tev.assign(4 * kTimingSlots, nullptr);
    for (auto& e : h->tev)
      if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  }
  if (h->tCount == kTimingSlots && harvest_one(h) != DFB_OK) return nullptr;
  cudaEvent_t* e = &h->tev[4 * h->tHead];
  h->tHead = (h->tHead + 1) % kTimingSlots;
  h->tCount += 1;
  return e;
}

// After the last frame's work has finished: report (and clear) a timed-out
// device-side wait of the launch that served this handle.
int take_device_error(dfb_ctx* h) {
  if (!h->lastErr) return DFB_OK;
  unsigned v = 0;
  cudaError_t e = cudaMemcpy(&v, h->lastErr, sizeof(unsigned), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_status(e);
  if (!v) return DFB_OK;
  e = cudaMemset(h->lastErr, 0, sizeof(unsigned));
  if (e != cudaSuccess) return cuda_status(e);
  return (v & dfb::kErrCheck) ? DFB_ERR_CHECK : DFB_ERR_TIMEOUT;
}

int end_one(dfb_ctx* h, cudaStream_t s) {
  FragRec* staged = nullptr;
  int st = grow_records(h, h->recs.size());
  if (st != DFB_OK) return st;
  const int buf = stage_records(h, &staged);
  if (buf < 0) return buf;
  BucketSet& b = h->sets[h->setIdx];
  h->setIdx ^= 1;
  const size_t n = h->recs.size();
  // header: the frame's arguments + the item prefix of a one-frame launch
  FrameHeader* hdr = reinterpret_cast<FrameHeader*>(staged);
  fill_frame_args(h, hdr->fa, 0, b.srecs, b.blocks);
  hdr->itemBase[0] = 0;
  hdr->itemBase[1] = h->nTiles * hdr->fa.chunks;
  const int items = hdr->itemBase[1];
  FrameArgs* dFa = reinterpret_cast<FrameArgs*>(b.dStage);
  const int* dItemBase = reinterpret_cast<const int*>(b.dStage + offsetof(FrameHeader, itemBase));
  const int* dTileOff = reinterpret_cast<const int*>(b.dStage + kHdrBytes + sizeof(FragRec) * n);
  // only BLEND_DEPTH items can need the exact re-do kernel
  const int nLong = h->cfg.mode == DFB_BLEND_DEPTH ? (int)h->longTiles.size() : 0;
  dfb::LongList lng;
  lng.items = nLong * h->chunks;
  for (int t : h->longTiles) lng.maxFragments = std::max(lng.maxFragments, h->fragCount[t]);
  // The bucketing reads only library-owned buffers, so it runs on the side
  // stream, overlapping the previous frame's composite (dfb_end_frames has
  // refused a capturing stream).
  cudaError_t e = cudaSuccess;
  cudaStream_t bs = h->bucketStream;
  if (h->lastStreamSet && h->lastStream != s) e = cudaStreamWaitEvent(s, h->frameDone, 0);
  if (e == cudaSuccess && b.used) e = cudaStreamWaitEvent(bs, b.released, 0);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b.dStage, staged, stage_bytes(h, n), cudaMemcpyHostToDevice, bs);
  if (e == cudaSuccess) e = cudaEventRecord(h->hRecDone[buf], bs);
  cudaEvent_t* ev = timing_slot(h);
  if (e == cudaSuccess && ev) e = cudaEventRecord(ev[0], bs);
  if (e == cudaSuccess)
    e = dfb::launch_bucket(b.dRecs, dTileOff, h->nTiles, b.srecs, b.blocks, b.redo, bs);
  if (e == cudaSuccess && ev) e = cudaEventRecord(ev[1], bs);
  if (e == cudaSuccess) e = cudaEventRecord(b.ready, bs);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b.ready, 0);
  if (e == cudaSuccess && h->hostCopies) e = cudaStreamWaitEvent(s, h->copyDone, 0);
  if (e == cudaSuccess && ev) e = cudaEventRecord(ev[2], s);
  if (e == cudaSuccess)
    e = dfb::launch_composite(dFa, dItemBase, 1, items, h->nTiles,
                              (h->cfg.flags & DFB_FLAG_ACCUMULATE) != 0, h->cfg.dtype,
                              tune_of(h, n, (size_t)h->nTiles),
                              ctl_of(h, b.redo), lng, &hdr->fa, hdr->itemBase,
                              ev ? ev[3] : nullptr, s);
  if (e == cudaSuccess) e = cudaEventRecord(b.released, s);
  if (e == cudaSuccess) e = cudaEventRecord(h->frameDone, s);
  b.used = true;
  h->launches += 1 + ((h->cfg.flags & DFB_FLAG_ACCUMULATE) ? 2 : 1) + (nLong ? 1 : 0);
  h->lastErr = h->errFlag;
  h->stallItem = -1;
  return cuda_status(e);
}

int end_batch(dfb_ctx* const* hs, int n, cudaStream_t s) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev >= 64) return DFB_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_batch_mu);
  BatchDev& bd = g_batch[dev];
  if (!bd.side && cudaStreamCreateWithFlags(&bd.side, cudaStreamNonBlocking) != cudaSuccess) {
    bd.side = nullptr;
    return DFB_ERR_CUDA;
  }
  BatchRes& b = bd.sets[bd.idx];
  bd.idx ^= 1;
  size_t nRec = 0, nTiles = 0, nItems = 0;
  for (int i = 0; i < n; ++i) {
    nRec += hs[i]->recs.size();
    nTiles += (size_t)hs[i]->nTiles;
    nItems += (size_t)hs[i]->nTiles * hs[i]->chunks;
  }
  int st = batch_reserve(b, nRec, nTiles, (size_t)n, nItems * (dfb::kItemPixels / 32));
  if (st != DFB_OK) return st;
  cudaError_t e = cudaSuccess;
  int tileBase = 0, items = 0;
  dfb::LongList lng;
  const int dtype = hs[0]->cfg.dtype;
  bool anyAcc = false;
  // per-global-tile counts, then every frame's records grouped by global tile
  b.counts.resize(nTiles);
  for (int i = 0; i < n; ++i) {
    const dfb_ctx* h = hs[i];
    std::copy(h->fragCount.begin(), h->fragCount.end(), b.counts.begin() + tileBase);
    tileBase += h->nTiles;
  }
  b.cursor.resize(nTiles);
  {
    int acc = 0;
    for (size_t t = 0; t < nTiles; ++t) {
      b.hOff[t] = acc;
      b.cursor[t] = acc;
      acc += b.counts[t];
    }
    b.hOff[nTiles] = acc;
  }
  tileBase = 0;
  for (int i = 0; i < n; ++i) {
    dfb_ctx* h = hs[i];
    anyAcc |= (h->cfg.flags & DFB_FLAG_ACCUMULATE) != 0;
    for (const FragRec& fr : h->recs) {
      FragRec g = fr;
      g.tile += (uint32_t)tileBase;
      g.frame = (uint32_t)i;
      b.hRecs[b.cursor[g.tile]++] = g;
    }
    if (h->cfg.mode == DFB_BLEND_DEPTH) lng.items += (int)h->longTiles.size() * h->chunks;
    for (int t : h->longTiles) lng.maxFragments = std::max(lng.maxFragments, h->fragCount[t]);
    fill_frame_args(h, b.hFrames[i], tileBase, b.srecs, b.blocks);
    b.hItemBase[i] = items;
    items += h->nTiles * b.hFrames[i].chunks;
    tileBase += h->nTiles;
    if (h->lastStreamSet && h->lastStream != s && e == cudaSuccess)
      e = cudaStreamWaitEvent(s, h->frameDone, 0);
    if (h->hostCopies && e == cudaSuccess) e = cudaStreamWaitEvent(s, h->copyDone, 0);
  }
  b.hItemBase[n] = items;
  // Uploads and bucketing touch only this set, so they run on the device's
  // side stream, overlapping earlier work on `s`.
  cudaStream_t bs = bd.side;
  if (e == cudaSuccess && b.used) e = cudaStreamWaitEvent(bs, b.released, 0);
  if (e == cudaSuccess && nRec)
    e = cudaMemcpyAsync(b.dRecs, b.hRecs, sizeof(FragRec) * nRec, cudaMemcpyHostToDevice, bs);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b.dOff, b.hOff, sizeof(int) * (nTiles + 1), cudaMemcpyHostToDevice, bs);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b.dFrames, b.hFrames, sizeof(FrameArgs) * n, cudaMemcpyHostToDevice, bs);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b.dItemBase, b.hItemBase, sizeof(int) * (n + 1), cudaMemcpyHostToDevice,
                        bs);
  cudaEvent_t* ev = timing_slot(hs[0]);
  if (e == cudaSuccess && ev) e = cudaEventRecord(ev[0], bs);
  if (e == cudaSuccess)
    e = dfb::launch_bucket(b.dRecs, b.dOff, (int)nTiles, b.srecs, b.blocks, b.redo, bs);
  if (e == cudaSuccess && ev) e = cudaEventRecord(ev[1], bs);
  if (e == cudaSuccess) e = cudaEventRecord(b.ready, bs);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b.ready, 0);
  if (e == cudaSuccess && ev) e = cudaEventRecord(ev[2], s);
  if (e == cudaSuccess)
    e = dfb::launch_composite(b.dFrames, b.dItemBase, n, items, tileBase, anyAcc, dtype,
                              tune_of(hs[0], nRec, nTiles), ctl_of(hs[0], b.redo), lng, b.hFrames,
                              b.hItemBase,
                              ev ? ev[3] : nullptr, s);
  if (e == cudaSuccess) e = cudaEventRecord(b.released, s);
  b.used = true;
  hs[0]->launches += 1 + (anyAcc ? 2 : 1) + (lng.items ? 1 : 0);
  hs[0]->stallItem = -1;
  for (int i = 0; i < n && e == cudaSuccess; ++i) {
    e = cudaEventRecord(hs[i]->frameDone, s);
    hs[i]->lastErr = hs[0]->errFlag;
  }
  return cuda_status(e);
}

}  // namespace

extern "C" {

int dfb_end_frames(const dfb_handle* hs, int n, void* stream) {
  return guarded([&]() -> int {
    if (!hs || n < 1) return DFB_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i) {
      if (!hs[i]) return DFB_ERR_INVALID_ARG;
      for (int j = 0; j < i; ++j)
        if (hs[j] == hs[i]) return DFB_ERR_INVALID_ARG;
      if (!hs[i]->inFrame) return DFB_ERR_STATE;
      if (n > 1 && hs[i]->cfg.dtype != hs[0]->cfg.dtype) return DFB_ERR_INVALID_ARG;
    }
    for (int i = 0; i < n; ++i) {
      const int st = check_trees(hs[i]);
      if (st != DFB_OK) return st;
    }
    cudaStream_t s = (cudaStream_t)stream;
    {
      // A captured end of frame would replay an upload from a staging buffer
      // that later frames overwrite: refused (dfb_graph_* captures batches).
      cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
      if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) cudaGetLastError();
      else if (cap != cudaStreamCaptureStatusNone) return DFB_ERR_STATE;
    }
    for (int i = 0; i < n; ++i) {
      const int st = allocate(hs[i]);
      if (st != DFB_OK) return st;
    }
    const int st = n == 1 ? end_one(hs[0], s) : end_batch(hs, n, s);
    if (st != DFB_OK) return st;
    for (int i = 0; i < n; ++i) {
      dfb_ctx* h = hs[i];
      if (h->hostCopies) {
        cudaEventRecord(h->arenaFree[h->arenaIdx], s);
        h->arenaUsed[h->arenaIdx] = true;
      }
      finish_stats(h);
      h->stats = h->pendingStats;
      h->accumN = h->pendingN;
      h->inFrame = false;
      h->haveFrame = true;
      h->lastStream = s;
      h->lastStreamSet = true;
    }
    return DFB_OK;
  });
}

int dfb_sync(dfb_handle h) {
  return guarded([&]() -> int {
    if (!h) return DFB_ERR_INVALID_ARG;
    if (!h->lastStreamSet) return DFB_OK;
    const int st = cuda_status(cudaEventSynchronize(h->frameDone));
    return st != DFB_OK ? st : take_device_error(h);
  });
}

}  // extern "C"

namespace {

// Copy `bytes` from device buffer `src` to `out` (host or device) after the
// last frame; host destinations wait for completion.
int copy_out(dfb_ctx* h, void* out, const void* src, size_t bytes) {
  cudaStream_t s = h->lastStream;
  const bool dev = is_device_ptr(out);
  cudaError_t e = cudaMemcpyAsync(out, src, bytes, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && !dev) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_status(e);
  return dev ? DFB_OK : take_device_error(h);
}

int ensure_read_tmp(dfb_ctx* h) {
  if (h->readTmp) return DFB_OK;
  return cuda_status(dalloc(&h->readTmp, (size_t)h->cfg.width * h->cfg.height));
}

}  // namespace

extern "C" {

int dfb_read_color(dfb_handle h, float* out) {
  return guarded([&]() -> int {
    if (!h || !out) return DFB_ERR_INVALID_ARG;
    if (!h->haveFrame || !(h->cfg.flags & DFB_FLAG_WRITE_COLOR)) return DFB_ERR_STATE;
    return copy_out(h, out, h->color, sizeof(float4) * (size_t)h->cfg.width * h->cfg.height);
  });
}

int dfb_read_rgba8(dfb_handle h, uint32_t* out) {
  return guarded([&]() -> int {
    if (!h || !out) return DFB_ERR_INVALID_ARG;
    if (!h->haveFrame || !(h->cfg.flags & DFB_FLAG_PACK_RGBA8)) return DFB_ERR_STATE;
    return copy_out(h, out, h->rgba8, sizeof(uint32_t) * (size_t)h->cfg.width * h->cfg.height);
  });
}

int dfb_read_accum(dfb_handle h, float* out) {
  return guarded([&]() -> int {
    if (!h || !out) return DFB_ERR_INVALID_ARG;
    if (!h->haveFrame || !(h->cfg.flags & DFB_FLAG_ACCUMULATE)) return DFB_ERR_STATE;
    const int64_t px = (int64_t)h->cfg.width * h->cfg.height;
    const bool dev = is_device_ptr(out);
    float4* dst = (float4*)out;
    if (!dev) {
      const int st = ensure_read_tmp(h);
      if (st != DFB_OK) return st;
      dst = h->readTmp;
    }
    const int n = h->accumN;
    cudaError_t e = dfb::launch_tiles_to_image(h->accum, n > h->cfg.kahan_after ? h->comp : nullptr,
                                               1.0f / (float)n, dst, h->cfg.width, h->cfg.height,
                                               h->cfg.tile_size, h->lastStream);
    if (e != cudaSuccess) return cuda_status(e);
    if (dev) return DFB_OK;
    return copy_out(h, out, h->readTmp, sizeof(float4) * (size_t)px);
  });
}

int dfb_read_variance(dfb_handle h, float* per_pixel, float* per_tile) {
  return guarded([&]() -> int {
    if (!h) return DFB_ERR_INVALID_ARG;
    if (!h->haveFrame || !(h->cfg.flags & DFB_FLAG_ACCUMULATE)) return DFB_ERR_STATE;
    const int64_t px = (int64_t)h->cfg.width * h->cfg.height;
    const int n = h->accumN;
    const float invNm1 = n > 1 ? 1.0f / (float)(n - 1) : 0.0f;
    if (per_pixel) {
      const bool dev = is_device_ptr(per_pixel);
      float4* dst = (float4*)per_pixel;
      if (!dev) {
        const int st = ensure_read_tmp(h);
        if (st != DFB_OK) return st;
        dst = h->readTmp;
      }
      cudaError_t e = dfb::launch_tiles_to_image(h->m2, nullptr, invNm1, dst, h->cfg.width,
                                                 h->cfg.height, h->cfg.tile_size, h->lastStream);
      if (e != cudaSuccess) return cuda_status(e);
      if (!dev) {
        const int st = copy_out(h, per_pixel, h->readTmp, sizeof(float4) * (size_t)px);
        if (st != DFB_OK) return st;
      }
    }
    if (per_tile) return copy_out(h, per_tile, h->tileVar, sizeof(float) * h->nTiles);
    return DFB_OK;
  });
}

int dfb_get_stats(dfb_handle h, dfb_frame_stats* out) {
  return guarded([&]() -> int {
    if (!h || !out) return DFB_ERR_INVALID_ARG;
    *out = h->stats;
    return DFB_OK;
  });
}

int dfb_get_tiles(dfb_handle h, int* tiles_x, int* tiles_y) {
  return guarded([&]() -> int {
    if (!h || !tiles_x || !tiles_y) return DFB_ERR_INVALID_ARG;
    *tiles_x = h->tilesX;
    *tiles_y = h->tilesY;
    return DFB_OK;
  });
}

// Tile-major state buffer -> caller's row-major image (host or device).
int state_out(dfb_ctx* h, float* out, const float4* src) {
  const bool dev = is_device_ptr(out);
  float4* dst = dev ? reinterpret_cast<float4*>(out) : nullptr;
  if (!dev) {
    const int st = ensure_read_tmp(h);
    if (st != DFB_OK) return st;
    dst = h->readTmp;
  }
  cudaError_t e = dfb::launch_tiles_to_image(src, nullptr, 1.0f, dst, h->cfg.width, h->cfg.height,
                                             h->cfg.tile_size, h->lastStream);
  if (e != cudaSuccess) return cuda_status(e);
  if (dev) return DFB_OK;
  return copy_out(h, out, h->readTmp, sizeof(float4) * (size_t)h->cfg.width * h->cfg.height);
}

int dfb_save_accum(dfb_handle h, float* sum, float* comp, float* m2, int* frames) {
  return guarded([&]() -> int {
    if (!h || !sum || !comp || !m2 || !frames) return DFB_ERR_INVALID_ARG;
    if (!h->haveFrame || !(h->cfg.flags & DFB_FLAG_ACCUMULATE)) return DFB_ERR_STATE;
    const size_t bytes = sizeof(float4) * (size_t)h->cfg.width * h->cfg.height;
    int st = state_out(h, sum, h->accum);
    if (st == DFB_OK) {
      if (h->accumN > h->cfg.kahan_after) st = state_out(h, comp, h->comp);
      else {
        const bool dev = is_device_ptr(comp);
        if (dev) st = cuda_status(cudaMemsetAsync(comp, 0, bytes, h->lastStream));
        else memset(comp, 0, bytes);
      }
    }
    if (st == DFB_OK) st = state_out(h, m2, h->m2);
    if (st == DFB_OK) *frames = h->accumN;
    return st;
  });
}

int dfb_load_accum(dfb_handle h, const float* sum, const float* comp, const float* m2,
                   int frames) {
  return guarded([&]() -> int {
    if (!h || !sum || !comp || !m2 || frames < 1) return DFB_ERR_INVALID_ARG;
    if (h->inFrame || !(h->cfg.flags & DFB_FLAG_ACCUMULATE)) return DFB_ERR_STATE;
    int st = allocate(h);
    if (st == DFB_OK) st = ensure_read_tmp(h);
    if (st != DFB_OK) return st;
    const size_t bytes = sizeof(float4) * (size_t)h->cfg.width * h->cfg.height;
    cudaStream_t s = h->lastStreamSet ? h->lastStream : (cudaStream_t)0;
    const float* srcs[3] = {sum, comp, m2};
    float4* dsts[3] = {h->accum, h->comp, h->m2};
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 3 && e == cudaSuccess; ++i) {
      e = cudaMemcpyAsync(h->readTmp, srcs[i], bytes, cudaMemcpyDefault, s);
      if (e == cudaSuccess)
        e = dfb::launch_image_to_tiles(h->readTmp, dsts[i], h->cfg.width, h->cfg.height,
                                       h->cfg.tile_size, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e);
    h->accumN = frames;
    h->haveFrame = true;
    return DFB_OK;
  });
}

int dfb_convert_tiles(const float* src, void* dst, float* scales, int n_tiles, int tile_pixels,
                      int dtype, void* stream) {
  return guarded([&]() -> int {
    if (!src || !dst || n_tiles < 0 || tile_pixels < 1) return DFB_ERR_INVALID_ARG;
    if (dtype != DFB_F16 && dtype != DFB_BF16 && dtype != DFB_FP8E4M3) return DFB_ERR_INVALID_ARG;
    if (dtype == DFB_FP8E4M3 && !scales) return DFB_ERR_INVALID_ARG;
    if (n_tiles == 0) return DFB_OK;
    return cuda_status(dfb::launch_convert(src, dst, scales, n_tiles, tile_pixels, dtype,
                                           (cudaStream_t)stream));
  });
}

int dfb_set_timing(dfb_handle h, int enable) {
  return guarded([&]() -> int {
    if (!h) return DFB_ERR_INVALID_ARG;
    h->timing = enable != 0;
    return DFB_OK;
  });
}

int dfb_read_timing(dfb_handle h, dfb_timing* out, int reset) {
  return guarded([&]() -> int {
    if (!h || !out) return DFB_ERR_INVALID_ARG;
    while (h->tCount) {
      const int st = harvest_one(h);
      if (st != DFB_OK) return st;
    }
    *out = h->tSum;
    if (reset) h->tSum = dfb_timing{};
    return DFB_OK;
  });
}

int dfb_set_tuning(dfb_handle h, int ring_kb, int ctas_per_sm, int groups) {
  return guarded([&]() -> int {
    if (!h || !valid_tuning(ring_kb, ctas_per_sm, groups)) return DFB_ERR_INVALID_ARG;
    h->tune = dfb::TuneParams{ring_kb, ctas_per_sm, groups};
    return DFB_OK;
  });
}

int dfb_set_wait_limit(dfb_handle h, double seconds) {
  return guarded([&]() -> int {
    if (!h || !(seconds > 0.0) || seconds > 3600.0) return DFB_ERR_INVALID_ARG;
    h->waitNs = (unsigned long long)(seconds * 1e9);
    return DFB_OK;
  });
}

int dfb_inject_stall(dfb_handle h, int item) {
  return guarded([&]() -> int {
    if (!h || item < -1) return DFB_ERR_INVALID_ARG;
    h->stallItem = item;
    return DFB_OK;
  });
}

}  // extern "C"

// ============================================================================
// batched frames in a CUDA graph
// ============================================================================
struct dfb_graph_t {
  std::vector<dfb_ctx*> hs;
  int dtype = 0;
  bool anyAcc = false;
  int nRec = 0, nTiles = 0, items = 0;
  FragRec* dRecs = nullptr;        // records grouped by global tile
  int* dOff = nullptr;             // their tile offsets (nTiles + 1)
  FragRec* srecs = nullptr;
  dfb::TileBlock* blocks = nullptr;
  int* redo = nullptr;             // re-do list of the composite: [count, units...]
  FrameArgs* dFrames = nullptr;
  std::vector<FrameArgs> hostFrames;  // host copies of dFrames and dItemBase
  std::vector<int> hostItemBase;
  int* dItemBase = nullptr;
  dfb::LongList lng;
  unsigned* err = nullptr;
  dfb::TuneParams tune{0, 0, 0};
  cudaStream_t capStream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t done = nullptr;
  bool launched = false;
};

namespace {

void graph_release_capture(dfb_graph_t* g) {
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  g->exec = nullptr;
  g->graph = nullptr;
}

// (Re)capture the device work of the graph with its current tuning.
int graph_capture(dfb_graph_t* g) {
  graph_release_capture(g);
  const dfb::TuneParams tune =
      g->tune.ringKB ? g->tune
                     : dfb::default_tune(g->dtype, (double)g->nRec / (double)(g->nTiles ? g->nTiles : 1));
  // per-device launch set-up happens outside the capture (no work is enqueued)
  const dfb::LaunchCtl ctl{2000000000ull, -1, g->err, g->redo};
  cudaError_t e = dfb::launch_composite(g->dFrames, g->dItemBase, 1, 0, 0, false, g->dtype, tune,
                                        ctl, dfb::LongList{}, nullptr, nullptr, nullptr,
                                        g->capStream);
  if (e != cudaSuccess) return cuda_status(e);
  e = cudaStreamBeginCapture(g->capStream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_status(e);
  cudaError_t le = dfb::launch_bucket(g->dRecs, g->dOff, g->nTiles, g->srecs, g->blocks, g->redo,
                                      g->capStream);
  if (le == cudaSuccess)
    le = dfb::launch_composite(g->dFrames, g->dItemBase, (int)g->hs.size(), g->items, g->nTiles,
                               g->anyAcc, g->dtype, tune, ctl, g->lng, g->hostFrames.data(),
                               g->hostItemBase.data(), nullptr, g->capStream);
  e = cudaStreamEndCapture(g->capStream, &g->graph);
  if (le != cudaSuccess) return cuda_status(le);
  if (e != cudaSuccess) return cuda_status(e);
  e = cudaGraphInstantiate(&g->exec, g->graph, 0);
  return cuda_status(e);
}

void graph_free(dfb_graph_t* g) {
  if (g->launched && g->done) cudaEventSynchronize(g->done);
  graph_release_capture(g);
  cudaFree(g->dRecs); cudaFree(g->dOff); cudaFree(g->srecs); cudaFree(g->blocks);
  cudaFree(g->redo);
  cudaFree(g->dFrames); cudaFree(g->dItemBase); cudaFree(g->err);
  if (g->capStream) cudaStreamDestroy(g->capStream);
  if (g->done) cudaEventDestroy(g->done);
  delete g;
}

// The rest of dfb_graph_create once the graph object exists: record
// tables, device copies, capture.  Frees `g` on a returned error; an
// exception (a host vector that cannot grow) is the caller's to handle.
int graph_build(dfb_graph_t* g, const dfb_handle* hs, int n, dfb_graph* out) {
  g->hs.assign(hs, hs + n);
  g->dtype = hs[0]->cfg.dtype;
  std::vector<FrameArgs> fa((size_t)n);
  std::vector<int> itemBase((size_t)n + 1);
  std::vector<int> counts;  // records per global tile
  int tileBase = 0, items = 0, nRec = 0;
  for (int i = 0; i < n; ++i) {
    dfb_ctx* h = hs[i];
    g->anyAcc |= (h->cfg.flags & DFB_FLAG_ACCUMULATE) != 0;
    if (h->cfg.mode == DFB_BLEND_DEPTH) g->lng.items += (int)h->longTiles.size() * h->chunks;
    for (int t : h->longTiles) g->lng.maxFragments = std::max(g->lng.maxFragments, h->fragCount[t]);
    counts.insert(counts.end(), h->fragCount.begin(), h->fragCount.end());
    nRec += (int)h->recs.size();
    items += h->nTiles * h->chunks;
    tileBase += h->nTiles;
  }
  // the records of every frame, grouped by global tile (submission order kept)
  std::vector<FragRec> recs((size_t)nRec);
  std::vector<int> off((size_t)tileBase + 1), cursor((size_t)tileBase);
  {
    int acc = 0;
    for (int t = 0; t < tileBase; ++t) {
      off[t] = acc;
      cursor[t] = acc;
      acc += counts[t];
    }
    off[tileBase] = acc;
  }
  tileBase = 0;
  for (int i = 0; i < n; ++i) {
    for (const FragRec& fr : hs[i]->recs) {
      FragRec r = fr;
      r.tile += (uint32_t)tileBase;
      r.frame = (uint32_t)i;
      recs[cursor[r.tile]++] = r;
    }
    tileBase += hs[i]->nTiles;
  }
  g->nRec = nRec;
  g->nTiles = tileBase;
  cudaError_t e = cudaSuccess;
  const size_t rc = recs.empty() ? 1 : recs.size();
  e = dalloc(&g->dRecs, rc);
  if (e == cudaSuccess) e = dalloc(&g->dOff, (size_t)tileBase + 1);
  if (e == cudaSuccess) e = dalloc(&g->srecs, rc);
  if (e == cudaSuccess) e = dalloc(&g->blocks, (size_t)tileBase);
  if (e == cudaSuccess) e = dalloc(&g->redo, (size_t)items * (dfb::kItemPixels / 32) + 1);
  if (e == cudaSuccess) e = dalloc(&g->dFrames, (size_t)n);
  if (e == cudaSuccess) e = dalloc(&g->dItemBase, (size_t)n + 1);
  if (e == cudaSuccess) e = dalloc(&g->err, 1);
  if (e == cudaSuccess) e = cudaMemset(g->err, 0, sizeof(unsigned));
  if (e != cudaSuccess) {
    graph_free(g);
    return cuda_status(e);
  }
  tileBase = 0;
  items = 0;
  for (int i = 0; i < n; ++i) {
    fill_frame_args(hs[i], fa[i], tileBase, g->srecs, g->blocks);
    itemBase[i] = items;
    items += hs[i]->nTiles * fa[i].chunks;
    tileBase += hs[i]->nTiles;
  }
  itemBase[n] = items;
  g->items = items;
  if (!recs.empty())
    e = cudaMemcpy(g->dRecs, recs.data(), sizeof(FragRec) * recs.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(g->dOff, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice);
  g->hostFrames = fa;
  g->hostItemBase = itemBase;
  if (e == cudaSuccess)
    e = cudaMemcpy(g->dFrames, fa.data(), sizeof(FrameArgs) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(g->dItemBase, itemBase.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g->capStream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->done, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    graph_free(g);
    return cuda_status(e);
  }
  g->tune = hs[0]->tune;
  const int st = graph_capture(g);
  if (st != DFB_OK) {
    graph_free(g);
    return st;
  }
  for (int i = 0; i < n; ++i) {
    dfb_ctx* h = hs[i];
    finish_stats(h);
    h->stats = h->pendingStats;
    h->accumN = h->pendingN;
    h->inFrame = false;
  }
  *out = g;
  return DFB_OK;
}


}  // namespace

extern "C" {

int dfb_graph_create(const dfb_handle* hs, int n, dfb_graph* out) {
  return guarded([&]() -> int {
    if (!hs || n < 1 || !out) return DFB_ERR_INVALID_ARG;
    *out = nullptr;
    for (int i = 0; i < n; ++i) {
      if (!hs[i]) return DFB_ERR_INVALID_ARG;
      for (int j = 0; j < i; ++j)
        if (hs[j] == hs[i]) return DFB_ERR_INVALID_ARG;
      if (!hs[i]->inFrame) return DFB_ERR_STATE;
      if (hs[i]->cfg.dtype != hs[0]->cfg.dtype) return DFB_ERR_INVALID_ARG;
    }
    for (int i = 0; i < n; ++i) {
      const int st = check_trees(hs[i]);
      if (st != DFB_OK) return st;
    }
    for (int i = 0; i < n; ++i) {
      const int st = allocate(hs[i]);
      if (st != DFB_OK) return st;
      if (hs[i]->lastStreamSet) cudaEventSynchronize(hs[i]->frameDone);
      if (hs[i]->hostCopies) cudaEventSynchronize(hs[i]->copyDone);
    }
    dfb_graph_t* g = new (std::nothrow) dfb_graph_t();
    if (!g) return DFB_ERR_OOM;
    try {
      return graph_build(g, hs, n, out);
    } catch (...) {
      graph_free(g);
      throw;
    }
  });
}

int dfb_graph_launch(dfb_graph g, void* stream) {
  return guarded([&]() -> int {
    if (!g || !g->exec) return DFB_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaGraphLaunch(g->exec, s);
    if (e == cudaSuccess) e = cudaEventRecord(g->done, s);
    for (size_t i = 0; i < g->hs.size() && e == cudaSuccess; ++i) {
      dfb_ctx* h = g->hs[i];
      e = cudaEventRecord(h->frameDone, s);
      h->lastStream = s;
      h->lastStreamSet = true;
      h->haveFrame = true;
      h->lastErr = g->err;
      h->launches += 1 + (g->anyAcc ? 2 : 1) + (g->lng.items ? 1 : 0);
    }
    g->launched = true;
    return cuda_status(e);
  });
}

int dfb_graph_set_tuning(dfb_graph g, int ring_kb, int ctas_per_sm, int groups) {
  return guarded([&]() -> int {
    if (!g || !valid_tuning(ring_kb, ctas_per_sm, groups)) return DFB_ERR_INVALID_ARG;
    if (g->launched) cudaEventSynchronize(g->done);
    g->tune = dfb::TuneParams{ring_kb, ctas_per_sm, groups};
    return graph_capture(g);
  });
}

int dfb_graph_autotune(dfb_graph g, void* stream, int reps, int* ring_kb, int* ctas_per_sm,
                       int* groups, float* best_ms) {
  return guarded([&]() -> int {
    if (!g || reps < 1) return DFB_ERR_INVALID_ARG;
    // {ring KB, CTAs per SM, groups}; shapes whose ring is too small for the
    // dtype's largest item fail to launch and are skipped
    static const int cand[][3] = {{110, 2, 2}, {100, 2, 2}, {110, 2, 1}, {72, 3, 1},
                                  {64, 3, 1}, {220, 1, 2}};
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    float best = 1e30f;
    dfb::TuneParams bestT =
        dfb::default_tune(g->dtype, (double)g->nRec / (double)(g->nTiles ? g->nTiles : 1));
    for (const auto& c : cand) {
      if (e != cudaSuccess) break;
      if (dfb_graph_set_tuning(g, c[0], c[1], c[2]) != DFB_OK) continue;  // does not fit
      cudaError_t le = cudaGraphLaunch(g->exec, s);  // warm-up
      if (le == cudaSuccess) le = cudaEventRecord(a, s);
      for (int r = 0; r < reps && le == cudaSuccess; ++r) le = cudaGraphLaunch(g->exec, s);
      if (le == cudaSuccess) le = cudaEventRecord(b, s);
      if (le == cudaSuccess) le = cudaEventSynchronize(b);
      float ms = 0.f;
      if (le == cudaSuccess) le = cudaEventElapsedTime(&ms, a, b);
      if (le != cudaSuccess) {
        // a shape the device rejects is skipped; an error that persists is not
        cudaGetLastError();
        e = cudaDeviceSynchronize();
        continue;
      }
      if (ms / reps < best) {
        best = ms / reps;
        bestT = dfb::TuneParams{c[0], c[1], c[2]};
      }
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (e != cudaSuccess) return cuda_status(e);
    const int st = dfb_graph_set_tuning(g, bestT.ringKB, bestT.ctasPerSm, bestT.groups);
    if (st != DFB_OK) return st;
    for (dfb_ctx* h : g->hs) h->tune = bestT;
    if (ring_kb) *ring_kb = bestT.ringKB;
    if (ctas_per_sm) *ctas_per_sm = bestT.ctasPerSm;
    if (groups) *groups = bestT.groups;
    if (best_ms) *best_ms = best;
    return DFB_OK;
  });
}

int dfb_graph_destroy(dfb_graph g) {
  return guarded([&]() -> int {
    if (!g) return DFB_OK;
    graph_free(g);
    return DFB_OK;
  });
}

}  // extern "C"

// ============================================================================
// prepared submissions and the one-call server step
// ============================================================================
struct dfb_tileset_t {
  int width = 0, height = 0, tileSize = 0, dtype = 0;
  std::vector<FragRec> recs;
  std::vector<int> tiles, counts;  // generation-1 arrivals per touched tile
  int64_t fragmentPixels = 0;
};

namespace {

bool same_geometry(const dfb_ctx* h, const dfb_tileset_t* s) {
  return s->width == h->cfg.width && s->height == h->cfg.height &&
         s->tileSize == h->cfg.tile_size && s->dtype == h->cfg.dtype;
}

void submit_set(dfb_ctx* h, const dfb_tileset_t* s) {
  h->recs.insert(h->recs.end(), s->recs.begin(), s->recs.end());
  for (size_t i = 0; i < s->tiles.size(); ++i) {
    h->recvGen1[s->tiles[i]] += s->counts[i];
    count_frags(h, s->tiles[i], s->counts[i]);
  }
  h->pendingStats.fragments += (int64_t)s->recs.size();
  h->pendingStats.fragment_pixels += s->fragmentPixels;
}

}  // namespace

extern "C" {

int dfb_tileset_create(dfb_handle h, int n, const int* tile_ids, const float* order_keys,
                       const void* const* rgba, const float* const* depth, const float* scales,
                       dfb_tileset* out) {
  return guarded([&]() -> int {
    if (!h || n < 0 || !out) return DFB_ERR_INVALID_ARG;
    *out = nullptr;
    const int st = validate_arrays(h, n, tile_ids, order_keys, rgba, depth, scales);
    if (st != DFB_OK) return st;
    dfb_tileset_t* s = new (std::nothrow) dfb_tileset_t();
    if (!s) return DFB_ERR_OOM;
    try {
      s->width = h->cfg.width;
      s->height = h->cfg.height;
      s->tileSize = h->cfg.tile_size;
      s->dtype = h->cfg.dtype;
      s->recs.resize((size_t)n);
      std::vector<int> perTile((size_t)h->nTiles, 0);
      s->fragmentPixels = build_records(h, n, tile_ids, order_keys, rgba, depth, scales,
                                        s->recs.data(), perTile.data());
      for (int t = 0; t < h->nTiles; ++t)
        if (perTile[t]) {
          s->tiles.push_back(t);
          s->counts.push_back(perTile[t]);
        }
    } catch (const std::bad_alloc&) {
      delete s;
      return DFB_ERR_OOM;
    }
    *out = s;
    return DFB_OK;
  });
}

int dfb_tileset_destroy(dfb_tileset s) {
  return guarded([&]() -> int {
    delete s;
    return DFB_OK;
  });
}

int dfb_submit_tileset(dfb_handle h, dfb_tileset s) {
  return guarded([&]() -> int {
    if (!h || !s) return DFB_ERR_INVALID_ARG;
    if (!h->inFrame) return DFB_ERR_STATE;
    if (!same_geometry(h, s)) return DFB_ERR_INVALID_ARG;
    submit_set(h, s);
    return DFB_OK;
  });
}

int dfb_run_frames(const dfb_handle* hs, const dfb_tileset* sets, const int* accumulate, int n,
                   void* stream) {
  return guarded([&]() -> int {
    if (!hs || !sets || n < 1) return DFB_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i) {
      if (!hs[i] || !sets[i]) return DFB_ERR_INVALID_ARG;
      if (hs[i]->inFrame) return DFB_ERR_STATE;
      if (!same_geometry(hs[i], sets[i])) return DFB_ERR_INVALID_ARG;
      if (hs[i]->cfg.dtype != hs[0]->cfg.dtype) return DFB_ERR_INVALID_ARG;
    }
    {
      std::vector<const dfb_ctx*> sorted(hs, hs + n);
      std::sort(sorted.begin(), sorted.end());
      if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end())
        return DFB_ERR_INVALID_ARG;
    }
    {
      cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;  // as in dfb_end_frames
      if (cudaStreamIsCapturing((cudaStream_t)stream, &cap) != cudaSuccess) cudaGetLastError();
      else if (cap != cudaStreamCaptureStatusNone) return DFB_ERR_STATE;
    }
    for (int i = 0; i < n; ++i) {
      const int st = dfb_begin_frame(hs[i], accumulate ? accumulate[i] : 0);
      if (st != DFB_OK) return st;
      submit_set(hs[i], sets[i]);
    }
    return dfb_end_frames(hs, n, stream);
  });
}

}  // extern "C"
