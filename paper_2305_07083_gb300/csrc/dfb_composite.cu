// Composite kernel of the DFB path (K2/K3 with the fused K4 epilogue) for
// sm_103a: a persistent, warp-specialised, bulk-copy pipeline.
//
// Per pixel it computes the AlphaBlend tile operation of Sec. 4.2 /
// Listing 4 (sort the pixel's fragments by depth -- ties by order key, then
// submit index -- and blend them front to back with the premultiplied "over"
// operator, then the generation-0 background of Listing 3), the ordered
// "list" form of Sec. 4.2 (blend in key order), depth compositing (Sec. 2.1:
// the nearest fragment's RGBA), or the mean of redundantly rendered tiles
// (Sec. 4.1.1), and an optional pixel operation before the display
// conversion (Sec. 3.1.2).  The epilogue updates the
// progressive accumulation and variance tiles of Listing 1 (running sum,
// Kahan-compensated past a threshold; Welford M2; per-tile variance for
// Sec. 4.1.1) and writes the RGBA8 display format of Sec. 3.1.
//
// The work is bound by HBM bandwidth (~0.4 flop per byte), so the design goal
// is to keep enough bytes in flight:
//   * CTA = G consumer groups of 8 warps (one pixel per thread, 256 pixels =
//     one work item; the groups take alternate items) + 1 producer warp, PER
//     CTAs per SM (by default G = 1, PER = 2).  CTAs are persistent and walk
//     the work items of all frames of the launch with a static stride, which
//     keeps the chunks of a tile on neighbouring CTAs that run in step.
//   * The producer warp fetches each item's tile block (fragment count,
//     list offset and sorted records, written by the bucketing) with one bulk
//     copy kMetaQ items ahead, so locating an item's fragments needs no
//     dependent global loads.  It then issues one-dimensional bulk copies
//     (cp.async.bulk, the TMA engine) of each fragment's depth slab and RGBA
//     slab straight into a shared-memory ring, completing on the fill's
//     mbarrier.  Fills take only the ring bytes they need (n fragments x slab
//     size), so the ring holds as many fills in flight as their sizes allow,
//     up to kSlots (each consumer group owns kSlots / G of them).
//   * An item of at most kStageFragments fragments is one fill.  A longer
//     one streams through the ring in fills of kFill fragments; its
//     consumers carry the per-pixel blend across the fills (BLEND_DEPTH
//     speculatively in list order), so a long list costs the same bytes per
//     fragment as a short one.  The rare 32-pixel units whose depths turn
//     out to be out of list order are redone exactly by k_composite_redo.
//   * The accumulation state (sum, M2, Kahan compensation) is stored
//     tile-major, so an item's state is one contiguous run per buffer.  In
//     frames with few fragments per tile the producer streams it into the
//     item's last fill; in the others the consumers load it into registers
//     before they wait for the fragments, so that the ring holds fragments
//     only (the state's bytes would occupy it for the item's whole stay and
//     leave room for fewer items in flight).  Consumers read the fragments
//     from shared memory, sort and blend, and release the ring space before
//     the epilogue.
//   * The epilogue writes one variance partial per warp with plain stores;
//     a small second kernel sums each tile's partials in a fixed order.
// Every wait is bounded in time; on expiry the kernel sets an error bit,
// drains its own bulk copies and returns.
#include <string.h>

#include <utility>

#include "dfb_device.cuh"
#include "dfb_internal.h"

namespace dfb {

// sRGB encode tables (SrgbTables), uploaded by the host.
__device__ SrgbTables g_srgb;

cudaError_t upload_srgb_tables(const SrgbTables& host) {
  return cudaMemcpyToSymbol(g_srgb, &host, sizeof(SrgbTables));
}

// Copy the sRGB tables into shared memory (every thread of the CTA calls it).
__device__ __forceinline__ void load_srgb(SrgbTables* dst, int nThreads) {
  const uint32_t* src = reinterpret_cast<const uint32_t*>(&g_srgb);
  uint32_t* d = reinterpret_cast<uint32_t*>(dst);
  for (int i = threadIdx.x; i < (int)(sizeof(SrgbTables) / 4); i += nThreads) d[i] = src[i];
}

namespace {

constexpr int kP = kItemPixels;          // pixels per item = threads of a consumer group
constexpr int kCW = kP / 32;             // warps of a consumer group
// Threads of a CTA with G consumer groups (items k, k+1, ... composited in
// parallel) and one producer warp.
template <int G>
struct Shape {
  static constexpr int threads = G * kP + 32;
  static_assert(threads <= 1024, "threads per CTA");
};
// Launch shapes: G consumer groups per CTA, PER resident CTAs per SM.
//   (G, PER) = (1, 2), (2, 2), (1, 3), (2, 1), (3, 1)
constexpr int kN = kStageFragments;
constexpr int kSlots = 16;               // items in flight at most
constexpr int kMetaQ = 8;                // tile blocks fetched ahead
constexpr uint32_t kWindowBytes = kSortWindow * kP * 8;

// Descriptor of one fill of the ring: up to kN fragments of one work item
// (all of them for an item of at most kN fragments, else kFill), and the
// item's state rows in its last fill when the frame streams them.
struct ItemMeta {
  int n;               // fragments in this fill
  int total;           // fragments of the item
  int first;           // list index of the fill's first fragment
  int pad;
  uint32_t start;      // byte offset of the fill's data in the ring
  uint32_t bytes;      // bytes of the fill's fragments from `start` (state rows follow)
  unsigned long long end;  // producer's head position after this fill
  const void* rgba[kN];
  float scale[kN];
};
static_assert(sizeof(ItemMeta) <= 256, "item meta");

// Shared memory: [sRGB tables 2.75 KB][barriers 512 B][flags 128 B][metas 4 KB]
//                [tile-block queue][ring]
constexpr int kOffBars = (int)sizeof(SrgbTables);
constexpr int kOffFlags = kOffBars + 512;
constexpr int kOffMetas = kOffFlags + 128;
constexpr int kOffQueue = kOffMetas + kSlots * 256;
constexpr int kOffQLoc = kOffQueue + kMetaQ * (int)sizeof(TileBlock);
constexpr int kHeader = kOffQLoc + 128;
static_assert((2 * kSlots + kMetaQ) * 8 <= 512, "barrier space");
static_assert(kOffQueue % 128 == 0 && kHeader % 128 == 0, "alignment");
static_assert(kMetaQ * 16 <= 128, "queue locations");
static_assert(32 % kFill == 0 && kFill <= kN, "fills never straddle a window of 32 records");

template <int DT>
struct Bytes {
  static constexpr int px = PxBytes<DT>::value;
  // largest fill the ring must hold: kN fragments plus three rows of
  // framebuffer state (sum, M2, Kahan compensation)
  static constexpr uint32_t maxItem = (uint32_t)kN * kP * (4 + px) + 3u * kP * 16u;
};

// Where a launch's frame arguments are read from.
constexpr int kGlobalTable = 0;  // the frame table and item prefix in global memory
constexpr int kOneFrame = 1;     // one frame, its arguments a kernel parameter
constexpr int kParamTable = 2;   // up to kParamFrames frames, the tables a kernel parameter
constexpr int kParamFrames = 48;
struct FrameTable {
  int itemBase[kParamFrames + 1];
  FrameArgs f[kParamFrames];
};
static_assert(sizeof(FrameTable) <= 16384, "kernel parameter size");
template <int FR>
struct FrameParams {
  using type = int;  // unused
};
template <>
struct FrameParams<kOneFrame> {
  using type = FrameArgs;
};
template <>
struct FrameParams<kParamTable> {
  using type = FrameTable;
};

__device__ __forceinline__ int find_frame(const int* itemBase, int nFrames, int item) {
  int lo = 0, hi = nFrames - 1;  // last frame whose first item <= item
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (itemBase[mid] <= item) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Bounded wait on an mbarrier phase.  Returns false when the wait expired or
// another role of the CTA has given up.
__device__ __forceinline__ bool wait_phase(uint64_t* bar, uint32_t parity, const LaunchCtl& ctl,
                                           volatile int* abort) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t spin = 1;; ++spin) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((spin & 63) == 0) {
      if (*abort) return false;
      if (global_ns() - t0 > ctl.waitNs) return false;
    }
  }
}

__device__ __forceinline__ void give_up(const LaunchCtl& ctl, volatile int* abort) {
  *abort = 1;
  atomicOr(ctl.err, kErrTimeout);
}

// Insert k into the sorted per-thread window kb[0..m-1] (stride kP),
// shifting larger keys up one slot; slot m must be free.
__device__ __forceinline__ void window_insert(uint64_t* kb, int m, uint64_t k) {
  int j = m - 1;
  while (j >= 0) {
    const uint64_t v = kb[j * kP];
    if (v < k) break;
    kb[(j + 1) * kP] = v;
    --j;
  }
  kb[(j + 1) * kP] = k;
}

// Where a work item lies: frame, frame-local tile, chunk, global tile.
struct ItemLoc {
  int f, tile, chunk, gt;
};

// FR: where the launch's frame arguments are (FrameSource); with kOneFrame
// `frames` points to a single frame's arguments in the kernel's parameter
// space (read through the constant cache, no loads).
template <int FR>
__device__ __forceinline__ ItemLoc locate(const FrameArgs* frames, const int* itemBase,
                                          int nFrames, int item) {
  ItemLoc L;
  L.f = FR == kOneFrame ? 0 : find_frame(itemBase, nFrames, item);
  const FrameArgs* A = frames + L.f;
  const int local = FR == kOneFrame ? item : item - itemBase[L.f];
  L.tile = local >> A->logChunks;
  L.chunk = local & (A->chunks - 1);
  L.gt = A->tileBase + L.tile;
  return L;
}

// ---------------------------------------------------------------------------
// producer warp
// ---------------------------------------------------------------------------
// Fills of the ring.  Consumer group g owns the slots g*S .. g*S+S-1 (S =
// kSlots / G) and takes its items' fills from them in order.  Ring bytes are
// reclaimed in the global order of the fills; a fill may reuse a slot once
// the slot's previous fill has been released.
template <int DT, int G, int FR>
__device__ void producer(const FrameArgs* __restrict__ frames, const int* __restrict__ itemBase,
                         int nFrames, int totalItems, const LaunchCtl& ctl, unsigned char* ring,
                         uint32_t ringBytes, ItemMeta* metas, TileBlock* queue, int4* qLoc,
                         uint64_t* fullB, uint64_t* emptyB, uint64_t* queueB,
                         volatile int* abort) {
  constexpr int px = Bytes<DT>::px;
  constexpr int S = kSlots / G;
  const int lane = threadIdx.x & 31;
  unsigned long long head = 0, tail = 0;  // monotonic ring positions
  int curFill = 0, tailFill = 0;          // fills issued / reclaimed (global order)
  int gf0 = 0, gf1 = 0, gf2 = 0;          // fills issued per consumer group
  // lane-distributed tables: lane e < kSlots holds the slot and the parity
  // of outstanding fill e (mod kSlots); lane s < kSlots holds the global
  // index of the last fill of slot s
  int fifoSlot = 0, fifoPar = 0, slotFill = -1;
  uint32_t armed = 0, armedPar = 0;       // per ring slot: armed / parity of last arm
  uint32_t qArmed = 0, qPar = 0;          // per queue slot
  // tile block of local item kk -> queue slot kk % kMetaQ (lane 0)
  auto fetch = [&](int kk) {
    const int it = blockIdx.x + kk * (int)gridDim.x;
    if (it >= totalItems || lane != 0) return;
    const ItemLoc L = locate<FR>(frames, itemBase, nFrames, it);
    if (!DFB_CHECK(L.f >= 0 && L.f < nFrames && L.tile >= 0 && L.tile < frames[L.f].nTiles,
                   ctl.err))
      return;
    const int q = kk % kMetaQ;
    qLoc[q] = make_int4(L.f, L.tile, L.chunk, L.gt);
    fence_proxy_async();  // the slot's previous block was read through the generic proxy
    mbar_arrive_expect_tx(&queueB[q], (uint32_t)sizeof(TileBlock));
    bulk_g2s(queue + q, frames[L.f].blocks + L.gt, (uint32_t)sizeof(TileBlock), &queueB[q]);
    qArmed |= 1u << q;
    qPar = (qPar & ~(1u << q)) | ((uint32_t)((kk / kMetaQ) & 1) << q);
  };
  for (int kk = 0; kk < kMetaQ; ++kk) fetch(kk);
  bool ok = true;
  int k = 0;
  for (int item = blockIdx.x; item < totalItems && ok; item += gridDim.x, ++k) {
    const int q = k % kMetaQ;
    if (!wait_phase(&queueB[q], (uint32_t)(k / kMetaQ) & 1u, ctl, abort)) {
      ok = false;
      break;
    }
    // The item's tile block stays in queue slot q until its fills are
    // issued; the next fetch into the slot follows them.
    const TileBlock* blk = queue + q;
    const int n = blk->n;
    const int4 loc = qLoc[q];
    const FrameArgs* A = frames + loc.x;
    const int P = A->P, mode = A->mode;
    const size_t p0 = (size_t)loc.z * P;  // the item's first pixel in its tile
    // An item of more than kN fragments is streamed in fills of kFill; its
    // records past the tile block come from the sorted list.
    const int per = n > kN ? kFill : kN;
    const int fills = n > kN ? (n + kFill - 1) / kFill : 1;
    const uint32_t dBytes = mode == DFB_BLEND_DEPTH || mode == DFB_ZCOMPOSITE ? (uint32_t)P * 4u : 0u;
    const uint32_t cBytes = mode != DFB_ZCOMPOSITE ? (uint32_t)P * px : 0u;
    // accumulation state of the item's pixels, one contiguous run per
    // buffer, when the frame streams it with the fragments
    const bool loadState = (A->flags & DFB_FLAG_ACCUMULATE) && A->frameN != 1 && A->stateInRing;
    const int nState = loadState ? (A->kahan && !A->kahanFirst ? 3 : 2) : 0;
    const int g = G == 1 ? 0 : k % G;
    for (int f = 0; f < fills; ++f) {
      const int i0 = f * per;
      const int nf = min(per, n - i0);
      const bool lastFill = f == fills - 1;
      const uint32_t fragBytes = (uint32_t)nf * (dBytes + cBytes);
      const uint32_t need = fragBytes + (lastFill ? nState * (uint32_t)P * 16u : 0u);  // multiple of 16
      // ring space: no fill straddles the end of the ring
      if ((uint32_t)(head % ringBytes) + need > ringBytes) head += ringBytes - head % ringBytes;
      const int jg = g == 0 ? gf0 : (g == 1 ? gf1 : gf2);
      const int s = g * S + jg % S;
      const uint32_t par = (uint32_t)(jg / S) & 1u;
      const int prev = __shfl_sync(0xffffffffu, slotFill, s);
      while (tailFill < curFill && (tailFill <= prev || head + need - tail > ringBytes)) {
        const int e = tailFill % kSlots;
        const int es = __shfl_sync(0xffffffffu, fifoSlot, e);
        const int ep = __shfl_sync(0xffffffffu, fifoPar, e);
        if (!wait_phase(&emptyB[es], (uint32_t)ep, ctl, abort)) {
          ok = false;
          break;
        }
        tail = metas[es].end;
        ++tailFill;
      }
      if (!ok) break;
      if (tailFill == curFill) tail = head;  // nothing outstanding: the padding is free too
      if (!DFB_CHECK((uint64_t)(head % ringBytes) + need <= ringBytes &&
                         head + need - tail <= ringBytes && nf <= kN &&
                         (loc.z + 1) * P <= A->T * A->T,
                     ctl.err)) {
        ok = false;
        break;
      }
      const uint32_t start = (uint32_t)(head % ringBytes);
      head += need;
      ItemMeta* meta = metas + s;
      // lane li < nf takes fragment i0 + li: from the tile block for the
      // first kN, else from the sorted list in global memory
      const void* rRgba = nullptr;
      const float* rDepth = nullptr;
      if (lane < nf) {
        const int i = i0 + lane;
        const FragRec* rec = i < kN ? blk->recs + i : A->srecs + blk->off + i;
        rRgba = rec->rgba;
        rDepth = rec->depth;
        meta->rgba[lane] = rRgba;
        meta->scale[lane] = rec->scale;
      }
      if (lane == 0) {
        meta->n = nf;
        meta->total = n;
        meta->first = i0;
        meta->start = start;
        meta->bytes = fragBytes;
        meta->end = head;
      }
      if (lane == curFill % kSlots) {
        fifoSlot = s;
        fifoPar = (int)par;
      }
      if (lane == s) slotFill = curFill;
      ++curFill;
      if (g == 0) ++gf0; else if (g == 1) ++gf1; else ++gf2;
      __syncwarp();
      if (f != 0 || item != ctl.stallItem) {  // test fault injection: never signal this item
        if (lane == 0) mbar_arrive_expect_tx(&fullB[s], need);
        armed |= 1u << s;
        armedPar = (armedPar & ~(1u << s)) | (par << s);
        __syncwarp();
        unsigned char* base = ring + start;
        if (lane < nf) {
          if (dBytes) bulk_g2s(base + lane * dBytes, rDepth + p0, dBytes, &fullB[s]);
          if (cBytes)
            bulk_g2s(base + nf * dBytes + lane * cBytes,
                     static_cast<const unsigned char*>(rRgba) + p0 * px, cBytes, &fullB[s]);
        }
        if (lastFill && lane < nState) {
          // state runs: [sum | M2 | comp], P pixels of 16 bytes each
          const float4* src = lane == 0 ? A->accum : (lane == 1 ? A->m2 : A->comp);
          bulk_g2s(base + fragBytes + lane * (uint32_t)P * 16u,
                   src + (size_t)loc.y * A->T * A->T + p0, (uint32_t)P * 16u, &fullB[s]);
        }
      }
    }
    __syncwarp();
    fetch(k + kMetaQ);  // every lane is done with the slot's block
  }
  if (!ok && lane == 0) give_up(ctl, abort);
  // Leave no bulk copy in flight into this CTA's shared memory.
  auto drain = [&](uint64_t* bars, uint32_t mask, uint32_t parv, int count) {
    for (int qq = 0; qq < count; ++qq)
      if (mask & (1u << qq)) {
        const uint64_t t0 = global_ns();
        while (!mbar_try_wait(&bars[qq], (parv >> qq) & 1u)) {
          if (global_ns() - t0 > ctl.waitNs) {
            if (lane == 0) atomicOr(ctl.err, kErrDrain);
            break;
          }
        }
      }
  };
  drain(fullB, armed, armedPar, kSlots);
  qArmed = __shfl_sync(0xffffffffu, qArmed, 0);
  qPar = __shfl_sync(0xffffffffu, qPar, 0);
  drain(queueB, qArmed, qPar, kMetaQ);
}

// ---------------------------------------------------------------------------
// consumer warps: one pixel per thread
// ---------------------------------------------------------------------------
// A depth that takes part in the blend: not +inf and not NaN (both read as an
// empty fragment; NaN maps to +inf).  The speculative in-order passes compare
// such depths as floats, which orders them exactly as their canonical keys
// (depth_bits) do: -0 equals +0 and -inf comes first.
__device__ __forceinline__ bool covers(float z) { return z <= 3.402823466e38f; }

// Returns false only in DFB_ZCOMPOSITE for a pixel no fragment covers.
template <int DT>
__device__ __forceinline__ bool composite_staged(int mode, int n, int P, const unsigned char* base,
                                                 const ItemMeta* meta, int t, int p,
                                                 float& c0, float& c1, float& c2, float& al) {
  constexpr int px = Bytes<DT>::px;
  const float* sD = reinterpret_cast<const float*>(base);
  // floats per depth slab (no depth is staged in the modes that ignore it)
  const int dStride = mode == DFB_BLEND_DEPTH || mode == DFB_ZCOMPOSITE ? P : 0;
  const unsigned char* sC = base + (size_t)n * dStride * 4;
  if (mode == DFB_BLEND_ORDERED) {
    for (int i = 0; i < n; ++i) over(Px<DT>::shared(sC + (size_t)i * P * px, t, meta->scale[i]), c0, c1, c2, al);
  } else if (mode == DFB_AVERAGE) {
    // equal-weight mean of the redundant tiles, summed in list order
    for (int i = 0; i < n; ++i) {
      const float4 f = Px<DT>::shared(sC + (size_t)i * P * px, t, meta->scale[i]);
      c0 += f.x; c1 += f.y; c2 += f.z; al += f.w;
    }
    if (n > 0) {
      const float k = (float)n;
      c0 = __fdiv_rn(c0, k); c1 = __fdiv_rn(c1, k); c2 = __fdiv_rn(c2, k); al = __fdiv_rn(al, k);
    }
  } else if (mode == DFB_ZCOMPOSITE) {
    uint64_t best = ~0ull;
    for (int i = 0; i < n; ++i) {
      const uint64_t k = ((uint64_t)depth_bits(sD[i * P + t]) << 32) | (uint32_t)i;
      best = k < best ? k : best;
    }
    if (n == 0 || (uint32_t)(best >> 32) == kInfBits) return false;
    const int i = (int)(uint32_t)best;
    const float4 f = Px<DT>::global(meta->rgba[i], p, meta->scale[i]);
    c0 = f.x; c1 = f.y; c2 = f.z; al = f.w;
  } else {
    // Speculative pass in list order.  For bricks whose key order is their
    // depth order (the common case) the finite-depth fragments are already
    // in blend order, so they are blended as they are read while the order
    // is checked.  Fragments empty at this pixel (depth +inf, which sort
    // after every finite depth) are not blended here: blending an all-zero
    // RGBA is an exact no-op anywhere, so only non-zero empty fragments need
    // the second pass, in list order, after the finite ones.  If the check
    // fails the pixel starts over on the sorting path below.
    {
      float last = -INFINITY;
      uint32_t emptyBits = 0;
      bool inOrder = true;
      for (int i = 0; i < n; ++i) {
        const float z = sD[i * P + t];
        const float4 f = Px<DT>::shared(sC + (size_t)i * P * px, t, meta->scale[i]);
        if (covers(z)) {
          inOrder = inOrder && z >= last;
          last = z;
          over(f, c0, c1, c2, al);
        } else {
          emptyBits |= __float_as_uint(f.x) | __float_as_uint(f.y) | __float_as_uint(f.z) |
                       __float_as_uint(f.w);
        }
      }
      if (inOrder) {
        if (emptyBits) {
          for (int i = 0; i < n; ++i)
            if (!covers(sD[i * P + t]))
              over(Px<DT>::shared(sC + (size_t)i * P * px, t, meta->scale[i]), c0, c1, c2, al);
        }
        return true;
      }
      c0 = c1 = c2 = al = 0.0f;
    }
    // General case: insertion sort of fragment indices (4-bit slots of
    // `perm`) by depth key.  The list arrives in key order, so ties stay in
    // (key, submit index) order; empty fragments go to a second list kept in
    // list order and blended last.
    uint64_t perm = 0, infs = 0;
    int m = 0, mi = 0;
    uint32_t lastKey = 0;
    for (int i = 0; i < n; ++i) {
      const uint32_t key = depth_bits(sD[i * P + t]);
      const bool isInf = key == kInfBits;
      const bool app = !isInf && (m == 0 || key >= lastKey);
      if (!isInf && !app) {
        int j = m - 1;
        while (j > 0 && depth_bits(sD[(int)((perm >> (4 * (j - 1))) & 15u) * P + t]) > key) --j;
        const uint64_t lowMask = (j == 0) ? 0ull : ((1ull << (4 * j)) - 1ull);
        perm = (perm & lowMask) | ((uint64_t)i << (4 * j)) | ((perm & ~lowMask) << 4);
        ++m;
      }
      // appends to either list without a branch
      const uint64_t bit = (uint64_t)i << (4 * (isInf ? mi : m));
      infs |= isInf ? bit : 0ull;
      perm |= app ? bit : 0ull;
      lastKey = app ? key : lastKey;
      mi += isInf ? 1 : 0;
      m += app ? 1 : 0;
    }
    // one loop of exactly n steps: the finite list, then the empty ones
    for (int r = 0; r < n; ++r) {
      const bool fin = r < m;
      const uint64_t src = fin ? perm : infs;
      const int rr = fin ? r : r - m;
      const int i = (int)((src >> (4 * rr)) & 15u);
      over(Px<DT>::shared(sC + (size_t)i * P * px, t, meta->scale[i]), c0, c1, c2, al);
    }
  }
  return true;
}

// Exact BLEND_DEPTH order for one pixel of a long list, fragments read from
// HBM: rounds of a per-pixel window of the kSortWindow nearest (depth key,
// list index) keys above the last one blended, blended in that order.  The
// list arrives in (key, submit index) order, so ties on depth keep it.
template <int DT>
__device__ __forceinline__ void composite_exact(int n, const FragRec* list, uint64_t* kbAll,
                                                int t, int p, float& c0, float& c1, float& c2,
                                                float& al) {
  uint64_t* kb = kbAll + t;
  uint64_t lo = 0;
  int done = 0;
  while (done < n) {
    int m = 0;
    uint64_t last = 0;
    for (int ib = 0; ib < n; ib += 8) {
      float z[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) z[u] = (ib + u < n) ? __ldg(list[ib + u].depth + p) : 0.0f;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int i = ib + u;
        if (i < n) {
          const uint64_t k = ((uint64_t)depth_bits(z[u]) << 32) | (uint32_t)i;
          if (done == 0 || k > lo) {
            if (m < kSortWindow) {
              if (m == 0 || k > last) {
                kb[m * kP] = k;
                last = k;
              } else {
                window_insert(kb, m, k);
              }
              ++m;
            } else if (k < last) {
              window_insert(kb, kSortWindow - 1, k);  // drops the largest
              last = kb[(kSortWindow - 1) * kP];
            }
          }
        }
      }
    }
    for (int r = 0; r < m; r += 4) {
      float4 c[4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (r + u < m) {
          const int i = (int)(uint32_t)kb[(r + u) * kP];
          c[u] = Px<DT>::global(list[i].rgba, p, list[i].scale);
        }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (r + u < m) over(c[u], c0, c1, c2, al);
    }
    lo = last;
    done += m;
  }
}

// One pixel of one work item.
struct PixWork {
  const FrameArgs* A;
  int tile, chunk, p, P;
  bool active;
  uint32_t pix;   // row-major image index (frames hold at most 2^31 pixels)
  uint32_t sidx;  // tile-major state index (tile-major state of at most 2^32 pixels)
};

template <int FR>
__device__ __forceinline__ PixWork prepare(const FrameArgs* frames, const int* itemBase,
                                           int nFrames, int item, int t) {
  PixWork w;
  const int f = FR == kOneFrame ? 0 : find_frame(itemBase, nFrames, item);
  const FrameArgs* A = frames + f;
  w.A = A;
  const int local = FR == kOneFrame ? item : item - itemBase[f];
  const int T = A->T;
  w.P = A->P;
  w.tile = local >> A->logChunks;
  w.chunk = local & (A->chunks - 1);
  // tile / tilesX without a division: (tile + 0.5) / tilesX is never within
  // float rounding of an integer for tile counts below 2^20
  const int ty = __float2int_rz(((float)w.tile + 0.5f) * A->invTilesX);
  const int tx = w.tile - ty * A->tilesX;
  w.p = w.chunk * w.P + t;
  w.sidx = (uint32_t)w.tile * (uint32_t)(T * T) + (uint32_t)w.p;
  const int x = tx * T + (w.p & (T - 1));
  const int y = ty * T + (w.p >> A->logT);
  w.active = (t < w.P) && (x < A->W) && (y < A->H);
  w.pix = (uint32_t)y * (uint32_t)A->W + (uint32_t)x;
  return w;
}

// Background (generation 0), then the K4 epilogue of one pixel: colour,
// running sum (Kahan-compensated past the threshold), Welford M2, mean, RGBA8,
// and one variance partial per warp of 32 pixels.  S, M, CP are the pixel's
// previous sum, M2 and compensation.  Every lane of the warp calls it (the
// partial is a warp reduction); inactive lanes contribute zero.
__device__ __forceinline__ void finish_pixel(const FrameArgs* A, const PixWork& w, int lane,
                                             int warp, float c0, float c1, float c2, float al,
                                             bool covered, float4 S, float4 M, float4 CP,
                                             const SrgbTables* tb, unsigned* err) {
  const unsigned flags = A->flags;
  const bool acc = (flags & DFB_FLAG_ACCUMULATE) != 0;
  float vsum = 0.0f;
  if (w.active) {
    if (A->mode != DFB_ZCOMPOSITE) {
      over(make_float4(A->bgR, A->bgG, A->bgB, A->bgA), c0, c1, c2, al);  // generation 0
    } else if (!covered) {
      c0 = A->bgR; c1 = A->bgG; c2 = A->bgB; al = A->bgA;
    }
    const float4 col = make_float4(c0, c1, c2, al);
    const bool pixOk = DFB_CHECK(w.pix < (size_t)A->W * A->H, err);
    const bool stateOk = DFB_CHECK(w.sidx < (size_t)A->nTiles * A->T * A->T, err);
    if ((flags & DFB_FLAG_WRITE_COLOR) && pixOk) A->color[w.pix] = col;
    float4 out = col;
    if (acc) {
      float4 Sn, tot;
      if (A->kahan) {
        float4 cn;
#define DFB_KAHAN(ch)                 \
  {                                   \
    const float yk = col.ch - CP.ch;  \
    const float tk = S.ch + yk;       \
    cn.ch = (tk - S.ch) - yk;         \
    Sn.ch = tk;                       \
    tot.ch = tk - cn.ch;              \
  }
        DFB_KAHAN(x) DFB_KAHAN(y) DFB_KAHAN(z) DFB_KAHAN(w)
#undef DFB_KAHAN
        if (stateOk) A->comp[w.sidx] = cn;
      } else {
        Sn = make_float4(S.x + col.x, S.y + col.y, S.z + col.z, S.w + col.w);
        tot = Sn;
      }
      const float iN = A->invN, iN1 = A->invNm1;
      const float4 mean = make_float4(tot.x * iN, tot.y * iN, tot.z * iN, tot.w * iN);
      if (A->frameN != 1) {
        // Welford: M2 += (x - mean_{n-1}) (x - mean_n), mean_{n-1} = S_{n-1}/(n-1)
        M.x = fmaf(col.x - S.x * iN1, col.x - mean.x, M.x);
        M.y = fmaf(col.y - S.y * iN1, col.y - mean.y, M.y);
        M.z = fmaf(col.z - S.z * iN1, col.z - mean.z, M.z);
        M.w = fmaf(col.w - S.w * iN1, col.w - mean.w, M.w);
      }
      if (stateOk) {
        A->accum[w.sidx] = Sn;
        A->m2[w.sidx] = M;
      }
      vsum = (M.x + M.y + M.z) * iN1;
      out = mean;
    }
    if ((flags & DFB_FLAG_PACK_RGBA8) && pixOk)
      A->rgba8[w.pix] = pack_rgba8(pixel_op(out, A), tb);
  }
  if (acc && warp * 32 < w.P) {
    // one partial per warp of 32 pixels, summed per tile by k_tile_variance
    float v = vsum;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const size_t slot = (size_t)w.tile * A->slots + ((w.chunk * w.P + warp * 32) >> 5);
    if (lane == 0 && DFB_CHECK(slot < (size_t)A->nTiles * A->slots, err)) A->varPartial[slot] = v;
  }
}

// A multi-fill item's fills, for one blend mode: the consumer group takes
// them from its slots in order (jg counts its fills) and carries the
// per-pixel blend across them; streamed state rows come with the last fill.
// BLEND_DEPTH blends speculatively in list order; `exact` turns false for a
// pixel whose finite depths are out of list order or that has a non-zero
// empty fragment.  Returns false when a wait ran out.
template <int DT, int MODE, int G>
__device__ __forceinline__ bool multi_fill(int total, const PixWork& w, int t, int lane,
                                           const LaunchCtl& ctl, unsigned char* ring,
                                           ItemMeta* metas, uint64_t* fullB, uint64_t* emptyB,
                                           volatile int* abort, uint32_t ringBytes, int group,
                                           int& jg, uint32_t stateRows, float& c0, float& c1,
                                           float& c2, float& al, bool& covered, bool& exact,
                                           float4& S0, float4& M, float4& CP) {
  constexpr int S = kSlots / G;
  constexpr int px = Bytes<DT>::px;
  const int fills = (total + kFill - 1) / kFill;
  const int P = w.P;
  float last = -INFINITY;
  uint32_t emptyBits = 0u;
  bool inOrder = true;
  uint64_t best = ~0ull;
  const void* bestRgba = nullptr;
  float bestScale = 1.0f;
  for (int f = 0; f < fills; ++f) {
    const int s = group * S + jg % S;
    if (f > 0 && !wait_phase(&fullB[s], (uint32_t)(jg / S) & 1u, ctl, abort)) {
      if (lane == 0) give_up(ctl, abort);
      return false;
    }
    const ItemMeta* meta = metas + s;
    const unsigned char* base = ring + meta->start;
    const int nf = meta->n;
    const bool lastFill = f == fills - 1;
    const bool inRing = DFB_CHECK(
        nf <= kN && (uint64_t)meta->start + meta->bytes +
                            (uint64_t)(lastFill ? stateRows : 0u) * P * 16u <=
                        ringBytes,
        ctl.err);
    if (w.active && inRing) {
      const float* sD = reinterpret_cast<const float*>(base);
      constexpr bool hasD = MODE == DFB_BLEND_DEPTH || MODE == DFB_ZCOMPOSITE;
      const unsigned char* sC = base + (hasD ? (size_t)nf * P * 4 : 0);
      if (MODE == DFB_BLEND_ORDERED) {
        for (int i = 0; i < nf; ++i)
          over(Px<DT>::shared(sC + (size_t)i * P * px, t, meta->scale[i]), c0, c1, c2, al);
      } else if (MODE == DFB_AVERAGE) {
        for (int i = 0; i < nf; ++i) {
          const float4 v = Px<DT>::shared(sC + (size_t)i * P * px, t, meta->scale[i]);
          c0 += v.x; c1 += v.y; c2 += v.z; al += v.w;
        }
      } else if (MODE == DFB_ZCOMPOSITE) {
        const int first = meta->first;
        for (int i = 0; i < nf; ++i) {
          const uint64_t k = ((uint64_t)depth_bits(sD[i * P + t]) << 32) | (uint32_t)(first + i);
          if (k < best) {
            best = k;
            bestRgba = meta->rgba[i];
            bestScale = meta->scale[i];
          }
        }
      } else {
        for (int i = 0; i < nf; ++i) {
          const float z = sD[i * P + t];
          const float4 v = Px<DT>::shared(sC + (size_t)i * P * px, t, meta->scale[i]);
          if (covers(z)) {
            inOrder = inOrder && z >= last;
            last = z;
            over(v, c0, c1, c2, al);
          } else {
            emptyBits |= __float_as_uint(v.x) | __float_as_uint(v.y) | __float_as_uint(v.z) |
                         __float_as_uint(v.w);
          }
        }
      }
    }
    if (lastFill && stateRows && inRing) {
      const float4* sState = reinterpret_cast<const float4*>(base + meta->bytes);
      S0 = sState[t];
      M = sState[P + t];
      if (stateRows == 3u) CP = sState[2 * P + t];
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&emptyB[s]);
    ++jg;
  }
  if (MODE == DFB_AVERAGE) {
    const float kk = (float)total;
    c0 = __fdiv_rn(c0, kk); c1 = __fdiv_rn(c1, kk); c2 = __fdiv_rn(c2, kk); al = __fdiv_rn(al, kk);
  } else if (MODE == DFB_ZCOMPOSITE) {
    covered = (uint32_t)(best >> 32) != kInfBits;
    if (covered && w.active) {
      const float4 v = Px<DT>::global(bestRgba, w.p, bestScale);
      c0 = v.x; c1 = v.y; c2 = v.z; al = v.w;
    }
  } else if (MODE == DFB_BLEND_DEPTH) {
    exact = inOrder && emptyBits == 0u;
  }
  return true;
}

// Consumer group: one pixel per thread.  Its items' fills come from its own
// slots, in order.
template <int DT, int G, int PER, int FR>
__device__ void consumer(const FrameArgs* __restrict__ frames, const int* __restrict__ itemBase,
                         int nFrames, int totalItems, const LaunchCtl& ctl, unsigned char* ring,
                         ItemMeta* metas, uint64_t* fullB, uint64_t* emptyB, volatile int* abort,
                         const SrgbTables* tb, uint32_t ringBytes) {
  constexpr int S = kSlots / G;
  const int group = threadIdx.x / kP;
  const int t = threadIdx.x - group * kP;  // pixel of the item, 0 .. kP-1
  const int lane = t & 31, warp = t >> 5;
  int jg = 0;  // this group's fills taken
  const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
  // The pixel's accumulation state comes with the item's last fill, or, in
  // frames that do not stream it, is loaded by the consumer itself
  // (tile-major: each warp reads 512 contiguous bytes per buffer) at the
  // item's start, before the wait for its fragments.  For the narrow
  // storage formats in single-frame launches of 2 CTAs per SM with one
  // group, the loads are issued one item ahead -- while the group waits
  // for, blends and finishes the item before -- so that their latency is
  // hidden (FP16 at 5.5 fragments per tile: 0.1029 against 0.1058 ms).
  // Elsewhere that costs more than it hides: FP32 gains nothing, the
  // multi-frame launches pay a second frame search per item (batched graph
  // 1.99 against 1.74 ms), 3 CTAs per SM lose registers, and several groups
  // per CTA would spill.
  constexpr bool ahead = G == 1 && PER == 2 && FR == kOneFrame && DT != DFB_F32;
  auto load_state = [&](int it, float4& s0, float4& m2, float4& cp) {
    s0 = m2 = cp = zero4;
    if (it >= totalItems) return;
    const PixWork v = prepare<FR>(frames, itemBase, nFrames, it, t);
    const FrameArgs* B = v.A;
    if (v.active && (B->flags & DFB_FLAG_ACCUMULATE) && B->frameN != 1 && !B->stateInRing &&
        DFB_CHECK(v.sidx < (size_t)B->nTiles * B->T * B->T, ctl.err)) {
      s0 = B->accum[v.sidx];
      m2 = B->m2[v.sidx];
      if (B->kahan && !B->kahanFirst) cp = B->comp[v.sidx];
    }
  };
  float4 nS0, nM, nCP;  // the next item's state (loads one item ahead)
  if constexpr (ahead) load_state(blockIdx.x, nS0, nM, nCP);
  for (int k = group; ; k += G) {
    const int item = blockIdx.x + k * (int)gridDim.x;
    if (item >= totalItems) break;
    const PixWork w = prepare<FR>(frames, itemBase, nFrames, item, t);
    const FrameArgs* A = w.A;
    const bool accRead = w.active && (A->flags & DFB_FLAG_ACCUMULATE) && A->frameN != 1 &&
                         DFB_CHECK(w.sidx < (size_t)A->nTiles * A->T * A->T, ctl.err);
    const uint32_t stateRows =
        accRead && A->stateInRing ? ((A->kahan && !A->kahanFirst) ? 3u : 2u) : 0u;
    float4 S0, M, CP;
    if constexpr (ahead) {
      S0 = nS0;
      M = nM;
      CP = nCP;
      load_state(item + (int)gridDim.x, nS0, nM, nCP);
    } else {
      S0 = M = CP = zero4;
      if (accRead && !A->stateInRing) {
        S0 = A->accum[w.sidx];
        M = A->m2[w.sidx];
        if (A->kahan && !A->kahanFirst) CP = A->comp[w.sidx];
      }
    }
    int s = group * S + jg % S;
    if (!wait_phase(&fullB[s], (uint32_t)(jg / S) & 1u, ctl, abort)) {
      if (lane == 0) give_up(ctl, abort);
      break;
    }
    const ItemMeta* meta = metas + s;
    const int total = meta->total;
    const int P = w.P;
    float c0 = 0.f, c1 = 0.f, c2 = 0.f, al = 0.f;
    bool covered = true;
    if (total <= kN) {
      const unsigned char* base = ring + meta->start;
      // checked build: the item's fragments and state rows lie inside the ring
      const bool inRing = DFB_CHECK(
          meta->n <= kN && (uint64_t)meta->start + meta->bytes + (uint64_t)stateRows * P * 16u <=
                               ringBytes,
          ctl.err);
      if (w.active && inRing)
        covered = composite_staged<DT>(A->mode, total, P, base, meta, t, w.p, c0, c1, c2, al);
      // streamed state: from the ring into registers; then the ring space
      // goes back to the producer before the epilogue's math and stores
      if (stateRows && inRing) {
        const float4* sState = reinterpret_cast<const float4*>(base + meta->bytes);
        S0 = sState[t];
        M = sState[P + t];
        if (stateRows == 3u) CP = sState[2 * P + t];
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&emptyB[s]);  // ring space free for the producer
      ++jg;
    } else {
      // multi-fill item: kFill fragments per fill
      bool ok, exact = true;
      switch (A->mode) {
        case DFB_BLEND_DEPTH:
          ok = multi_fill<DT, DFB_BLEND_DEPTH, G>(total, w, t, lane, ctl, ring, metas, fullB,
                                                  emptyB, abort, ringBytes, group, jg, stateRows,
                                                  c0, c1, c2, al, covered, exact, S0, M, CP);
          break;
        case DFB_BLEND_ORDERED:
          ok = multi_fill<DT, DFB_BLEND_ORDERED, G>(total, w, t, lane, ctl, ring, metas, fullB,
                                                    emptyB, abort, ringBytes, group, jg, stateRows,
                                                    c0, c1, c2, al, covered, exact, S0, M, CP);
          break;
        case DFB_ZCOMPOSITE:
          ok = multi_fill<DT, DFB_ZCOMPOSITE, G>(total, w, t, lane, ctl, ring, metas, fullB,
                                                 emptyB, abort, ringBytes, group, jg, stateRows,
                                                 c0, c1, c2, al, covered, exact, S0, M, CP);
          break;
        default:
          ok = multi_fill<DT, DFB_AVERAGE, G>(total, w, t, lane, ctl, ring, metas, fullB, emptyB,
                                              abort, ringBytes, group, jg, stateRows, c0, c1,
                                              c2, al, covered, exact, S0, M, CP);
          break;
      }
      if (!ok) break;
      if (__any_sync(0xffffffffu, w.active && !exact)) {
        // out-of-order depths (or a non-zero empty fragment) in this warp's
        // 32 pixels: the exact re-do kernel composites them after this launch
        if (lane == 0) {
          const int slot = atomicAdd(ctl.redo, 1);
          ctl.redo[1 + slot] = item * (kP / 32) + warp;
        }
        continue;
      }
    }
    finish_pixel(A, w, lane, warp, c0, c1, c2, al, covered, S0, M, CP, tb, ctl.err);
  }
}

// FR = kOneFrame: a single-frame launch, whose arguments come as the kernel
// parameter `prm`; kParamTable: the frame table (and work-item prefix) of a
// launch of at most kParamFrames frames comes as `prm`; both are read from
// the parameter space.  kGlobalTable: `frames` and `itemBase` are the
// launch's tables in global memory.
template <int DT, int G, int PER, int FR>
__global__ void __launch_bounds__(Shape<G>::threads, PER)
    k_composite(const FrameArgs* __restrict__ frames, const int* __restrict__ itemBase,
                int nFrames, int totalItems, uint32_t ringBytes, LaunchCtl ctl,
                const __grid_constant__ typename FrameParams<FR>::type prm) {
  if constexpr (FR == kOneFrame) frames = &prm;
  if constexpr (FR == kParamTable) {
    frames = prm.f;
    itemBase = prm.itemBase;
  }
  extern __shared__ __align__(128) unsigned char smem[];
  SrgbTables* tb = reinterpret_cast<SrgbTables*>(smem);
  uint64_t* fullB = reinterpret_cast<uint64_t*>(smem + kOffBars);
  uint64_t* emptyB = fullB + kSlots;
  volatile int* abort = reinterpret_cast<volatile int*>(smem + kOffFlags);
  ItemMeta* metas = reinterpret_cast<ItemMeta*>(smem + kOffMetas);
  TileBlock* queue = reinterpret_cast<TileBlock*>(smem + kOffQueue);
  int4* qLoc = reinterpret_cast<int4*>(smem + kOffQLoc);
  uint64_t* queueB = emptyB + kSlots;
  unsigned char* ring = smem + kHeader;
  load_srgb(tb, Shape<G>::threads);
  if (threadIdx.x == 0) {
    for (int q = 0; q < kSlots; ++q) {
      mbar_init(&fullB[q], 1);
      mbar_init(&emptyB[q], kCW);
    }
    for (int q = 0; q < kMetaQ; ++q) mbar_init(&queueB[q], 1);
    *abort = 0;
    fence_barrier_init();
  }
  // The set-up above reads nothing that earlier kernels write; with a
  // programmatic launch it overlaps the end of the kernel before.
  grid_dependency_wait();
  allow_dependents();
  __syncthreads();
  if (threadIdx.x >= G * kP)
    producer<DT, G, FR>(frames, itemBase, nFrames, totalItems, ctl, ring, ringBytes, metas, queue, qLoc,
                 fullB, emptyB, queueB, abort);
  else
    consumer<DT, G, PER, FR>(frames, itemBase, nFrames, totalItems, ctl, ring, metas, fullB,
                             emptyB, abort, tb, ringBytes);
}

// Exact re-do of the 32-pixel units (work item, warp) that the persistent
// kernel left: multi-fill BLEND_DEPTH items whose depths were out of list
// order at some pixel, or that had a non-zero empty fragment.  Each warp of a
// CTA takes one unit at a time; each pixel reads its fragments from HBM and
// blends them in exact (depth, key, submit index) order through the
// windowed rounds of composite_exact, then goes through the same
// epilogue.  Units are rare on brick scenes, whose key order is their depth
// order; the kernel returns at once when there are none.
template <int DT>
__global__ void __launch_bounds__(kP, 2) k_composite_redo(const FrameArgs* __restrict__ frames,
                                                       const int* __restrict__ itemBase,
                                                       int nFrames, LaunchCtl ctl) {
  extern __shared__ __align__(128) unsigned char lsmem[];
  SrgbTables* tb = reinterpret_cast<SrgbTables*>(lsmem);
  uint64_t* window = reinterpret_cast<uint64_t*>(lsmem + sizeof(SrgbTables) + 128);
  const int count = *(volatile int*)ctl.redo;
  if ((int)blockIdx.x * (kP / 32) >= count) return;
  load_srgb(tb, kP);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  for (int u = blockIdx.x * (kP / 32) + (threadIdx.x >> 5); u < count;
       u += gridDim.x * (kP / 32)) {
    const int entry = ctl.redo[1 + u];
    const int item = entry / (kP / 32), iw = entry % (kP / 32);
    const int f = find_frame(itemBase, nFrames, item);
    const FrameArgs* A = frames + f;
    const int local = item - __ldg(itemBase + f);
    const int gt = A->tileBase + (local >> A->logChunks);
    if (!DFB_CHECK(f >= 0 && f < nFrames && (local >> A->logChunks) < A->nTiles, ctl.err))
      continue;
    const TileBlock* blk = A->blocks + gt;
    const int n = blk->n;
    const FragRec* list = A->srecs + blk->off;
    const PixWork w = prepare<kGlobalTable>(frames, itemBase, nFrames, item, iw * 32 + lane);
    float c0 = 0.f, c1 = 0.f, c2 = 0.f, al = 0.f;
    if (w.active) composite_exact<DT>(n, list, window, threadIdx.x, w.p, c0, c1, c2, al);
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 S = zero4, M = zero4, CP = zero4;
    if (w.active && (A->flags & DFB_FLAG_ACCUMULATE) && A->frameN != 1) {
      S = A->accum[w.sidx];
      M = A->m2[w.sidx];
      if (A->kahan && !A->kahanFirst) CP = A->comp[w.sidx];
    }
    finish_pixel(A, w, lane, iw, c0, c1, c2, al, true, S, M, CP, tb, ctl.err);
  }
}

// Per-tile variance: one warp per global tile sums the tile's per-warp
// partials in slot order.
__global__ void k_tile_variance(const FrameArgs* __restrict__ frames, int nFrames,
                                int totalTiles) {
  grid_dependency_wait();  // the composite's partials
  allow_dependents();
  const int gt = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (gt >= totalTiles) return;
  int lo = 0, hi = nFrames - 1;  // frame with the largest tileBase <= gt
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (frames[mid].tileBase <= gt) lo = mid; else hi = mid - 1;
  }
  const FrameArgs* A = frames + lo;
  if (!(A->flags & DFB_FLAG_ACCUMULATE)) return;
  const int tile = gt - A->tileBase;
  const int slots = A->slots;
  float sum = 0.0f;
  for (int q = lane; q < slots; q += 32) sum += A->varPartial[(size_t)tile * slots + q];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  if (lane == 0) {
    const int T = A->T;
    const int tx = tile % A->tilesX, ty = tile / A->tilesX;
    const int w = min(T, A->W - tx * T), h = min(T, A->H - ty * T);
    A->tileVar[tile] = sum / (3.0f * (float)(w * h));
  }
}

// Launch with programmatic stream serialisation: the kernel's blocks may be
// scheduled before the previous kernel in the stream has finished; the
// kernel's grid_dependency_wait() keeps its dependent accesses after it.
template <typename... Params, typename... Args>
cudaError_t launch_programmatic(void (*kernel)(Params...), int grid, int threads, size_t smem,
                                cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

template <int DT, int G, int PER>
cudaError_t launch_shape(const FrameArgs* frames, const int* itemBase, int nFrames,
                         int totalItems, int ringKB, const LaunchCtl& ctl,
                         const FrameArgs* hostFrames, const int* hostItemBase, cudaStream_t s) {
  auto kTable = k_composite<DT, G, PER, kGlobalTable>;
  auto kOne = k_composite<DT, G, PER, kOneFrame>;
  auto kParam = k_composite<DT, G, PER, kParamTable>;
  constexpr int per = PER;  // CTAs per SM
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  static int sms[64] = {0};
  static int smemMax[64] = {0};
  if (!sms[dev]) {
    int optin = 0, perSm = 0;
    e = cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
      e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess)
      e = cudaDeviceGetAttribute(&perSm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(kTable, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(kOne, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(kParam, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (e != cudaSuccess) {
      sms[dev] = 0;
      return e;
    }
    // per CTA: what `per` CTAs can share, less the 1 KB of shared memory CUDA
    // reserves for each CTA
    const int share = perSm / per - 1024;
    smemMax[dev] = share < optin ? share : optin;
  }
  uint32_t ring = (uint32_t)ringKB * 1024u;
  const uint32_t cap = (uint32_t)(smemMax[dev] - kHeader) & ~127u;
  if (ring > cap) ring = cap;
  if (ring < Bytes<DT>::maxItem) return cudaErrorInvalidConfiguration;
  int grid = sms[dev] * per;
  if (grid > totalItems) grid = totalItems;
  if (grid < 1) return cudaSuccess;
  const size_t smem = kHeader + ring;
  if (hostFrames && nFrames == 1)
    return launch_programmatic(kOne, grid, Shape<G>::threads, smem, s, frames, itemBase, nFrames,
                               totalItems, ring, ctl, hostFrames[0]);
  if (hostFrames && hostItemBase && nFrames <= kParamFrames) {
    FrameTable tab;
    memcpy(tab.itemBase, hostItemBase, sizeof(int) * (nFrames + 1));
    memcpy(tab.f, hostFrames, sizeof(FrameArgs) * nFrames);
    return launch_programmatic(kParam, grid, Shape<G>::threads, smem, s, frames, itemBase,
                               nFrames, totalItems, ring, ctl, tab);
  }
  return launch_programmatic(kTable, grid, Shape<G>::threads, smem, s, frames, itemBase, nFrames,
                             totalItems, ring, ctl, 0);
}

template <int DT>
cudaError_t launch_dt(const FrameArgs* frames, const int* itemBase, int nFrames, int totalItems,
                      const TuneParams& tune, const LaunchCtl& ctl, const FrameArgs* hostFrames,
                      const int* hostItemBase, cudaStream_t s) {
  const int per = tune.ctasPerSm, g = tune.groups;
#define DFB_SHAPE(G_, PER_)                                                                   \
  if (g == G_ && per == PER_)                                                                 \
    return launch_shape<DT, G_, PER_>(frames, itemBase, nFrames, totalItems, tune.ringKB, ctl,  \
                                      hostFrames, hostItemBase, s);
  DFB_SHAPE(1, 2)
  DFB_SHAPE(2, 2)
  DFB_SHAPE(1, 3)
  DFB_SHAPE(2, 1)
  DFB_SHAPE(3, 1)
#undef DFB_SHAPE
  return cudaErrorInvalidConfiguration;
}

}  // namespace

// Measured (composite launch, 16-frame accumulation): FP32 takes 2 CTAs per
// SM with one consumer group each and the largest ring they share.  The
// narrower formats fit their fills into the rings of 3 CTAs per SM, which is
// faster unless the frames are fragment-heavy: FP16 at 5.5 fragments per
// tile 0.1058 ms with 2 CTAs against 0.1095 ms with 3; at 4.4 fragments per
// tile 0.1028 against 0.0945 ms; at one fragment per tile 3 CTAs are faster
// too.  One CTA per SM is slower everywhere: its single producer warp sets
// the pace.
TuneParams default_tune(int dtype, double fragmentsPerTile) {
  if (dtype == DFB_F32 || fragmentsPerTile >= 5.0) return TuneParams{110, 2, 1};
  return TuneParams{72, 3, 1};
}

cudaError_t launch_composite(const FrameArgs* frames, const int* itemBase, int nFrames,
                             int totalItems, int totalTiles, bool accumulate, int dtype,
                             const TuneParams& tune, const LaunchCtl& ctl, const LongList& lng,
                             const FrameArgs* hostFrames, const int* hostItemBase,
                             cudaEvent_t afterMain, cudaStream_t s) {
  cudaError_t e;
  switch (dtype) {
    case DFB_F32:
      e = launch_dt<DFB_F32>(frames, itemBase, nFrames, totalItems, tune, ctl, hostFrames,
                                 hostItemBase, s);
      break;
    case DFB_F16:
      e = launch_dt<DFB_F16>(frames, itemBase, nFrames, totalItems, tune, ctl, hostFrames,
                                 hostItemBase, s);
      break;
    case DFB_BF16:
      e = launch_dt<DFB_BF16>(frames, itemBase, nFrames, totalItems, tune, ctl, hostFrames,
                                 hostItemBase, s);
      break;
    default:
      e = launch_dt<DFB_FP8E4M3>(frames, itemBase, nFrames, totalItems, tune, ctl, hostFrames,
                                 hostItemBase, s);
      break;
  }
  if (e == cudaSuccess && afterMain) e = cudaEventRecord(afterMain, s);
  // One-time set-up of the re-do kernel per device, done on any launch (so
  // that it never first happens inside a stream capture).
  static int sms[64] = {0};
  int dev = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess && (dev < 0 || dev >= 64)) e = cudaErrorInvalidDevice;
  const int smem = (int)(sizeof(SrgbTables) + 128 + kWindowBytes);
  if (e == cudaSuccess && !sms[dev]) {
    int count = 0;
    e = cudaDeviceGetAttribute(&count, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_composite_redo<DFB_F32>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_composite_redo<DFB_F16>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_composite_redo<DFB_BF16>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_composite_redo<DFB_FP8E4M3>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) sms[dev] = count;
  }
  if (e == cudaSuccess && lng.items > 0) {
    // at most one unit per warp of the long items; the count is on the device
    const int grid = lng.items < 2 * sms[dev] ? lng.items : 2 * sms[dev];
    switch (dtype) {
      case DFB_F32:
        k_composite_redo<DFB_F32><<<grid, kP, smem, s>>>(frames, itemBase, nFrames, ctl);
        break;
      case DFB_F16:
        k_composite_redo<DFB_F16><<<grid, kP, smem, s>>>(frames, itemBase, nFrames, ctl);
        break;
      case DFB_BF16:
        k_composite_redo<DFB_BF16><<<grid, kP, smem, s>>>(frames, itemBase, nFrames, ctl);
        break;
      default:
        k_composite_redo<DFB_FP8E4M3><<<grid, kP, smem, s>>>(frames, itemBase, nFrames, ctl);
        break;
    }
    e = cudaGetLastError();
  }
  if (e != cudaSuccess || !accumulate || totalTiles < 1) return e;
  return launch_programmatic(k_tile_variance, (totalTiles * 32 + 255) / 256, 256, 0, s, frames,
                             nFrames, totalTiles);
}

}  // namespace dfb
