// CUDA kernels of the DFB compositing path for sm_103a.
//
//   K1  bucket:     records -> per-tile lists sorted by (order key, submit
//                   index): the routing of setTile to the tile owner
//                   (Sec. 3.1) and the rank order of the list tree (Sec. 4.2).
//   K2  composite:  per pixel, the AlphaBlend tile operation (Sec. 4.2,
//                   Listing 4: sort the fragments by depth, blend "over"
//                   front to back, then the generation-0 background), the
//                   ordered list form, or depth (z) compositing (Sec. 2.1);
//                   fused with
//   K4  epilogue:   progressive accumulation (Listing 1: accumulation tile,
//                   accumulationID), Welford variance with a per-tile
//                   reduction (Listing 1: variance tile; Sec. 4.1.1), and the
//                   RGBA8 display conversion (Sec. 3.1).
//   K6  convert:    producer-side FP16 / BF16 / FP8-e4m3 storage of tiles.
//
// The path is bound by HBM bandwidth (about 0.4 flop per byte), so no tensor
// cores are used: every fragment pixel is streamed from HBM exactly once with
// coalesced 16-byte (FP32) / 8-byte (FP16, BF16) / 4-byte (FP8) loads, and
// the framebuffer state is read and written once per frame.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "dfb_internal.h"

namespace dfb {

// sRGB code boundaries: code c (1..255) starts at linear value g_srgb_thr[c-1];
// g_srgb_thr[255] = +inf.  Filled by ensure_tables() from the inverse of the
// IEC 61966-2-1 curve evaluated in double on the host.
__device__ float g_srgb_thr[256];

// ----------------------------------------------------------------------------
// helpers
// ----------------------------------------------------------------------------
__device__ __forceinline__ uint32_t depth_bits(float z) {
  uint32_t b = __float_as_uint(z);
  if ((b & 0x7fffffffu) > 0x7f800000u) b = 0x7f800000u;  // NaN reads as +inf
  if (b == 0x80000000u) b = 0u;                           // -0 reads as +0
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
constexpr uint32_t kInfBits = 0xff800000u;  // depth_bits(+inf)

__device__ __forceinline__ float2 e4m3x2_to_float2(uint32_t two_codes) {
  uint32_t h2;
  const unsigned short v = (unsigned short)(two_codes & 0xffffu);
  asm("cvt.rn.f16x2.e4m3x2 %0, %1;" : "=r"(h2) : "h"(v));
  return make_float2(__half2float(__ushort_as_half((unsigned short)(h2 & 0xffffu))),
                     __half2float(__ushort_as_half((unsigned short)(h2 >> 16))));
}

template <int DT>
struct Px;

template <>
struct Px<DFB_F32> {
  static __device__ __forceinline__ float4 load(const void* base, int p, float) {
    return __ldg(reinterpret_cast<const float4*>(base) + p);
  }
};

template <>
struct Px<DFB_F16> {
  static __device__ __forceinline__ float4 load(const void* base, int p, float) {
    const uint2 v = __ldg(reinterpret_cast<const uint2*>(base) + p);
    return make_float4(__half2float(__ushort_as_half((unsigned short)(v.x & 0xffffu))),
                       __half2float(__ushort_as_half((unsigned short)(v.x >> 16))),
                       __half2float(__ushort_as_half((unsigned short)(v.y & 0xffffu))),
                       __half2float(__ushort_as_half((unsigned short)(v.y >> 16))));
  }
};

template <>
struct Px<DFB_BF16> {
  static __device__ __forceinline__ float4 load(const void* base, int p, float) {
    const uint2 v = __ldg(reinterpret_cast<const uint2*>(base) + p);
    return make_float4(__uint_as_float(v.x << 16), __uint_as_float(v.x & 0xffff0000u),
                       __uint_as_float(v.y << 16), __uint_as_float(v.y & 0xffff0000u));
  }
};

template <>
struct Px<DFB_FP8E4M3> {
  static __device__ __forceinline__ float4 load(const void* base, int p, float scale) {
    const uint32_t v = __ldg(reinterpret_cast<const unsigned int*>(base) + p);
    const float2 rg = e4m3x2_to_float2(v);
    const float2 ba = e4m3x2_to_float2(v >> 16);
    return make_float4(rg.x * scale, rg.y * scale, ba.x * scale, ba.y * scale);
  }
};

__device__ __forceinline__ uint32_t srgb_code(float x, const float* thr) {
  // number of code boundaries <= x; NaN compares false everywhere -> 0
  uint32_t c = 0;
#pragma unroll
  for (uint32_t s = 128; s >= 1; s >>= 1)
    if (x >= thr[c + s - 1]) c += s;
  return c;
}

__device__ __forceinline__ uint32_t pack_rgba8(float4 v, const float* thr) {
  const float a = fminf(fmaxf(v.w, 0.0f), 1.0f);  // fmaxf(NaN, 0) = 0
  const uint32_t A = (uint32_t)__float2int_rd(fmaf(255.0f, a, 0.5f));
  return srgb_code(v.x, thr) | (srgb_code(v.y, thr) << 8) | (srgb_code(v.z, thr) << 16) |
         (A << 24);
}

// ----------------------------------------------------------------------------
// K1: bucketing
// ----------------------------------------------------------------------------
__global__ void k1_count(const FragRec* __restrict__ recs, int n, int* __restrict__ counts) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) atomicAdd(&counts[recs[i].tile], 1);
}

// One CTA of 1024 threads: exclusive scan of the per-tile counts.
__global__ void __launch_bounds__(1024) k1_scan(const int* __restrict__ counts, int nTiles,
                                                int* __restrict__ offsets,
                                                int* __restrict__ cursor) {
  __shared__ int warpSum[32];
  __shared__ int carry;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < nTiles; base += 1024) {
    const int i = base + threadIdx.x;
    const int v = i < nTiles ? counts[i] : 0;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warpSum[warp] = x;
    __syncthreads();
    if (warp == 0) {
      int w = warpSum[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      warpSum[lane] = w;
    }
    __syncthreads();
    const int excl = carry + (warp ? warpSum[warp - 1] : 0) + x - v;
    if (i < nTiles) {
      offsets[i] = excl;
      cursor[i] = excl;
    }
    __syncthreads();
    if (threadIdx.x == 1023) carry = excl + v;
    __syncthreads();
  }
}

__global__ void k1_scatter(const FragRec* __restrict__ recs, int n, int* __restrict__ cursor,
                           uint32_t* __restrict__ tmp) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) tmp[atomicAdd(&cursor[recs[i].tile], 1)] = (uint32_t)i;
}

// One warp per tile: each element's final position is its rank under the
// total order (key bits, record index), so the result does not depend on the
// order in which the scatter's atomics placed the records.
__global__ void k1_segsort(const FragRec* __restrict__ recs, const int* __restrict__ counts,
                           const int* __restrict__ offsets, int nTiles,
                           const uint32_t* __restrict__ tmp, uint32_t* __restrict__ sorted) {
  const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (t >= nTiles) return;
  const int n = counts[t], off = offsets[t];
  for (int jb = 0; jb < n; jb += 32) {
    const int j = jb + lane;
    uint32_t rj = 0;
    uint64_t kj = ~0ull;
    if (j < n) {
      rj = tmp[off + j];
      kj = ((uint64_t)recs[rj].key << 32) | rj;
    }
    int rank = 0;
    for (int mb = 0; mb < n; mb += 32) {
      const int m = mb + lane;
      uint64_t km = ~0ull;
      if (m < n) {
        const uint32_t rm = tmp[off + m];
        km = ((uint64_t)recs[rm].key << 32) | rm;
      }
      const int cnt = min(32, n - mb);
      for (int s = 0; s < cnt; ++s) rank += (__shfl_sync(0xffffffffu, km, s) < kj) ? 1 : 0;
    }
    if (j < n) sorted[off + rank] = rj;
  }
}

cudaError_t launch_bucket(const FragRec* recs, int nRec, int nTilesTotal, int* counts,
                          int* offsets, int* cursor, uint32_t* tmp, uint32_t* sorted,
                          cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(int) * (size_t)nTilesTotal, s);
  if (e != cudaSuccess) return e;
  if (nRec > 0) k1_count<<<(nRec + 255) / 256, 256, 0, s>>>(recs, nRec, counts);
  k1_scan<<<1, 1024, 0, s>>>(counts, nTilesTotal, offsets, cursor);
  if (nRec > 0) {
    k1_scatter<<<(nRec + 255) / 256, 256, 0, s>>>(recs, nRec, cursor, tmp);
    k1_segsort<<<(nTilesTotal * 32 + 255) / 256, 256, 0, s>>>(recs, counts, offsets,
                                                               nTilesTotal, tmp, sorted);
  }
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// K2/K3 + K4: one work item = kItemPixels pixels of one tile
// ----------------------------------------------------------------------------
struct ItemSmem {
  const void* rgba[kRecSmem];
  const float* depth[kRecSmem];
  float scale[kRecSmem];
  float thr[256];
  float red[kItemPixels / 32];
  int last;
};

struct FragView {
  const ItemSmem& sm;
  const FragRec* recs;
  const uint32_t* list;
  __device__ __forceinline__ const void* rgba(int i) const {
    return i < kRecSmem ? sm.rgba[i] : recs[list[i]].rgba;
  }
  __device__ __forceinline__ const float* depth(int i) const {
    return i < kRecSmem ? sm.depth[i] : recs[list[i]].depth;
  }
  __device__ __forceinline__ float scale(int i) const {
    return i < kRecSmem ? sm.scale[i] : recs[list[i]].scale;
  }
};

// Front-to-back "over": the fragment goes behind what is accumulated.
__device__ __forceinline__ void over(float4 f, float& c0, float& c1, float& c2, float& al) {
  const float t = 1.0f - al;
  c0 = fmaf(t, f.x, c0);
  c1 = fmaf(t, f.y, c1);
  c2 = fmaf(t, f.z, c2);
  al = fmaf(t, f.w, al);
}

// Insert key k into the sorted per-thread window kb[0..m-1] (stride
// kItemPixels), shifting larger keys up by one slot.  Slot m must be free.
__device__ __forceinline__ void window_insert(uint64_t* kb, int m, uint64_t k) {
  int j = m - 1;
  while (j >= 0) {
    const uint64_t v = kb[j * kItemPixels];
    if (v < k) break;
    kb[(j + 1) * kItemPixels] = v;
    --j;
  }
  kb[(j + 1) * kItemPixels] = k;
}

template <int MODE, int DT>
__device__ __forceinline__ void composite_item(const FrameArgs& a, int tile, int chunk,
                                               ItemSmem& sm, uint64_t* kbufAll) {
  const int tid = threadIdx.x;
  const int gt = a.tileBase + tile;
  const int n = a.counts[gt];
  const uint32_t* list = a.sorted + a.offsets[gt];
  const unsigned flags = a.flags;
  for (int i = tid; i < min(n, kRecSmem); i += kItemPixels) {
    const FragRec r = a.recs[list[i]];
    sm.rgba[i] = r.rgba;
    sm.depth[i] = r.depth;
    sm.scale[i] = r.scale;
  }
  if (flags & DFB_FLAG_PACK_RGBA8) sm.thr[tid] = g_srgb_thr[tid];
  __syncthreads();
  const FragView fv{sm, a.recs, list};

  const int T = a.T;
  const int tx = tile % a.tilesX, ty = tile / a.tilesX;
  const int p = chunk * kItemPixels + tid;
  const int x = tx * T + (p & (T - 1));
  const int y = ty * T + (p >> a.logT);
  const bool active = (p < T * T) && (x < a.W) && (y < a.H);

  float c0 = 0.0f, c1 = 0.0f, c2 = 0.0f, al = 0.0f;
  if (active) {
    if (MODE == DFB_BLEND_ORDERED) {
      for (int ib = 0; ib < n; ib += 8) {
        float4 c[8];
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (ib + u < n) c[u] = Px<DT>::load(fv.rgba(ib + u), p, fv.scale(ib + u));
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (ib + u < n) over(c[u], c0, c1, c2, al);
      }
    } else if (MODE == DFB_ZCOMPOSITE) {
      uint64_t best = ~0ull;
      for (int ib = 0; ib < n; ib += 8) {
        float z[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) z[u] = (ib + u < n) ? __ldg(fv.depth(ib + u) + p) : 0.0f;
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (ib + u < n) {
            const uint64_t k = ((uint64_t)depth_bits(z[u]) << 32) | (uint32_t)(ib + u);
            best = k < best ? k : best;
          }
      }
      if (n > 0 && (uint32_t)(best >> 32) != kInfBits) {
        const int i = (int)(uint32_t)best;
        const float4 f = Px<DT>::load(fv.rgba(i), p, fv.scale(i));
        c0 = f.x; c1 = f.y; c2 = f.z; al = f.w;
      } else {
        c0 = a.bgR; c1 = a.bgG; c2 = a.bgB; al = a.bgA;
      }
    } else {
      // Per-pixel sort by (depth, list position) in rounds of kSortWindow:
      // each round keeps the window's nearest keys above the last blended
      // one, then blends them in order.  Lists arrive sorted by key, so for
      // bricks whose key order matches their depth order every insertion is
      // an append.
      uint64_t* kb = kbufAll + tid;
      uint64_t lo = 0;
      int done = 0;
      while (done < n) {
        int m = 0;
        uint64_t last = 0;
        for (int ib = 0; ib < n; ib += 8) {
          float z[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) z[u] = (ib + u < n) ? __ldg(fv.depth(ib + u) + p) : 0.0f;
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int i = ib + u;
            if (i < n) {
              const uint64_t k = ((uint64_t)depth_bits(z[u]) << 32) | (uint32_t)i;
              if (done == 0 || k > lo) {
                if (m < kSortWindow) {
                  if (m == 0 || k > last) {
                    kb[m * kItemPixels] = k;
                    last = k;
                  } else {
                    window_insert(kb, m, k);
                  }
                  ++m;
                } else if (k < last) {
                  window_insert(kb, kSortWindow - 1, k);  // drops the largest
                  last = kb[(kSortWindow - 1) * kItemPixels];
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
              const int i = (int)(uint32_t)kb[(r + u) * kItemPixels];
              c[u] = Px<DT>::load(fv.rgba(i), p, fv.scale(i));
            }
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (r + u < m) over(c[u], c0, c1, c2, al);
        }
        lo = last;
        done += m;
      }
    }
    if (MODE != DFB_ZCOMPOSITE) over(make_float4(a.bgR, a.bgG, a.bgB, a.bgA), c0, c1, c2, al);
  }

  // ---- K4 epilogue: accumulate, variance, pack ----
  float vsum = 0.0f;
  if (active) {
    const float4 col = make_float4(c0, c1, c2, al);
    const size_t pix = (size_t)y * a.W + x;
    if (flags & DFB_FLAG_WRITE_COLOR) a.color[pix] = col;
    float4 out = col;
    if (flags & DFB_FLAG_ACCUMULATE) {
      const bool first = a.frameN == 1;
      const float4 S = first ? make_float4(0.f, 0.f, 0.f, 0.f) : a.accum[pix];
      float4 M = first ? make_float4(0.f, 0.f, 0.f, 0.f) : a.m2[pix];
      float4 Sn, tot;
      if (a.kahan) {
        const float4 cp = a.kahanFirst ? make_float4(0.f, 0.f, 0.f, 0.f) : a.comp[pix];
        float4 cn;
#define DFB_KAHAN(ch)                      \
  {                                        \
    const float yk = col.ch - cp.ch;       \
    const float tk = S.ch + yk;            \
    cn.ch = (tk - S.ch) - yk;              \
    Sn.ch = tk;                            \
    tot.ch = tk - cn.ch;                   \
  }
        DFB_KAHAN(x) DFB_KAHAN(y) DFB_KAHAN(z) DFB_KAHAN(w)
#undef DFB_KAHAN
        a.comp[pix] = cn;
      } else {
        Sn = make_float4(S.x + col.x, S.y + col.y, S.z + col.z, S.w + col.w);
        tot = Sn;
      }
      const float4 mean =
          make_float4(tot.x * a.invN, tot.y * a.invN, tot.z * a.invN, tot.w * a.invN);
      if (!first) {
        // Welford: M2 += (x - mean_{n-1}) (x - mean_n), mean_{n-1} = S_{n-1}/(n-1)
        M.x = fmaf(col.x - S.x * a.invNm1, col.x - mean.x, M.x);
        M.y = fmaf(col.y - S.y * a.invNm1, col.y - mean.y, M.y);
        M.z = fmaf(col.z - S.z * a.invNm1, col.z - mean.z, M.z);
        M.w = fmaf(col.w - S.w * a.invNm1, col.w - mean.w, M.w);
      }
      a.accum[pix] = Sn;
      a.m2[pix] = M;
      vsum = (M.x + M.y + M.z) * a.invNm1;
      out = mean;
    }
    if (flags & DFB_FLAG_PACK_RGBA8) a.rgba8[pix] = pack_rgba8(out, sm.thr);
  }

  if (flags & DFB_FLAG_ACCUMULATE) {
    // per-tile variance: warp shuffles, then the CTA, then the tile's last
    // finishing item sums the per-item partials in item order (deterministic)
    float v = vsum;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((tid & 31) == 0) sm.red[tid >> 5] = v;
    __syncthreads();
    if (tid == 0) {
      float s = 0.0f;
#pragma unroll
      for (int w = 0; w < kItemPixels / 32; ++w) s += sm.red[w];
      a.varPartial[(size_t)tile * a.chunks + chunk] = s;
      __threadfence();
      const unsigned prev = atomicAdd(&a.tileDone[tile], 1u);
      sm.last = (prev == (unsigned)a.chunks - 1u) ? 1 : 0;
    }
    __syncthreads();
    if (sm.last && tid == 0) {
      __threadfence();
      float s = 0.0f;
      for (int c = 0; c < a.chunks; ++c) s += __ldcg(&a.varPartial[(size_t)tile * a.chunks + c]);
      const int w = min(T, a.W - tx * T), h = min(T, a.H - ty * T);
      a.tileVar[tile] = s / (3.0f * (float)(w * h));
      a.tileDone[tile] = 0u;
    }
  }
  __syncthreads();  // shared memory is reused by the next item
}

template <int MODE, int DT>
__global__ void __launch_bounds__(kItemPixels) k_composite(const FrameArgs a) {
  __shared__ ItemSmem sm;
  extern __shared__ uint64_t kbuf[];
  composite_item<MODE, DT>(a, blockIdx.y, blockIdx.x, sm, kbuf);
}

constexpr size_t kKbufBytes = sizeof(uint64_t) * kSortWindow * kItemPixels;

template <int DT>
static cudaError_t launch_composite_dt(const FrameArgs& a, cudaStream_t s) {
  const dim3 grid(a.chunks, a.nTiles);
  switch (a.mode) {
    case DFB_BLEND_DEPTH:
      k_composite<DFB_BLEND_DEPTH, DT><<<grid, kItemPixels, kKbufBytes, s>>>(a);
      break;
    case DFB_BLEND_ORDERED:
      k_composite<DFB_BLEND_ORDERED, DT><<<grid, kItemPixels, 0, s>>>(a);
      break;
    default:
      k_composite<DFB_ZCOMPOSITE, DT><<<grid, kItemPixels, 0, s>>>(a);
      break;
  }
  return cudaGetLastError();
}

cudaError_t launch_composite(const FrameArgs& a, cudaStream_t s) {
  switch (a.dtype) {
    case DFB_F32: return launch_composite_dt<DFB_F32>(a, s);
    case DFB_F16: return launch_composite_dt<DFB_F16>(a, s);
    case DFB_BF16: return launch_composite_dt<DFB_BF16>(a, s);
    default: return launch_composite_dt<DFB_FP8E4M3>(a, s);
  }
}

// ----------------------------------------------------------------------------
// K5: persistent work-queue form over a batch of frames
// ----------------------------------------------------------------------------
template <int DT>
__global__ void __launch_bounds__(kItemPixels) k_composite_batch(
    const FrameArgs* __restrict__ frames, const int* __restrict__ itemBase, int nFrames,
    int totalItems, unsigned* __restrict__ queue) {
  __shared__ ItemSmem sm;
  __shared__ FrameArgs fa;
  __shared__ int sItem, sFrame;
  extern __shared__ uint64_t kbuf[];
  for (;;) {
    if (threadIdx.x == 0) {
      const int item = (int)atomicAdd(queue, 1u);
      sItem = item;
      if (item >= totalItems) {
        // every CTA fails exactly one fetch; the last one resets the queue
        if (item == totalItems + (int)gridDim.x - 1) *queue = 0u;
      } else {
        int lo = 0, hi = nFrames - 1;  // last frame with itemBase <= item
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (itemBase[mid] <= item) lo = mid; else hi = mid - 1;
        }
        sFrame = lo;
      }
    }
    __syncthreads();
    const int item = sItem;
    if (item >= totalItems) break;
    {
      const int* src = reinterpret_cast<const int*>(frames + sFrame);
      int* dst = reinterpret_cast<int*>(&fa);
      for (int w = threadIdx.x; w < (int)(sizeof(FrameArgs) / sizeof(int)); w += kItemPixels)
        dst[w] = src[w];
    }
    __syncthreads();
    const int local = item - itemBase[sFrame];
    const int tile = local / fa.chunks, chunk = local - tile * fa.chunks;
    switch (fa.mode) {
      case DFB_BLEND_DEPTH: composite_item<DFB_BLEND_DEPTH, DT>(fa, tile, chunk, sm, kbuf); break;
      case DFB_BLEND_ORDERED: composite_item<DFB_BLEND_ORDERED, DT>(fa, tile, chunk, sm, kbuf); break;
      default: composite_item<DFB_ZCOMPOSITE, DT>(fa, tile, chunk, sm, kbuf); break;
    }
  }
}

template <int DT>
static cudaError_t launch_batch_dt(const FrameArgs* frames, const int* itemBase, int nFrames,
                                   int totalItems, unsigned* queue, int ctasPerSm,
                                   cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  int grid = sms * (ctasPerSm > 0 ? ctasPerSm : 4);
  if (grid > totalItems) grid = totalItems > 0 ? totalItems : 1;
  k_composite_batch<DT><<<grid, kItemPixels, kKbufBytes, s>>>(frames, itemBase, nFrames,
                                                               totalItems, queue);
  return cudaGetLastError();
}

cudaError_t launch_composite_batch(const FrameArgs* frames, const int* itemBase, int nFrames,
                                   int totalItems, int dtype, unsigned* queue, int ctasPerSm,
                                   cudaStream_t s) {
  switch (dtype) {
    case DFB_F32: return launch_batch_dt<DFB_F32>(frames, itemBase, nFrames, totalItems, queue, ctasPerSm, s);
    case DFB_F16: return launch_batch_dt<DFB_F16>(frames, itemBase, nFrames, totalItems, queue, ctasPerSm, s);
    case DFB_BF16: return launch_batch_dt<DFB_BF16>(frames, itemBase, nFrames, totalItems, queue, ctasPerSm, s);
    default: return launch_batch_dt<DFB_FP8E4M3>(frames, itemBase, nFrames, totalItems, queue, ctasPerSm, s);
  }
}

// ----------------------------------------------------------------------------
// read-back helpers
// ----------------------------------------------------------------------------
__global__ void k_normalise(const float4* __restrict__ accum, const float4* __restrict__ comp,
                            int kahan, float invN, float4* __restrict__ out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    float4 s = accum[i];
    if (kahan) {
      const float4 c = comp[i];
      s = make_float4(s.x - c.x, s.y - c.y, s.z - c.z, s.w - c.w);
    }
    out[i] = make_float4(s.x * invN, s.y * invN, s.z * invN, s.w * invN);
  }
}

__global__ void k_variance(const float4* __restrict__ m2, float invNm1, float4* __restrict__ out,
                           int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float4 m = m2[i];
    out[i] = make_float4(m.x * invNm1, m.y * invNm1, m.z * invNm1, m.w * invNm1);
  }
}

static int grid_for(int64_t n) {
  int64_t g = (n + 255) / 256;
  return (int)(g > 4096 ? 4096 : (g < 1 ? 1 : g));
}

cudaError_t launch_normalise(const float4* accum, const float4* comp, int kahan, float invN,
                             float4* out, int64_t n, cudaStream_t s) {
  k_normalise<<<grid_for(n), 256, 0, s>>>(accum, comp, kahan, invN, out, n);
  return cudaGetLastError();
}

cudaError_t launch_variance(const float4* m2, float invNm1, float4* out, int64_t n,
                            cudaStream_t s) {
  k_variance<<<grid_for(n), 256, 0, s>>>(m2, invNm1, out, n);
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// K6: producer-side storage conversion
// ----------------------------------------------------------------------------
__global__ void k_to_f16(const float* __restrict__ src, __half* __restrict__ dst, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = __float2half_rn(src[i]);
}

__global__ void k_to_bf16(const float* __restrict__ src, __nv_bfloat16* __restrict__ dst,
                          int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = __float2bfloat16_rn(src[i]);
}

// One CTA per tile: amax, scale = amax / 448 (1 for an all-zero tile), then
// code = e4m3(x / scale) with round-to-nearest-even and saturation.
__global__ void __launch_bounds__(256) k_to_fp8(const float* __restrict__ src,
                                                uint8_t* __restrict__ dst,
                                                float* __restrict__ scales, int tileVals) {
  __shared__ float red[8];
  const float* s = src + (size_t)blockIdx.x * tileVals;
  uint8_t* d = dst + (size_t)blockIdx.x * tileVals;
  float m = 0.0f;
  for (int i = threadIdx.x; i < tileVals; i += 256) m = fmaxf(m, fabsf(s[i]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  float amax = 0.0f;
#pragma unroll
  for (int w = 0; w < 8; ++w) amax = fmaxf(amax, red[w]);
  const float scale = amax > 0.0f ? __fdiv_rn(amax, 448.0f) : 1.0f;
  if (threadIdx.x == 0) scales[blockIdx.x] = scale;
  for (int i = 2 * threadIdx.x; i < tileVals; i += 512) {
    const float lo = __fdiv_rn(s[i], scale);
    const float hi = (i + 1 < tileVals) ? __fdiv_rn(s[i + 1], scale) : 0.0f;
    unsigned short two;
    asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(two) : "f"(hi), "f"(lo));
    d[i] = (uint8_t)(two & 0xffu);
    if (i + 1 < tileVals) d[i + 1] = (uint8_t)(two >> 8);
  }
}

cudaError_t launch_convert(const float* src, void* dst, float* scales, int nTiles,
                           int tilePixels, int dtype, cudaStream_t s) {
  const int64_t n = (int64_t)nTiles * tilePixels * 4;
  switch (dtype) {
    case DFB_F16: k_to_f16<<<grid_for(n), 256, 0, s>>>(src, (__half*)dst, n); break;
    case DFB_BF16: k_to_bf16<<<grid_for(n), 256, 0, s>>>(src, (__nv_bfloat16*)dst, n); break;
    case DFB_FP8E4M3:
      k_to_fp8<<<nTiles, 256, 0, s>>>(src, (uint8_t*)dst, scales, tilePixels * 4);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// tables
// ----------------------------------------------------------------------------
cudaError_t upload_srgb_table(const float* host256) {
  return cudaMemcpyToSymbol(g_srgb_thr, host256, sizeof(float) * 256);
}

}  // namespace dfb
