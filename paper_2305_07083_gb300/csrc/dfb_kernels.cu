// CUDA kernels of the DFB path for sm_103a, apart from the composite kernel
// (dfb_composite.cu):
//
//   K1  bucket:     per-tile lists (grouped by the host) sorted by (order key,
//                   submit index): the rank order of the list tree (Sec. 4.2)
//                   and the tile blocks the composite reads.
//   K6  convert:    producer-side FP16 / BF16 / FP8-e4m3 storage of tiles.
//   read-back:      normalised accumulation and per-pixel variance.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "dfb_internal.h"

namespace dfb {

// ----------------------------------------------------------------------------
// K1: bucketing
// ----------------------------------------------------------------------------
// Lists longer than this are sorted with a bitonic network in shared memory
// (one warp per tile); longer ones than kSortSmem by rank counting.
constexpr int kOrderWarps = 8;
constexpr int kSortSmem = 256;

// One warp per tile.  The tile's records arrive grouped, in submission order;
// the element at position i gets the key (order-key bits << 32 | i), and its
// final place is its rank under that key: the (key, submit index) order.
// Lists of up to 32 are ranked in registers, longer ones sorted in shared
// memory.
__global__ void __launch_bounds__(kOrderWarps * 32) k1_order(const FragRec* __restrict__ grouped,
                                                            const int* __restrict__ tileOff,
                                                            int nTiles, FragRec* __restrict__ srecs,
                                                            TileBlock* __restrict__ blocks,
                                                            int* __restrict__ redo) {
  __shared__ uint64_t keys[kOrderWarps][kSortSmem];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = blockIdx.x * kOrderWarps + warp;
  if (redo && blockIdx.x == 0 && threadIdx.x == 0) redo[0] = 0;
  if (t >= nTiles) return;
  const int off = __ldg(tileOff + t);
  const int n = __ldg(tileOff + t + 1) - off;
  if (lane == 0) {
    blocks[t].n = n;
    blocks[t].off = off;
  }
  const FragRec* in = grouped + off;
  if (n <= 32) {
    FragRec r{};
    uint64_t k = ~0ull;
    if (lane < n) {
      r = in[lane];
      k = ((uint64_t)r.key << 32) | (uint32_t)lane;
    }
    int rank = 0;
    for (int j = 0; j < n; ++j) rank += (__shfl_sync(0xffffffffu, k, j) < k) ? 1 : 0;
    if (lane < n) {
      srecs[off + rank] = r;
      if (rank < kStageFragments) blocks[t].recs[rank] = r;
    }
    return;
  }
  if (n <= kSortSmem) {
    uint64_t* a = keys[warp];
    int m = 64;
    while (m < n) m <<= 1;
    for (int i = lane; i < m; i += 32)
      a[i] = i < n ? (((uint64_t)__ldg(&in[i].key) << 32) | (uint32_t)i) : ~0ull;
    __syncwarp();
    for (int k = 2; k <= m; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int i = lane; i < m; i += 32) {
          const int p = i ^ j;
          if (p > i) {
            const uint64_t x = a[i], y = a[p];
            const bool up = (i & k) == 0;
            if ((x > y) == up) {
              a[i] = y;
              a[p] = x;
            }
          }
        }
        __syncwarp();
      }
    }
    for (int i = lane; i < n; i += 32) {
      const FragRec r = in[(uint32_t)a[i]];
      srecs[off + i] = r;
      if (i < kStageFragments) blocks[t].recs[i] = r;
    }
    return;
  }
  // very long lists: rank of each element by counting the smaller keys
  for (int jb = 0; jb < n; jb += 32) {
    const int j = jb + lane;
    const uint64_t kj = j < n ? (((uint64_t)__ldg(&in[j].key) << 32) | (uint32_t)j) : ~0ull;
    int rank = 0;
    for (int mb = 0; mb < n; mb += 32) {
      const int m = mb + lane;
      const uint64_t km = m < n ? (((uint64_t)__ldg(&in[m].key) << 32) | (uint32_t)m) : ~0ull;
      const int cnt = min(32, n - mb);
      for (int q = 0; q < cnt; ++q) rank += (__shfl_sync(0xffffffffu, km, q) < kj) ? 1 : 0;
    }
    if (j < n) {
      const FragRec r = in[j];
      srecs[off + rank] = r;
      if (rank < kStageFragments) blocks[t].recs[rank] = r;
    }
  }
}

cudaError_t launch_bucket(const FragRec* grouped, const int* tileOff, int nTiles, FragRec* srecs,
                          TileBlock* blocks, int* redo, cudaStream_t s) {
  const int grid = nTiles > 0 ? (nTiles + kOrderWarps - 1) / kOrderWarps : 1;
  k1_order<<<grid, kOrderWarps * 32, 0, s>>>(grouped, tileOff, nTiles, srecs, blocks, redo);
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// read-back helpers
// ----------------------------------------------------------------------------
__global__ void k_tiles_to_image(const float4* __restrict__ a, const float4* __restrict__ b,
                                 float scale, float4* __restrict__ out, int W, int H, int T,
                                 int logT, int tilesX) {
  const int64_t n = (int64_t)W * H;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int y = (int)(i / W), x = (int)(i - (int64_t)y * W);
    const int64_t src = ((int64_t)(y >> logT) * tilesX + (x >> logT)) * ((int64_t)T * T) +
                        ((y & (T - 1)) << logT) + (x & (T - 1));
    float4 v = a[src];
    if (b) {
      const float4 c = b[src];
      v = make_float4(v.x - c.x, v.y - c.y, v.z - c.z, v.w - c.w);
    }
    out[i] = make_float4(v.x * scale, v.y * scale, v.z * scale, v.w * scale);
  }
}

__global__ void k_image_to_tiles(const float4* __restrict__ in, float4* __restrict__ out, int W,
                                 int H, int T, int logT, int tilesX) {
  const int64_t n = (int64_t)W * H;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int y = (int)(i / W), x = (int)(i - (int64_t)y * W);
    const int64_t dst = ((int64_t)(y >> logT) * tilesX + (x >> logT)) * ((int64_t)T * T) +
                        ((y & (T - 1)) << logT) + (x & (T - 1));
    out[dst] = in[i];
  }
}

static int grid_for(int64_t n) {
  int64_t g = (n + 255) / 256;
  return (int)(g > 4096 ? 4096 : (g < 1 ? 1 : g));
}

static int log2_of(int T) {
  int l = 0;
  while ((1 << l) < T) ++l;
  return l;
}

cudaError_t launch_tiles_to_image(const float4* a, const float4* b, float scale, float4* out,
                                  int W, int H, int T, cudaStream_t s) {
  k_tiles_to_image<<<grid_for((int64_t)W * H), 256, 0, s>>>(a, b, scale, out, W, H, T, log2_of(T),
                                                            (W + T - 1) / T);
  return cudaGetLastError();
}

cudaError_t launch_image_to_tiles(const float4* in, float4* out, int W, int H, int T,
                                  cudaStream_t s) {
  k_image_to_tiles<<<grid_for((int64_t)W * H), 256, 0, s>>>(in, out, W, H, T, log2_of(T),
                                                            (W + T - 1) / T);
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

}  // namespace dfb
