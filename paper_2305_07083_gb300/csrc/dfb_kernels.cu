// CUDA kernels of the DFB path for sm_103a, apart from the composite kernel
// (dfb_composite.cu):
//
//   K1  bucket:     records -> per-tile lists sorted by (order key, submit
//                   index): the routing of setTile to the tile owner
//                   (Sec. 3.1) and the rank order of the list tree (Sec. 4.2).
//   K6  convert:    producer-side FP16 / BF16 / FP8-e4m3 storage of tiles.
//   read-back:      normalised accumulation and per-pixel variance.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "dfb_internal.h"

namespace dfb {

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
// order in which the scatter's atomics placed the records.  The records are
// written in that order, and the tile's block gets its count, offset and
// first records.
__global__ void k1_segsort(const FragRec* __restrict__ recs, const int* __restrict__ counts,
                           const int* __restrict__ offsets, int nTiles,
                           const uint32_t* __restrict__ tmp, FragRec* __restrict__ srecs,
                           TileBlock* __restrict__ blocks) {
  const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (t >= nTiles) return;
  const int n = counts[t], off = offsets[t];
  if (lane == 0) {
    blocks[t].n = n;
    blocks[t].off = off;
  }
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
    if (j < n) {
      const FragRec r = recs[rj];
      srecs[off + rank] = r;
      if (rank < kStageFragments) blocks[t].recs[rank] = r;
    }
  }
}

cudaError_t launch_bucket(const FragRec* recs, int nRec, int nTilesTotal, int* counts,
                          int* offsets, int* cursor, uint32_t* tmp, FragRec* srecs,
                          TileBlock* blocks, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(int) * (size_t)nTilesTotal, s);
  if (e != cudaSuccess) return e;
  if (nRec > 0) k1_count<<<(nRec + 255) / 256, 256, 0, s>>>(recs, nRec, counts);
  k1_scan<<<1, 1024, 0, s>>>(counts, nTilesTotal, offsets, cursor);
  if (nRec > 0) k1_scatter<<<(nRec + 255) / 256, 256, 0, s>>>(recs, nRec, cursor, tmp);
  k1_segsort<<<(nTilesTotal * 32 + 255) / 256, 256, 0, s>>>(recs, counts, offsets, nTilesTotal,
                                                             tmp, srecs, blocks);
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
