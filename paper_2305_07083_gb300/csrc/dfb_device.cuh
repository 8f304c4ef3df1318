// Device helpers shared by the DFB kernels: order-preserving depth keys,
// storage-format decoders, the front-to-back "over" step, the pixel
// operations (Sec. 3.1.2: exposure, Reinhard, the user's tone curve), the
// sRGB pack and the mbarrier / bulk-copy PTX wrappers used by the pipelined
// composite.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "dfb_internal.h"

namespace dfb {

// Order-preserving 32-bit image of a depth: NaN reads as +inf, -0 as +0.
__device__ __forceinline__ uint32_t depth_bits(float z) {
  uint32_t b = __float_as_uint(z);
  if ((b & 0x7fffffffu) > 0x7f800000u) b = 0x7f800000u;
  if (b == 0x80000000u) b = 0u;
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

// Bytes of one pixel's RGBA in each storage dtype.
template <int DT>
struct PxBytes {
  static constexpr int value = DT == DFB_F32 ? 16 : (DT == DFB_FP8E4M3 ? 4 : 8);
};

// Decode pixel p of a fragment's RGBA (global or shared memory) to FP32.
template <int DT>
struct Px;

template <>
struct Px<DFB_F32> {
  static __device__ __forceinline__ float4 global(const void* base, int p, float) {
    return __ldg(reinterpret_cast<const float4*>(base) + p);
  }
  static __device__ __forceinline__ float4 shared(const unsigned char* base, int p, float) {
    return reinterpret_cast<const float4*>(base)[p];
  }
};

__device__ __forceinline__ float4 decode_f16(uint2 v) {
  return make_float4(__half2float(__ushort_as_half((unsigned short)(v.x & 0xffffu))),
                     __half2float(__ushort_as_half((unsigned short)(v.x >> 16))),
                     __half2float(__ushort_as_half((unsigned short)(v.y & 0xffffu))),
                     __half2float(__ushort_as_half((unsigned short)(v.y >> 16))));
}

template <>
struct Px<DFB_F16> {
  static __device__ __forceinline__ float4 global(const void* base, int p, float) {
    return decode_f16(__ldg(reinterpret_cast<const uint2*>(base) + p));
  }
  static __device__ __forceinline__ float4 shared(const unsigned char* base, int p, float) {
    return decode_f16(reinterpret_cast<const uint2*>(base)[p]);
  }
};

__device__ __forceinline__ float4 decode_bf16(uint2 v) {
  return make_float4(__uint_as_float(v.x << 16), __uint_as_float(v.x & 0xffff0000u),
                     __uint_as_float(v.y << 16), __uint_as_float(v.y & 0xffff0000u));
}

template <>
struct Px<DFB_BF16> {
  static __device__ __forceinline__ float4 global(const void* base, int p, float) {
    return decode_bf16(__ldg(reinterpret_cast<const uint2*>(base) + p));
  }
  static __device__ __forceinline__ float4 shared(const unsigned char* base, int p, float) {
    return decode_bf16(reinterpret_cast<const uint2*>(base)[p]);
  }
};

__device__ __forceinline__ float4 decode_fp8(uint32_t v, float scale) {
  const float2 rg = e4m3x2_to_float2(v);
  const float2 ba = e4m3x2_to_float2(v >> 16);
  return make_float4(rg.x * scale, rg.y * scale, ba.x * scale, ba.y * scale);
}

template <>
struct Px<DFB_FP8E4M3> {
  static __device__ __forceinline__ float4 global(const void* base, int p, float scale) {
    return decode_fp8(__ldg(reinterpret_cast<const unsigned int*>(base) + p), scale);
  }
  static __device__ __forceinline__ float4 shared(const unsigned char* base, int p, float scale) {
    return decode_fp8(reinterpret_cast<const unsigned int*>(base)[p], scale);
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

// Value of a user tone curve at x: piecewise linear between the samples t[j]
// at x_j = xMax * j / (n - 1), with x clamped to [0, xMax] (NaN -> 0) and
// scale = (n - 1) / xMax.
__device__ __forceinline__ float curve_at(const float* __restrict__ t, int n, float xMax,
                                          float scale, float x) {
  x = fminf(fmaxf(x, 0.0f), xMax);  // fmaxf(NaN, 0) = 0
  const float f = x * scale;
  const int i = min((int)f, n - 2);
  const float fr = f - (float)i;
  const float a = __ldg(t + i), b = __ldg(t + i + 1);
  return fmaf(fr, b - a, a);
}

// Pixel operation before the display conversion (enum dfb_pixel_op) of the
// frame's settings: RGB transformed, alpha unchanged.
__device__ __forceinline__ float4 pixel_op(float4 v, const FrameArgs* A) {
  const int op = A->pixelOp;
  if (op == DFB_PIXELOP_NONE) return v;
  const float e = A->exposure;
  const float x = e * v.x, y = e * v.y, z = e * v.z;
  if (op == DFB_PIXELOP_EXPOSURE) return make_float4(x, y, z, v.w);
  if (op == DFB_PIXELOP_REINHARD)
    return make_float4(__fdiv_rn(x, 1.0f + x), __fdiv_rn(y, 1.0f + y), __fdiv_rn(z, 1.0f + z),
                       v.w);
  const int n = A->curveN;
  const float xm = A->curveXMax, sc = A->curveScale;
  const float* t = A->curve;
  return make_float4(curve_at(t, n, xm, sc, x), curve_at(t + n, n, xm, sc, y),
                     curve_at(t + 2 * n, n, xm, sc, z), v.w);
}

// sRGB code of a linear value: the number of code boundaries <= x, after
// clamping x to [0, 1] (NaN -> 0), read from the bucket table (SrgbTables).
__device__ __forceinline__ uint32_t srgb_code(float x, const SrgbTables* tb) {
  x = fminf(fmaxf(x, 0.0f), 1.0f);  // fmaxf(NaN, 0) = 0
  int i = (int)(__float_as_uint(x) >> 16) - kSrgbLutBias;
  i = min(max(i, 0), kSrgbLutEntries - 1);
  const uint32_t c = tb->lut[i];
  return c + (x >= tb->thr[c] ? 1u : 0u);
}

__device__ __forceinline__ uint32_t pack_rgba8(float4 v, const SrgbTables* tb) {
  const float a = fminf(fmaxf(v.w, 0.0f), 1.0f);  // fmaxf(NaN, 0) = 0
  const uint32_t A = (uint32_t)__float2int_rd(fmaf(255.0f, a, 0.5f));
  return srgb_code(v.x, tb) | (srgb_code(v.y, tb) << 8) | (srgb_code(v.z, tb) << 16) | (A << 24);
}

// ---- mbarrier and bulk-copy wrappers (sm_90+ PTX) ----
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Orders this thread's earlier generic-proxy accesses to shared memory before
// its later async-proxy (bulk copy) accesses.
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Programmatic dependent launch.  A kernel launched with programmatic stream
// serialisation may start while the kernel before it in the stream is still
// running; grid_dependency_wait() returns once that kernel has completed and
// its memory operations are visible (at once for a plain launch), so it comes
// before the first global access that depends on earlier work.
// allow_dependents() lets the next such kernel in the stream be scheduled
// (its blocks then wait in their own grid_dependency_wait()).
__device__ __forceinline__ void grid_dependency_wait() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}
__device__ __forceinline__ void allow_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// One-dimensional bulk copy global -> shared, completing on `bar`.
// Both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

}  // namespace dfb
