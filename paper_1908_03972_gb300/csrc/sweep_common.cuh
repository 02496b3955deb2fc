// sweep_common.cuh -- CTA shapes and shared-memory prefetch layout of the
// residual-and-update kernels (binary64 and double-word variants).
#pragma once
#include "pmg_internal.h"

namespace pmg {

// Elements per CTA of the volume kernels.  Their threads are bound by FP64
// issue (binary64: 2 DFMA per clock per SM) or by the latency of their chain
// (double-word), so small CTAs of one or two warps spread even the coarse
// levels (4096 elements) over all 152 SMs.
template <int P>
struct ElemsPerBlock {
  static constexpr int N = (P + 1) * (P + 1);
  static constexpr int value = P == 0 ? 32 : P == 1 ? 8 : P == 2 ? 7 : P == 3 ? 4 : P == 4 ? 2 : 1;
};

// Prefetch layout of the residual-and-update sweep: the CTA's common face
// fluxes, block scales and (where they fit, VolPrefetch::blocks) block
// inverses are copied to shared memory by bulk asynchronous copies issued at
// entry, and the reference and forcing states are loaded into registers
// there too: the latency of these reads then overlaps the flux arithmetic
// instead of adding one L2 round trip per phase.
template <int P, class W>
struct VolPrefetch {
  static constexpr int n1 = P + 1, N = n1 * n1, EPB = ElemsPerBlock<P>::value, n = 4 * N;
  static constexpr bool blocks = (size_t)EPB * n * n * sizeof(W) <= 40 * 1024;
  static constexpr size_t dinv_bytes = blocks ? (size_t)EPB * n * n * sizeof(W) : 0;
  static constexpr size_t scale_bytes = (size_t)EPB * n * sizeof(double);   // rs, then cs
  static constexpr size_t flux_bytes = (size_t)EPB * 4 * n1 * sizeof(double);   // per equation
  static constexpr size_t smem = dinv_bytes + 2 * scale_bytes + 4 * flux_bytes;
};

// Loads four consecutive block entries (16-byte aligned for float, 32 for double).
__device__ __forceinline__ void ld4(const float* p, float a[4]) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  a[0] = t.x; a[1] = t.y; a[2] = t.z; a[3] = t.w;
}
__device__ __forceinline__ void ld4(const double* p, double a[4]) {
  const double2 t0 = reinterpret_cast<const double2*>(p)[0], t1 = reinterpret_cast<const double2*>(p)[1];
  a[0] = t0.x; a[1] = t0.y; a[2] = t1.x; a[3] = t1.y;
}
__device__ __forceinline__ void ldg4(const float* p, float a[4]) {
  const float4 t = __ldg(reinterpret_cast<const float4*>(p));
  a[0] = t.x; a[1] = t.y; a[2] = t.z; a[3] = t.w;
}
__device__ __forceinline__ void ldg4(const double* p, double a[4]) {
  const double2 t0 = __ldg(reinterpret_cast<const double2*>(p)), t1 = __ldg(reinterpret_cast<const double2*>(p) + 1);
  a[0] = t0.x; a[1] = t0.y; a[2] = t1.x; a[3] = t1.y;
}
// BF16 entries (8 bytes, 8-byte aligned), widened to FP32.
__device__ __forceinline__ void bf4_to_f(uint2 u, float a[4]) {
  const float2 lo = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.x));
  const float2 hi = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.y));
  a[0] = lo.x; a[1] = lo.y; a[2] = hi.x; a[3] = hi.y;
}
__device__ __forceinline__ void ld4(const __nv_bfloat16* p, float a[4]) {
  bf4_to_f(*reinterpret_cast<const uint2*>(p), a);
}
__device__ __forceinline__ void ldg4(const __nv_bfloat16* p, float a[4]) {
  bf4_to_f(__ldg(reinterpret_cast<const uint2*>(p)), a);
}

// rs .* F of a double-word F in the block precision W (rs: powers of two).
template <class W>
__device__ __forceinline__ typename Blk<W>::acc scaled_in_dw(dw F, double s);
template <>
__device__ __forceinline__ float scaled_in_dw<float>(dw F, double s) {
  return __fmul_rn(__fadd_rn(F.h, F.l), (float)s);
}
template <>
__device__ __forceinline__ double scaled_in_dw<double>(dw F, double s) {
  return dw_to_double(F) * s;
}
template <>
__device__ __forceinline__ float scaled_in_dw<__nv_bfloat16>(dw F, double s) {
  return __fmul_rn(__fadd_rn(F.h, F.l), (float)s);
}

}  // namespace pmg
