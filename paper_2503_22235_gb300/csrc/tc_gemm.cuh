// tcgen05 GEMM building blocks shared by the GEMM kernels and the small-latent
// rollout kernel: shared-memory and instruction descriptors, the MMA issue
// wrappers (kind::f16 bf16 and kind::f8f6f4 e4m3, one CTA or a CTA pair), and
// the erf GELU used by the epilogues.
#pragma once

#include "tc_ptx.cuh"

namespace wm {
namespace tc {

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes, 8-row core-matrix groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);   // start address
  d |= (uint64_t)1 << 16;                      // leading byte offset (ignored for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;            // stride byte offset
  d |= (uint64_t)1 << 46;                      // descriptor version
  d |= (uint64_t)2 << 61;                      // 128-byte swizzle
  return d;
}

// Instruction descriptor, kind::f16: D f32, A and B bf16, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Instruction descriptor, kind::f8f6f4: D f32, A and B E4M3 (format 0), both K-major.
__host__ __device__ constexpr uint32_t idesc_e4m3(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

template <bool PAIR>
__device__ __forceinline__ void umma_e4m3(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  if constexpr (PAIR)
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
  else
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

template <bool PAIR>
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  if constexpr (PAIR)
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
  else
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// GELU(z) = z Phi(z) = 0.5 z (1 + erf(z / sqrt 2)) with erf from Abramowitz &
// Stegun, Handbook of Mathematical Functions, formula 7.1.26 (Hastings):
//   erf(x) = 1 - (a1 t + a2 t^2 + a3 t^3 + a4 t^4 + a5 t^5) exp(-x^2),
//   t = 1 / (1 + p x), x >= 0, |error| <= 1.5e-7,
// odd in x. Used for the bf16 / e4m3 outputs, whose rounding (>= 2^-9
// relative) dwarfs that error; the reciprocal and 2^x run on the MUFU unit.
__device__ __forceinline__ float gelu_erf(float z) {
  const float x = fabsf(z) * 0.70710678118654752f;
  float t;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(t) : "f"(fmaf(0.3275911f, x, 1.f)));
  float poly = fmaf(1.061405429f, t, -1.453152027f);
  poly = fmaf(poly, t, 1.421413741f);
  poly = fmaf(poly, t, -0.284496736f);
  poly = fmaf(poly, t, 0.254829592f);
  poly *= t;
  float e;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(-1.4426950408889634f * x * x));
  const float erf_abs = fmaf(-poly, e, 1.f);
  const float erf_z = copysignf(erf_abs, z);
  return 0.5f * z * (1.f + erf_z);
}

// gelu_erf on two values with paired instructions; every lane rounds exactly
// as gelu_erf does (same operations, same order; the polynomial is carried
// negated, with negated coefficients, which is exact).
__device__ __forceinline__ void gelu_erf2(float& z0, float& z1) {
  const uint64_t k_isqrt2 = pack_f2(0.70710678118654752f, 0.70710678118654752f);
  const uint64_t k_p = pack_f2(0.3275911f, 0.3275911f), k_one = pack_f2(1.f, 1.f);
  const uint64_t k_a5 = pack_f2(-1.061405429f, -1.061405429f), k_a4 = pack_f2(1.453152027f, 1.453152027f);
  const uint64_t k_a3 = pack_f2(-1.421413741f, -1.421413741f), k_a2 = pack_f2(0.284496736f, 0.284496736f);
  const uint64_t k_a1 = pack_f2(-0.254829592f, -0.254829592f);
  const uint64_t k_nl2e = pack_f2(-1.4426950408889634f, -1.4426950408889634f), k_half = pack_f2(0.5f, 0.5f);
  float x0 = fabsf(z0), x1 = fabsf(z1);
  mul_f2(x0, x1, k_isqrt2);
  float d0, d1;
  fma_f2(d0, d1, x0, x1, k_p, k_one);
  float t0, t1;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(t0) : "f"(d0));
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(t1) : "f"(d1));
  const uint64_t t2 = pack_f2(t0, t1);
  float p0, p1;   // -poly
  fma_f2(p0, p1, t0, t1, k_a5, k_a4);
  fma_f2(p0, p1, p0, p1, t2, k_a3);
  fma_f2(p0, p1, p0, p1, t2, k_a2);
  fma_f2(p0, p1, p0, p1, t2, k_a1);
  mul_f2(p0, p1, t2);
  float y0 = x0, y1 = x1;
  mul_f2(y0, y1, k_nl2e);
  mul_f2(y0, y1, pack_f2(x0, x1));
  float e0, e1;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e0) : "f"(y0));
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e1) : "f"(y1));
  float r0, r1;
  fma_f2(r0, r1, p0, p1, pack_f2(e0, e1), k_one);
  r0 = copysignf(r0, z0);
  r1 = copysignf(r1, z1);
  float o0, o1;
  add_f2(o0, o1, 1.f, 1.f, r0, r1);
  mul_f2(z0, z1, k_half);
  mul_f2(z0, z1, pack_f2(o0, o1));
}

}  // namespace tc
}  // namespace wm
