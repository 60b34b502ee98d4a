// Packed pair of FP32 values for Blackwell's two-wide FP32 instructions
// (PTX add/sub/mul/fma .rn.f32x2).  Lane 0 (low 32 bits) and lane 1 (high
// 32 bits) hold the same quantity for two neighbouring lattice nodes, so one
// instruction advances both.  Every operation rounds to nearest even, like the
// scalar float operations it replaces.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace lbm {

struct f2 {
  unsigned long long v;
};

__device__ __forceinline__ f2 pack2(float lo, float hi) {
  f2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void unpack2(f2 a, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a.v));
}
__device__ __forceinline__ f2 operator+(f2 a, f2 b) {
  f2 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
  return d;
}
__device__ __forceinline__ f2 operator-(f2 a, f2 b) {
  f2 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
  return d;
}
__device__ __forceinline__ f2 operator*(f2 a, f2 b) {
  f2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
  return d;
}
__device__ __forceinline__ f2 fma_(f2 a, f2 b, f2 c) {
  f2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d.v) : "l"(a.v), "l"(b.v), "l"(c.v));
  return d;
}

// ---- the same vocabulary for scalar compute types -----------------------------
__device__ __forceinline__ float fma_(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_(double a, double b, double c) { return __fma_rn(a, b, c); }

template <typename T>
__device__ __forceinline__ T cst(double c) {
  return (T)c;
}
template <>
__device__ __forceinline__ f2 cst<f2>(double c) {
  return pack2((float)c, (float)c);
}

// -x: a sign flip that scalar FMAs take for free as a negated operand; the
// packed type subtracts from zero.
template <typename T>
__device__ __forceinline__ T neg_(T x) {
  return -x;
}
template <>
__device__ __forceinline__ f2 neg_<f2>(f2 x) {
  return cst<f2>(0.0) - x;
}

// -u^2 given nu = -u, u and u^2: scalar types negate u^2 (free in the FMA that
// takes it); the packed type multiplies nu by u, a product independent of u^2
// (the same value), which schedules better in the packed sweeps.
template <typename T>
__device__ __forceinline__ T neg_sq(T nu, T u, T usq) {
  return neg_(usq);
}
template <>
__device__ __forceinline__ f2 neg_sq<f2>(f2 nu, f2 u, f2 usq) {
  return nu * u;
}

// 1/x lane by lane, correctly rounded (as the scalar division 1/x).
__device__ __forceinline__ float rcp_(float x) { return __frcp_rn(x); }
// FP64: Newton's iteration for the reciprocal, y <- y + y (1 - x y), from the
// correctly rounded FP32 reciprocal of x rounded to FP32.  The seed's relative
// error is below 2^-23 (two FP32 roundings), each step squares it (2^-46, then
// 2^-92) and the last step's own rounding leaves the result within one FP64 ulp
// of 1/x.  For x in the normal FP32 range (here x is a density near 1; x = 0
// gives NaN, which the physical-range check flags).  Two DFMA pairs against the
// longer sequence of a general FP64 division, on a GPU whose FP64 rate bounds
// the FP64 sweeps.
__device__ __forceinline__ double rcp_(double x) {
  double y = (double)__frcp_rn((float)x);
  double e = __fma_rn(-x, y, 1.0);
  y = __fma_rn(y, e, y);
  e = __fma_rn(-x, y, 1.0);
  return __fma_rn(y, e, y);
}
__device__ __forceinline__ f2 rcp_(f2 x) {
  float a, b;
  unpack2(x, a, b);
  return pack2(__frcp_rn(a), __frcp_rn(b));
}

// Physical-range check of (rho, |u|^2) for every lane: rho > 0 and |u|^2 < 1
// (false for NaN).
__device__ __forceinline__ bool sane(float rho, float usq) { return rho > 0.f && usq < 1.f; }
__device__ __forceinline__ bool sane(double rho, double usq) { return rho > 0.0 && usq < 1.0; }
__device__ __forceinline__ bool sane(f2 rho, f2 usq) {
  float r0, r1, u0, u1;
  unpack2(rho, r0, r1);
  unpack2(usq, u0, u1);
  return r0 > 0.f && r1 > 0.f && u0 < 1.f && u1 < 1.f;
}

// ---- 16-bit storage pairs -----------------------------------------------------
// bf16 -> fp32 is exact: the bf16 bits are the high half of the fp32 bits.
__device__ __forceinline__ f2 bf16x2_bits_to_f2(uint32_t w) {
  f2 r;
  const uint32_t lo = w << 16, hi = w & 0xffff0000u;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "r"(lo), "r"(hi));
  return r;
}
__device__ __forceinline__ uint32_t f2_to_bf16x2_bits(f2 a) {
  float lo, hi;
  unpack2(a, lo, hi);
  uint32_t d;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}
__device__ __forceinline__ f2 f16x2_bits_to_f2(uint32_t w) {
  const __half2 h = *reinterpret_cast<const __half2*>(&w);
  const float2 p = __half22float2(h);
  return pack2(p.x, p.y);
}
__device__ __forceinline__ uint32_t f2_to_f16x2_bits(f2 a) {
  float lo, hi;
  unpack2(a, lo, hi);
  uint32_t d;
  asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}

}  // namespace lbm
