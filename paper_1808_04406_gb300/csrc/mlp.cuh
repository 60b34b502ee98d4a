// Warp-level BF16 tensor-core building blocks of the 20 -> 64 -> 64 -> 6
// relaxation-rate network (mma.sync m16n8k16, FP32 accumulation).
//
// Fragment layout of mma.m16n8k16 (g = lane / 4, t = lane % 4):
//   A 16x16 row-major: a0 = A[g][2t..2t+1], a1 = A[g+8][2t..], a2 = A[g][2t+8..],
//                      a3 = A[g+8][2t+8..]  (lower column in the low 16 bits)
//   B 16x8:            b0 = B[2t..2t+1][g], b1 = B[2t+8..2t+9][g]
//   C 16x8 FP32:       c0 = C[g][2t], c1 = C[g][2t+1], c2 = C[g+8][2t], c3 = C[g+8][2t+1]
// Two neighbouring 16x8 accumulator tiles are exactly the A fragment of one
// 16-wide k-chunk of the next layer, so activations stay in registers.
//
// Weight images (BF16), rows padded by 8 elements so that the eight row groups
// g of a B-fragment load fall on distinct banks (row strides of 20 and 36
// words: g * stride mod 32 = distinct multiples of 4, plus t):
//   forward:  w1t[64][40] = W1^T (k padded 20 -> 32 with zeros),
//             w2t[64][72] = W2^T,  w3t[8][72] = W3^T (rows 6, 7 zero)
//   backward: w2s[64][72] = W2,    w3s[64][8] = W3 (columns 6, 7 zero)
// Parameter vector (FP32): W1[20][64], b1[64], W2[64][64], b2[64], W3[64][6], b3[6].
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace lbm {
namespace mlp {

constexpr int kIn = 20, kInPad = 32, kH = 64, kOut = 6, kOutPad = 8;
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kIn * kH, kOffW2 = kOffB1 + kH, kOffB2 = kOffW2 + kH * kH,
              kOffW3 = kOffB2 + kH, kOffB3 = kOffW3 + kH * kOut, kParams = kOffB3 + kOut;  // 5894

constexpr int kLd1 = kInPad + 8, kLdH = kH + 8;

struct FwdW {
  __nv_bfloat16 w1t[kH][kLd1];
  __nv_bfloat16 w2t[kH][kLdH];
  __nv_bfloat16 w3t[kOutPad][kLdH];
  float b1[kH], b2[kH], b3[kOutPad];
};
static_assert(sizeof(FwdW) % 16 == 0, "FwdW is copied in 16-byte units");

struct BwdW {
  __nv_bfloat16 w2s[kH][kLdH];
  __nv_bfloat16 w3s[kH][kOutPad];
};

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  uint32_t d;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}
__device__ __forceinline__ uint32_t ld32(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }
__device__ __forceinline__ uint32_t pack2h(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ void mma(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Fill the forward image from the FP32 parameter vector (whole block; the
// image may live in shared or global memory).  Padding columns are zero.
__device__ __forceinline__ void load_fwd(const float* __restrict__ P, FwdW& s) {
  for (int i = threadIdx.x; i < kH * kLd1; i += blockDim.x) {
    const int n = i / kLd1, k = i % kLd1;
    s.w1t[n][k] = __float2bfloat16_rn(k < kIn ? P[kOffW1 + k * kH + n] : 0.0f);
  }
  for (int i = threadIdx.x; i < kH * kLdH; i += blockDim.x) {
    const int a = i / kLdH, b = i % kLdH;
    s.w2t[a][b] = __float2bfloat16_rn(b < kH ? P[kOffW2 + b * kH + a] : 0.0f);  // W2^T[n=a][k=b] = W2[b][a]
  }
  for (int i = threadIdx.x; i < kOutPad * kLdH; i += blockDim.x) {
    const int n = i / kLdH, k = i % kLdH;
    s.w3t[n][k] = __float2bfloat16_rn(n < kOut && k < kH ? P[kOffW3 + k * kOut + n] : 0.0f);
  }
  for (int i = threadIdx.x; i < kH; i += blockDim.x) {
    s.b1[i] = P[kOffB1 + i];
    s.b2[i] = P[kOffB2 + i];
  }
  for (int i = threadIdx.x; i < kOutPad; i += blockDim.x) s.b3[i] = i < kOut ? P[kOffB3 + i] : 0.0f;
}

__device__ __forceinline__ void load_bwd(const float* __restrict__ P, BwdW& s) {
  for (int i = threadIdx.x; i < kH * kLdH; i += blockDim.x) {
    const int a = i / kLdH, b = i % kLdH;
    s.w2s[a][b] = __float2bfloat16_rn(b < kH ? P[kOffW2 + a * kH + b] : 0.0f);
  }
  for (int i = threadIdx.x; i < kH * kOutPad; i += blockDim.x) {
    const int k = i / kOutPad, n = i % kOutPad;
    s.w3s[k][n] = __float2bfloat16_rn(n < kOut ? P[kOffW3 + k * kOut + n] : 0.0f);
  }
}

// Copy a prepared forward image (global, 16-byte aligned) into shared memory.
__device__ __forceinline__ void copy_fwd(const FwdW* __restrict__ src, FwdW& dst) {
  const uint4* a = reinterpret_cast<const uint4*>(src);
  uint4* b = reinterpret_cast<uint4*>(&dst);
  for (int i = threadIdx.x; i < (int)(sizeof(FwdW) / 16); i += blockDim.x) b[i] = a[i];
}

// Forward pass of 16 rows (samples) held by one warp.  xs: 16 rows of 32 BF16
// inputs (row stride ldx elements; kLd1 keeps the A-fragment loads conflict-free).  Outputs: the hidden activations as A
// fragments (h1a[4][4], h2a[4][4]) and the FP32 logits z3[4] (C fragment).
// If h1s / h2s are given, the BF16 activations are also written there (16 rows,
// row stride kH) for the weight-gradient GEMMs.
__device__ __forceinline__ void forward16(const FwdW& s, const __nv_bfloat16* xs, int ldx, uint32_t (&h1a)[4][4],
                                          uint32_t (&h2a)[4][4], float (&z3)[4], __nv_bfloat16* h1s,
                                          __nv_bfloat16* h2s) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  uint32_t xa[2][4];
#pragma unroll
  for (int kc = 0; kc < 2; ++kc) {
    xa[kc][0] = ld32(xs + g * ldx + 16 * kc + 2 * t);
    xa[kc][1] = ld32(xs + (g + 8) * ldx + 16 * kc + 2 * t);
    xa[kc][2] = ld32(xs + g * ldx + 16 * kc + 2 * t + 8);
    xa[kc][3] = ld32(xs + (g + 8) * ldx + 16 * kc + 2 * t + 8);
  }
  // layer 1: 8 output tiles of 8
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    float c[4];
    c[0] = c[2] = s.b1[8 * nt + 2 * t];
    c[1] = c[3] = s.b1[8 * nt + 2 * t + 1];
#pragma unroll
    for (int kc = 0; kc < 2; ++kc)
      mma(c, xa[kc], ld32(&s.w1t[8 * nt + g][16 * kc + 2 * t]), ld32(&s.w1t[8 * nt + g][16 * kc + 2 * t + 8]));
#pragma unroll
    for (int k = 0; k < 4; ++k) c[k] = fmaxf(c[k], 0.0f);
    const uint32_t lo = pack_bf16(c[0], c[1]), hi = pack_bf16(c[2], c[3]);
    h1a[nt >> 1][(nt & 1) ? 2 : 0] = lo;
    h1a[nt >> 1][(nt & 1) ? 3 : 1] = hi;
    if (h1s) {
      *reinterpret_cast<uint32_t*>(h1s + g * kH + 8 * nt + 2 * t) = lo;
      *reinterpret_cast<uint32_t*>(h1s + (g + 8) * kH + 8 * nt + 2 * t) = hi;
    }
  }
  // layer 2
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    float c[4];
    c[0] = c[2] = s.b2[8 * nt + 2 * t];
    c[1] = c[3] = s.b2[8 * nt + 2 * t + 1];
#pragma unroll
    for (int kc = 0; kc < 4; ++kc)
      mma(c, h1a[kc], ld32(&s.w2t[8 * nt + g][16 * kc + 2 * t]), ld32(&s.w2t[8 * nt + g][16 * kc + 2 * t + 8]));
#pragma unroll
    for (int k = 0; k < 4; ++k) c[k] = fmaxf(c[k], 0.0f);
    const uint32_t lo = pack_bf16(c[0], c[1]), hi = pack_bf16(c[2], c[3]);
    h2a[nt >> 1][(nt & 1) ? 2 : 0] = lo;
    h2a[nt >> 1][(nt & 1) ? 3 : 1] = hi;
    if (h2s) {
      *reinterpret_cast<uint32_t*>(h2s + g * kH + 8 * nt + 2 * t) = lo;
      *reinterpret_cast<uint32_t*>(h2s + (g + 8) * kH + 8 * nt + 2 * t) = hi;
    }
  }
  // layer 3: one tile of 8 (6 used)
  z3[0] = z3[2] = s.b3[2 * t];
  z3[1] = z3[3] = s.b3[2 * t + 1];
#pragma unroll
  for (int kc = 0; kc < 4; ++kc)
    mma(z3, h2a[kc], ld32(&s.w3t[g][16 * kc + 2 * t]), ld32(&s.w3t[g][16 * kc + 2 * t + 8]));
}

}  // namespace mlp
}  // namespace lbm
