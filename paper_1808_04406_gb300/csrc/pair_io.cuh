// Two-node (packed FP32x2) loads and stores of one population for the storage
// types that the two-node sweeps support: an aligned 2-element access, or two
// 1-element accesses (x-shifted or wrapped slots).  FP16 / BF16 hold offsets
// scaled by 1/w (kScaled), which the caller applies.
#pragma once

#include "f32x2.cuh"
#include "lbm_internal.cuh"

namespace lbm {

template <int S>
struct PairIO;

template <>
struct PairIO<LBM_F32> {
  using E = float;
  static __device__ __forceinline__ f2 load2(const E* p) {
    f2 r;
    r.v = *reinterpret_cast<const unsigned long long*>(p);
    return r;
  }
  static __device__ __forceinline__ f2 load11(const E* a, const E* b) { return pack2(*a, *b); }
  static __device__ __forceinline__ void store2(E* p, f2 v) {
    *reinterpret_cast<unsigned long long*>(p) = v.v;
  }
  static __device__ __forceinline__ void store11(E* a, E* b, f2 v) {
    float lo, hi;
    unpack2(v, lo, hi);
    *a = lo;
    *b = hi;
  }
  static constexpr bool kScaled = false;
};

template <>
struct PairIO<LBM_BF16> {
  using E = __nv_bfloat16;
  static __device__ __forceinline__ f2 load2(const E* p) {
    return bf16x2_bits_to_f2(*reinterpret_cast<const uint32_t*>(p));
  }
  static __device__ __forceinline__ f2 load11(const E* a, const E* b) {
    const uint32_t lo = *reinterpret_cast<const unsigned short*>(a);
    const uint32_t hi = *reinterpret_cast<const unsigned short*>(b);
    return bf16x2_bits_to_f2(lo | (hi << 16));
  }
  static __device__ __forceinline__ void store2(E* p, f2 v) {
    *reinterpret_cast<uint32_t*>(p) = f2_to_bf16x2_bits(v);
  }
  static __device__ __forceinline__ void store11(E* a, E* b, f2 v) {
    const uint32_t w = f2_to_bf16x2_bits(v);
    *reinterpret_cast<unsigned short*>(a) = (unsigned short)(w & 0xffffu);
    *reinterpret_cast<unsigned short*>(b) = (unsigned short)(w >> 16);
  }
  static constexpr bool kScaled = true;
};

template <>
struct PairIO<LBM_F16> {
  using E = __half;
  static __device__ __forceinline__ f2 load2(const E* p) {
    return f16x2_bits_to_f2(*reinterpret_cast<const uint32_t*>(p));
  }
  static __device__ __forceinline__ f2 load11(const E* a, const E* b) {
    const uint32_t lo = *reinterpret_cast<const unsigned short*>(a);
    const uint32_t hi = *reinterpret_cast<const unsigned short*>(b);
    return f16x2_bits_to_f2(lo | (hi << 16));
  }
  static __device__ __forceinline__ void store2(E* p, f2 v) {
    *reinterpret_cast<uint32_t*>(p) = f2_to_f16x2_bits(v);
  }
  static __device__ __forceinline__ void store11(E* a, E* b, f2 v) {
    const uint32_t w = f2_to_f16x2_bits(v);
    *reinterpret_cast<unsigned short*>(a) = (unsigned short)(w & 0xffffu);
    *reinterpret_cast<unsigned short*>(b) = (unsigned short)(w >> 16);
  }
  static constexpr bool kScaled = true;
};

}  // namespace lbm
