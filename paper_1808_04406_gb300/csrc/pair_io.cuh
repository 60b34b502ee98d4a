// Two-node (packed FP32x2) loads and stores of one population for the storage
// types that the two-node sweeps support: an aligned 2-element access, or two
// 1-element accesses (x-shifted or wrapped slots).  FP16 / BF16 hold offsets
// scaled by 1/w (kScaled), which the caller applies.
#pragma once

#include "f32x2.cuh"
#include "lbm_internal.cuh"

namespace lbm {

// Raw storage bits of one population of a node pair, as loaded.  They are
// decoded to FP32x2 only when the pair is collided, so that a thread can keep
// the loads of later rows in flight meanwhile.  a: lane 0 (or both lanes of an
// aligned 16-bit pair), b: lane 1.
struct RawPair {
  uint32_t a, b;
};

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
  static __device__ __forceinline__ void raw2(const E* p, RawPair& r) {
    const unsigned long long w = *reinterpret_cast<const unsigned long long*>(p);
    r.a = (uint32_t)w;
    r.b = (uint32_t)(w >> 32);
  }
  static __device__ __forceinline__ void raw11(const E* a, const E* b, RawPair& r) {
    r.a = __float_as_uint(*a);
    r.b = __float_as_uint(*b);
  }
  static __device__ __forceinline__ f2 dec2(RawPair r) { return pack2(__uint_as_float(r.a), __uint_as_float(r.b)); }
  static __device__ __forceinline__ f2 dec11(RawPair r) { return dec2(r); }
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
  static __device__ __forceinline__ void raw2(const E* p, RawPair& r) { r.a = *reinterpret_cast<const uint32_t*>(p); }
  static __device__ __forceinline__ void raw11(const E* a, const E* b, RawPair& r) {
    r.a = *reinterpret_cast<const unsigned short*>(a);
    r.b = *reinterpret_cast<const unsigned short*>(b);
  }
  static __device__ __forceinline__ f2 dec2(RawPair r) { return bf16x2_bits_to_f2(r.a); }
  static __device__ __forceinline__ f2 dec11(RawPair r) {  // bf16 bits are the high half of the fp32 bits
    return pack2(__uint_as_float(r.a << 16), __uint_as_float(r.b << 16));
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
  static __device__ __forceinline__ void raw2(const E* p, RawPair& r) { r.a = *reinterpret_cast<const uint32_t*>(p); }
  static __device__ __forceinline__ void raw11(const E* a, const E* b, RawPair& r) {
    r.a = *reinterpret_cast<const unsigned short*>(a);
    r.b = *reinterpret_cast<const unsigned short*>(b);
  }
  static __device__ __forceinline__ f2 dec2(RawPair r) { return f16x2_bits_to_f2(r.a); }
  static __device__ __forceinline__ f2 dec11(RawPair r) { return f16x2_bits_to_f2(r.a | (r.b << 16)); }
  static constexpr bool kScaled = true;
};

}  // namespace lbm
