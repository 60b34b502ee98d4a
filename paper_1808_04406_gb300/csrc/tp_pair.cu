// Fused stream + collide sweep, two neighbouring nodes (x0, x0 + 1) per thread,
// for FP32 / FP16 / BF16 offset storage on D2Q9 and D3Q27 (nx even).
//
// Same AA pattern and collision as the one-node sweep (tp_sweep.cu); the two
// nodes' values for one population sit in the two lanes of a packed FP32x2
// register, so every arithmetic instruction advances both nodes.
//
// Pairing.  The even sweep reads and writes the nodes' own slots, so it pairs
// (x0, x0 + 1) with x0 even and every access is one aligned 2-element access.
// The odd sweep touches slots shifted by e_x; it pairs (x0, x0 + 1 mod nx) with
// x0 odd, so that the shifted slots of e_x = -1 (x0 - 1, x0) and of e_x = +1
// (x0 + 1, x0 + 2, mod nx) start at an even x and stay aligned; only the nine
// populations with e_x = 0 need two 1-element accesses.  The last odd pair
// (nx - 1, 0) wraps around the row.
#include "tp_common.cuh"

namespace lbm {
namespace {

#ifndef LBM_PAIR_THREADS
#define LBM_PAIR_THREADS 128
#endif
#ifndef LBM_PAIR_MINB
#define LBM_PAIR_MINB 3
#endif
constexpr int kPairThreads = LBM_PAIR_THREADS;

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

template <int D, int S, bool ODD>
__global__ void __launch_bounds__(kPairThreads, LBM_PAIR_MINB)
    tp_pair_kernel(typename PairIO<S>::E* __restrict__ f, tp::Grid g, Rates r,
                   int* __restrict__ status) {
  using IO = PairIO<S>;
  using E = typename IO::E;
  constexpr int Q = tp::qof<D>();
  const int xp = blockIdx.x * blockDim.x + threadIdx.x;
  if (xp >= (g.nx >> 1)) return;
  const int x0 = 2 * xp + (ODD ? 1 : 0);                // lane 0's node
  const uint32_t x1 = (uint32_t)(x0 + 1 == g.nx ? 0 : x0 + 1);  // lane 1's node (odd sweep)
  const int y = blockIdx.y, z = blockIdx.z;
  f2 om[2 * D + 1];
#pragma unroll
  for (int n = 0; n <= 2 * D; ++n) om[n] = cst<f2>(r.w[n]);

  const uint32_t nx = (uint32_t)g.nx, nxy = (uint32_t)g.nx * (uint32_t)g.ny;
  // row offsets along y and z for e = -1, 0, +1 (periodic); the even sweep only uses e = 0
  uint32_t yo[3], zo[3];
  yo[1] = nx * (uint32_t)y;
  zo[1] = nxy * (uint32_t)z;
  if (ODD) {
    yo[0] = nx * (uint32_t)(y == 0 ? g.ny - 1 : y - 1);
    yo[2] = nx * (uint32_t)(y == g.ny - 1 ? 0 : y + 1);
    if (D == 3) {
      zo[0] = nxy * (uint32_t)(z == 0 ? g.nz - 1 : z - 1);
      zo[2] = nxy * (uint32_t)(z == g.nz - 1 ? 0 : z + 1);
    } else {
      zo[0] = zo[2] = 0;
    }
  }
  // aligned start of the slot pair for e_x = -1, 0 (even sweep), +1 (odd sweep: x1)
  const uint32_t xa[3] = {(uint32_t)(x0 - 1), (uint32_t)x0, x1};

  auto row = [&](int j) -> uint32_t {
    if (!ODD) return yo[1] + zo[1];
    return yo[tp::dig(j, 1)] + (D == 3 ? zo[tp::dig(j, 2)] : 0u);
  };

  f2 v[Q];
#pragma unroll
  for (int j = 0; j < Q; ++j) {
    const E* fj = f + (size_t)j * g.N + row(j);
    const int dx = tp::dig(j, 0);
    f2 val;
    if (!ODD)
      val = IO::load2(fj + x0);
    else if (dx == 1)
      val = IO::load11(fj + x0, fj + x1);
    else
      val = IO::load2(fj + xa[dx]);
    if (IO::kScaled) val = val * cst<f2>(tp::wq<D>(j));
    v[ODD ? tp::opp<D>(j) : j] = val;
  }
  const bool ok = tp::collide<f2, D>(v, om);
  if (!ok) atomicOr(status, 1);
#pragma unroll
  for (int j = 0; j < Q; ++j) {
    E* fj = f + (size_t)j * g.N + row(j);
    const int dx = tp::dig(j, 0);
    f2 val = ODD ? v[j] : v[tp::opp<D>(j)];
    if (IO::kScaled) val = val * cst<f2>(tp::iwq<D>(j));
    if (!ODD)
      IO::store2(fj + x0, val);
    else if (dx == 1)
      IO::store11(fj + x0, fj + x1, val);
    else
      IO::store2(fj + xa[dx], val);
  }
}

template <int D, int S>
cudaError_t launch(Sim* s, int odd) {
  using E = typename PairIO<S>::E;
  tp::Grid g{(int)s->nx, (int)s->ny, (int)s->nz, s->N};
  const int64_t pairs = s->nx / 2;
  dim3 block(kPairThreads);
  dim3 grid((unsigned)((pairs + kPairThreads - 1) / kPairThreads), (unsigned)s->ny, (unsigned)s->nz);
  E* f = static_cast<E*>(s->pop);
  if (odd)
    tp_pair_kernel<D, S, true><<<grid, block, 0, s->stream>>>(f, g, s->rates, status_word(s));
  else
    tp_pair_kernel<D, S, false><<<grid, block, 0, s->stream>>>(f, g, s->rates, status_word(s));
  return cudaGetLastError();
}

template <int D>
cudaError_t launch_d(Sim* s, int odd) {
  switch (s->storage) {
    case LBM_F32: return launch<D, LBM_F32>(s, odd);
    case LBM_F16: return launch<D, LBM_F16>(s, odd);
    case LBM_BF16: return launch<D, LBM_BF16>(s, odd);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

bool tp_pair_supported(const Sim* s) { return s->storage != LBM_F64 && (s->nx % 2) == 0; }

cudaError_t tp_launch_pair_sweep(Sim* s, int odd) {
  return s->D == 2 ? launch_d<2>(s, odd) : launch_d<3>(s, odd);
}

}  // namespace lbm
