// Per-node and per-node-pair sweep updates of the tensor-product lattices,
// shared by the single-grid sweeps (tp_sweep.cu, tp_pair.cu) and the batched
// sweep (batch.cu).  Each reads one node's (or pair's) populations in the AA
// layout of the given parity, collides, and writes them back to the slots the
// AA pattern prescribes.  Returns false when a node is unphysical.
#pragma once

#include "pair_io.cuh"
#include "tp_common.cuh"

namespace lbm {
namespace tp {

// One node (x, y, z): slot of population j in the AA layout of the parity.
template <int D, bool ODD>
struct NodeAddr {
  uint32_t node;
  uint32_t xo[3], yo[3], zo[3];
  __device__ __forceinline__ NodeAddr(const Grid& g, int x, int y, int z) {
    const uint32_t nx = (uint32_t)g.nx, nxy = (uint32_t)g.nx * (uint32_t)g.ny;
    node = (uint32_t)x + nx * (uint32_t)y + nxy * (uint32_t)z;
    // neighbour offsets along each axis for e = -1, 0, +1 (periodic)
    if (ODD) {
      xo[0] = (uint32_t)(x == 0 ? g.nx - 1 : x - 1);
      xo[1] = (uint32_t)x;
      xo[2] = (uint32_t)(x == g.nx - 1 ? 0 : x + 1);
      yo[0] = nx * (uint32_t)(y == 0 ? g.ny - 1 : y - 1);
      yo[1] = nx * (uint32_t)y;
      yo[2] = nx * (uint32_t)(y == g.ny - 1 ? 0 : y + 1);
      if (D == 3) {
        zo[0] = nxy * (uint32_t)(z == 0 ? g.nz - 1 : z - 1);
        zo[1] = nxy * (uint32_t)z;
        zo[2] = nxy * (uint32_t)(z == g.nz - 1 ? 0 : z + 1);
      } else {
        zo[0] = zo[1] = zo[2] = 0;
      }
    }
  }
  __device__ __forceinline__ uint32_t slot(int j) const {
    if (!ODD) return node;
    return xo[dig(j, 0)] + yo[dig(j, 1)] + (D == 3 ? zo[dig(j, 2)] : 0u);
  }
};

template <int D, int S, bool ODD>
__device__ __forceinline__ void node_load(const typename Store<S>::type* __restrict__ f, const Grid& g,
                                          const NodeAddr<D, ODD>& A, typename Store<S>::calc (&v)[qof<D>()]) {
#pragma unroll
  for (int j = 0; j < qof<D>(); ++j) {
    const auto val = decode<S, D>(f[(size_t)j * g.N + A.slot(j)], j);
    if (ODD)
      v[opp<D>(j)] = val;
    else
      v[j] = val;
  }
}

template <int D, int S, bool ODD>
__device__ __forceinline__ void node_store(typename Store<S>::type* __restrict__ f, const Grid& g,
                                           const NodeAddr<D, ODD>& A,
                                           const typename Store<S>::calc (&v)[qof<D>()]) {
#pragma unroll
  for (int j = 0; j < qof<D>(); ++j) f[(size_t)j * g.N + A.slot(j)] = encode<S, D>(ODD ? v[j] : v[opp<D>(j)], j);
}

// One node (x, y, z).  om[n]: rates of orders 0..2D in the compute type.
template <int D, int S, bool ODD>
__device__ __forceinline__ bool update_node(typename Store<S>::type* __restrict__ f, const Grid& g,
                                            const typename Store<S>::calc (&om)[2 * D + 1], int x, int y,
                                            int z) {
  using T = typename Store<S>::calc;
  const NodeAddr<D, ODD> A(g, x, y, z);
  T v[qof<D>()];
  node_load<D, S, ODD>(f, g, A, v);
  const bool ok = collide<T, D>(v, om);
  node_store<D, S, ODD>(f, g, A, v);
  return ok;
}

// Two nodes in packed FP32x2 (nx even).  Even sweep: pair (2 xp, 2 xp + 1), all
// accesses aligned.  Odd sweep: pair (2 xp + 1, 2 xp + 2 mod nx): the shifted
// slots of e_x = -1 and +1 start at an even x; only e_x = 0 needs two 1-element
// accesses.  The load and store halves are separate so that a caller walking
// several rows can issue the next row's loads before this row's collision (AA
// slots belong to exactly one node per step, so the reordering is race-free).
template <int D, bool ODD>
struct PairAddr {
  uint32_t yo[3], zo[3];
  uint32_t xa[3];
  int x0;
  uint32_t x1;
  __device__ __forceinline__ PairAddr(const Grid& g, int xp, int y, int z) {
    x0 = 2 * xp + (ODD ? 1 : 0);                        // lane 0's node
    x1 = (uint32_t)(x0 + 1 == g.nx ? 0 : x0 + 1);       // lane 1's node (odd sweep)
    const uint32_t nx = (uint32_t)g.nx, nxy = (uint32_t)g.nx * (uint32_t)g.ny;
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
    xa[0] = (uint32_t)(x0 - 1);
    xa[1] = (uint32_t)x0;
    xa[2] = x1;
  }
  __device__ __forceinline__ uint32_t row(int j) const {
    if (!ODD) return yo[1] + zo[1];
    return yo[dig(j, 1)] + (D == 3 ? zo[dig(j, 2)] : 0u);
  }
};

template <int D, int S, bool ODD>
__device__ __forceinline__ void pair_load_raw(const typename PairIO<S>::E* __restrict__ f, const Grid& g,
                                              const PairAddr<D, ODD>& A, RawPair (&r)[qof<D>()]) {
  using IO = PairIO<S>;
  using E = typename IO::E;
#pragma unroll
  for (int j = 0; j < qof<D>(); ++j) {
    const E* fj = f + (size_t)j * g.N + A.row(j);
    const int dx = dig(j, 0);
    if (!ODD)
      IO::raw2(fj + A.x0, r[j]);
    else if (dx == 1)
      IO::raw11(fj + A.x0, fj + A.x1, r[j]);
    else
      IO::raw2(fj + A.xa[dx], r[j]);
  }
}

template <int D, int S, bool ODD>
__device__ __forceinline__ void pair_decode(const RawPair (&r)[qof<D>()], f2 (&v)[qof<D>()]) {
  using IO = PairIO<S>;
#pragma unroll
  for (int j = 0; j < qof<D>(); ++j) {
    f2 val = (ODD && dig(j, 0) == 1) ? IO::dec11(r[j]) : IO::dec2(r[j]);
    if (IO::kScaled) val = val * cst<f2>(wq<D>(j));
    v[ODD ? opp<D>(j) : j] = val;
  }
}

template <int D, int S, bool ODD>
__device__ __forceinline__ void pair_load(const typename PairIO<S>::E* __restrict__ f, const Grid& g,
                                          const PairAddr<D, ODD>& A, f2 (&v)[qof<D>()]) {
  RawPair r[qof<D>()];
  pair_load_raw<D, S, ODD>(f, g, A, r);
  pair_decode<D, S, ODD>(r, v);
}

template <int D, int S, bool ODD>
__device__ __forceinline__ void pair_store(typename PairIO<S>::E* __restrict__ f, const Grid& g,
                                           const PairAddr<D, ODD>& A, const f2 (&v)[qof<D>()]) {
  using IO = PairIO<S>;
  using E = typename IO::E;
#pragma unroll
  for (int j = 0; j < qof<D>(); ++j) {
    E* fj = f + (size_t)j * g.N + A.row(j);
    const int dx = dig(j, 0);
    f2 val = ODD ? v[j] : v[opp<D>(j)];
    if (IO::kScaled) val = val * cst<f2>(iwq<D>(j));
    if (!ODD)
      IO::store2(fj + A.x0, val);
    else if (dx == 1)
      IO::store11(fj + A.x0, fj + A.x1, val);
    else
      IO::store2(fj + A.xa[dx], val);
  }
}

// Two nodes of one column in packed FP32x2 (2D, any nx): lane 0 is (x, y) and
// lane 1 is (x, y + 1), each lane reading and writing its own 1-element slots.
// This serves odd nx, where x-neighbour pairs are not aligned.  On the last row
// of an odd ny, lane 1 repeats lane 0's node: both lanes load the same slots,
// compute the same values and store them twice to the same places.
template <bool ODD>
struct YPairAddr {
  uint32_t xo[3];
  uint32_t ra[3], rb[3];  // row offsets of lane 0 and lane 1 for e_y = -1, 0, +1
  __device__ __forceinline__ YPairAddr(const Grid& g, int x, int y) {
    const uint32_t nx = (uint32_t)g.nx;
    const int y1 = y + 1 < g.ny ? y + 1 : y;
    xo[1] = (uint32_t)x;
    ra[1] = nx * (uint32_t)y;
    rb[1] = nx * (uint32_t)y1;
    if (ODD) {
      xo[0] = (uint32_t)(x == 0 ? g.nx - 1 : x - 1);
      xo[2] = (uint32_t)(x == g.nx - 1 ? 0 : x + 1);
      ra[0] = nx * (uint32_t)(y == 0 ? g.ny - 1 : y - 1);
      ra[2] = nx * (uint32_t)(y == g.ny - 1 ? 0 : y + 1);
      rb[0] = nx * (uint32_t)(y1 == 0 ? g.ny - 1 : y1 - 1);
      rb[2] = nx * (uint32_t)(y1 == g.ny - 1 ? 0 : y1 + 1);
    }
  }
  __device__ __forceinline__ uint32_t slot(int j, int lane) const {
    const int dx = ODD ? dig(j, 0) : 1, dy = ODD ? dig(j, 1) : 1;
    return xo[dx] + (lane ? rb[dy] : ra[dy]);
  }
};

template <int S, bool ODD>
__device__ __forceinline__ void ypair_load_raw(const typename PairIO<S>::E* __restrict__ f, const Grid& g,
                                               const YPairAddr<ODD>& A, RawPair (&r)[9]) {
  using IO = PairIO<S>;
#pragma unroll
  for (int j = 0; j < 9; ++j) {
    const typename IO::E* fj = f + (size_t)j * g.N;
    IO::raw11(fj + A.slot(j, 0), fj + A.slot(j, 1), r[j]);
  }
}

template <int S, bool ODD>
__device__ __forceinline__ void ypair_decode(const RawPair (&r)[9], f2 (&v)[9]) {
  using IO = PairIO<S>;
#pragma unroll
  for (int j = 0; j < 9; ++j) {
    f2 val = IO::dec11(r[j]);
    if (IO::kScaled) val = val * cst<f2>(wq<2>(j));
    v[ODD ? opp<2>(j) : j] = val;
  }
}

template <int S, bool ODD>
__device__ __forceinline__ void ypair_store(typename PairIO<S>::E* __restrict__ f, const Grid& g,
                                            const YPairAddr<ODD>& A, const f2 (&v)[9]) {
  using IO = PairIO<S>;
#pragma unroll
  for (int j = 0; j < 9; ++j) {
    typename IO::E* fj = f + (size_t)j * g.N;
    f2 val = ODD ? v[j] : v[opp<2>(j)];
    if (IO::kScaled) val = val * cst<f2>(iwq<2>(j));
    IO::store11(fj + A.slot(j, 0), fj + A.slot(j, 1), val);
  }
}

template <int D, int S, bool ODD>
__device__ __forceinline__ bool update_pair(typename PairIO<S>::E* __restrict__ f, const Grid& g,
                                            const f2 (&om)[2 * D + 1], int xp, int y, int z) {
  const PairAddr<D, ODD> A(g, xp, y, z);
  f2 v[qof<D>()];
  pair_load<D, S, ODD>(f, g, A, v);
  const bool ok = collide<f2, D>(v, om);
  pair_store<D, S, ODD>(f, g, A, v);
  return ok;
}

}  // namespace tp
}  // namespace lbm
