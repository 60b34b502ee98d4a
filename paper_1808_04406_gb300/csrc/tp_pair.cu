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
//
// D3Q27 with 16-bit offsets runs tp_pair_zrun_kernel: the same pairs, each
// thread walking several planes with the next plane's loads in flight.
#include <cstdlib>
#include <cstring>

#include "sweep_body.cuh"

namespace lbm {
namespace {

#ifndef LBM_PAIR_THREADS
#define LBM_PAIR_THREADS 128
#endif
#ifndef LBM_PAIR_MINB
#define LBM_PAIR_MINB 3
#endif
constexpr int kPairThreads = LBM_PAIR_THREADS;

template <int D, int S, bool ODD>
__global__ void __launch_bounds__(kPairThreads, LBM_PAIR_MINB)
    tp_pair_kernel(typename PairIO<S>::E* __restrict__ f, tp::Grid g, Rates r,
                   int* __restrict__ status, int z0) {
  const int xp = blockIdx.x * blockDim.x + threadIdx.x;
  if (xp >= (g.nx >> 1)) return;
  const int y = blockIdx.y, z = blockIdx.z + z0;  // z0: first plane of the swept range
  f2 om[2 * D + 1];
#pragma unroll
  for (int n = 0; n <= 2 * D; ++n) om[n] = cst<f2>(r.w[n]);
  if (!tp::update_pair<D, S, ODD>(f, g, om, xp, y, z)) atomicOr(status, 1);
}

// The same sweep for D3Q27 with 16-bit offsets, each thread walking kZRun
// consecutive planes of its pair column (x0, x0 + 1, y): the raw 16-bit words
// of the next plane's pair are loaded before the current pair is decoded and
// collided, so their latency overlaps the collision instead of stalling it.
// (AA slots belong to one node per sweep, so loading the next pair before the
// current one is stored is race-free.)  The node arithmetic is that of
// tp_pair_kernel, and so are the results, bit for bit.  At 4 blocks per SM the
// compiler keeps it within 128 registers without spills (the one-pair kernel
// needs 158-164 and so runs at 3).
constexpr int kZRun = 8;
constexpr int kZRunMinBlocks = 4;

template <int S, bool ODD>
__global__ void __launch_bounds__(kPairThreads, kZRunMinBlocks)
    tp_pair_zrun_kernel(typename PairIO<S>::E* __restrict__ f, tp::Grid g, Rates r, int* __restrict__ status,
                        int z0, int z1) {
  const int xp = blockIdx.x * blockDim.x + threadIdx.x;
  if (xp >= (g.nx >> 1)) return;
  const int y = blockIdx.y, zb = z0 + (int)blockIdx.z * kZRun;
  const int ze = zb + kZRun < z1 ? zb + kZRun : z1;  // planes zb .. ze - 1
  f2 om[7];
#pragma unroll
  for (int n = 0; n < 7; ++n) om[n] = cst<f2>(r.w[n]);
  RawPair raw[27];
  tp::pair_load_raw<3, S, ODD>(f, g, tp::PairAddr<3, ODD>(g, xp, y, zb), raw);
  bool ok = true;
  for (int z = zb; z < ze; ++z) {
    f2 v[27];
    tp::pair_decode<3, S, ODD>(raw, v);
    if (z + 1 < ze) tp::pair_load_raw<3, S, ODD>(f, g, tp::PairAddr<3, ODD>(g, xp, y, z + 1), raw);
    ok = tp::collide<f2, 3>(v, om) && ok;
    tp::pair_store<3, S, ODD>(f, g, tp::PairAddr<3, ODD>(g, xp, y, z), v);
  }
  if (!ok) atomicOr(status, 1);
}

// The plane-walking sweep with the totals of the consumed state, as
// tp_pair_totals_kernel computes them per node; each thread adds its nodes of
// all its planes in FP32 before the warp's shuffle tree, so there is one
// partial per warp of this grid (tp_pair_warps).
template <int S, bool ODD>
__global__ void __launch_bounds__(kPairThreads, 3)  // the running totals need more than 128 registers
    tp_pair_zrun_totals_kernel(typename PairIO<S>::E* __restrict__ f, tp::Grid g, Rates r,
                               int* __restrict__ status, float* __restrict__ partials, int z0, int z1) {
  const int xp = blockIdx.x * blockDim.x + threadIdx.x;
  float acc[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
  if (xp < (g.nx >> 1)) {
    const int y = blockIdx.y, zb = z0 + (int)blockIdx.z * kZRun;
    const int ze = zb + kZRun < z1 ? zb + kZRun : z1;
    f2 om[7];
#pragma unroll
    for (int n = 0; n < 7; ++n) om[n] = cst<f2>(r.w[n]);
    RawPair raw[27];
    tp::pair_load_raw<3, S, ODD>(f, g, tp::PairAddr<3, ODD>(g, xp, y, zb), raw);
    bool ok = true;
    for (int z = zb; z < ze; ++z) {
      f2 v[27];
      tp::pair_decode<3, S, ODD>(raw, v);
      if (z + 1 < ze) tp::pair_load_raw<3, S, ODD>(f, g, tp::PairAddr<3, ODD>(g, xp, y, z + 1), raw);
      tp::NodeMoments<f2, 3> m;
      ok = tp::collide<f2, 3, true>(v, om, &m) && ok;
      tp::pair_store<3, S, ODD>(f, g, tp::PairAddr<3, ODD>(g, xp, y, z), v);
      float d0, d1, jj0 = 0.0f, jj1 = 0.0f;
      unpack2(m.drho, d0, d1);
      acc[0] += d0 + d1;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        float j0, j1;
        unpack2(m.j[d], j0, j1);
        acc[1 + d] += j0 + j1;
        jj0 += j0 * j0;
        jj1 += j1 * j1;
      }
      acc[4] += __fdividef(0.5f * jj0, 1.0f + d0) + __fdividef(0.5f * jj1, 1.0f + d1);
    }
    if (!ok) atomicOr(status, 1);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 5; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_down_sync(0xffffffffu, acc[k], o);
  if (lane == 0) {
    const size_t b = (size_t)blockIdx.x + (size_t)gridDim.x * ((size_t)blockIdx.y + (size_t)gridDim.y * blockIdx.z);
    const size_t w = b * (kPairThreads / 32) + (size_t)wid;
#pragma unroll
    for (int k = 0; k < 5; ++k) partials[w * 8 + k] = acc[k];
  }
}

// The same sweep, which also writes per block the FP64 totals of the state it
// consumed: sum (rho - 1), sum rho u_d, sum rho |u|^2 / 2 (as the grid
// reduction defines them, per node from the collision's own moments) to
// partials[warp * 8 + k] (FP32), one entry per warp of the grid.  A warp sums
// its 64 nodes in FP32 (a fixed shuffle tree); the warps' sums are added in
// FP64 afterwards.  (FP64 arithmetic runs at a small fraction of the FP32 rate on
// this GPU: per-node FP64 sums would double the sweep's time; and no block
// barrier holds finished warps back.)
template <int D, int S, bool ODD>
__global__ void __launch_bounds__(kPairThreads, LBM_PAIR_MINB)
    tp_pair_totals_kernel(typename PairIO<S>::E* __restrict__ f, tp::Grid g, Rates r, int* __restrict__ status,
                          float* __restrict__ partials, int z0) {
  const int xp = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y, z = blockIdx.z + z0;
  float acc[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
  if (xp < (g.nx >> 1)) {
    f2 om[2 * D + 1];
#pragma unroll
    for (int n = 0; n <= 2 * D; ++n) om[n] = cst<f2>(r.w[n]);
    const tp::PairAddr<D, ODD> A(g, xp, y, z);
    f2 v[tp::qof<D>()];
    tp::pair_load<D, S, ODD>(f, g, A, v);
    tp::NodeMoments<f2, D> m;
    const bool ok = tp::collide<f2, D, true>(v, om, &m);
    tp::pair_store<D, S, ODD>(f, g, A, v);
    if (!ok) atomicOr(status, 1);
    float d0, d1, jj0 = 0.0f, jj1 = 0.0f;
    unpack2(m.drho, d0, d1);
    acc[0] = d0 + d1;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      float j0, j1;
      unpack2(m.j[d], j0, j1);
      acc[1 + d] = j0 + j1;
      jj0 += j0 * j0;
      jj1 += j1 * j1;
    }
    acc[4] = __fdividef(0.5f * jj0, 1.0f + d0) + __fdividef(0.5f * jj1, 1.0f + d1);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 5; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_down_sync(0xffffffffu, acc[k], o);
  if (lane == 0) {
    const size_t b = (size_t)blockIdx.x + (size_t)gridDim.x * ((size_t)blockIdx.y + (size_t)gridDim.y * blockIdx.z);
    const size_t w = b * (kPairThreads / 32) + (size_t)wid;
#pragma unroll
    for (int k = 0; k < 5; ++k) partials[w * 8 + k] = acc[k];
  }
}

// LBM_TP_ZRUN=0 keeps one pair per thread for 16-bit D3Q27 (read at every
// launch; used to compare the two kernels).
bool zrun_enabled() {
  const char* e = std::getenv("LBM_TP_ZRUN");
  return !(e && std::strcmp(e, "0") == 0);
}

template <int S>
cudaError_t launch_zrun(Sim* s, int odd) {
  using E = typename PairIO<S>::E;
  tp::Grid g{(int)s->nx, (int)s->ny, (int)s->nz, s->N};
  const int64_t pairs = s->nx / 2, nzs = active_nz(s);
  dim3 grid((unsigned)((pairs + kPairThreads - 1) / kPairThreads), (unsigned)s->ny,
            (unsigned)((nzs + kZRun - 1) / kZRun));
  const int z0 = (int)active_z0(s), z1 = (int)(active_z0(s) + nzs);
  E* f = static_cast<E*>(s->pop);
  if (odd)
    tp_pair_zrun_kernel<S, true><<<grid, kPairThreads, 0, s->stream>>>(f, g, s->rates, status_word(s), z0, z1);
  else
    tp_pair_zrun_kernel<S, false><<<grid, kPairThreads, 0, s->stream>>>(f, g, s->rates, status_word(s), z0, z1);
  return cudaGetLastError();
}

template <int D, int S>
cudaError_t launch(Sim* s, int odd) {
  using E = typename PairIO<S>::E;
  if constexpr (D == 3 && S != LBM_F32) {
    if (zrun_enabled()) return launch_zrun<S>(s, odd);
  }
  tp::Grid g{(int)s->nx, (int)s->ny, (int)s->nz, s->N};
  const int64_t pairs = s->nx / 2;
  dim3 block(kPairThreads);
  dim3 grid((unsigned)((pairs + kPairThreads - 1) / kPairThreads), (unsigned)s->ny, (unsigned)active_nz(s));
  const int z0 = (int)active_z0(s);
  E* f = static_cast<E*>(s->pop);
  if (odd)
    tp_pair_kernel<D, S, true><<<grid, block, 0, s->stream>>>(f, g, s->rates, status_word(s), z0);
  else
    tp_pair_kernel<D, S, false><<<grid, block, 0, s->stream>>>(f, g, s->rates, status_word(s), z0);
  return cudaGetLastError();
}

template <int S>
cudaError_t launch_zrun_totals(Sim* s, int odd, float* partials) {
  using E = typename PairIO<S>::E;
  tp::Grid g{(int)s->nx, (int)s->ny, (int)s->nz, s->N};
  const int64_t pairs = s->nx / 2, nzs = active_nz(s);
  dim3 grid((unsigned)((pairs + kPairThreads - 1) / kPairThreads), (unsigned)s->ny,
            (unsigned)((nzs + kZRun - 1) / kZRun));
  const int z0 = (int)active_z0(s), z1 = (int)(active_z0(s) + nzs);
  E* f = static_cast<E*>(s->pop);
  if (odd)
    tp_pair_zrun_totals_kernel<S, true><<<grid, kPairThreads, 0, s->stream>>>(f, g, s->rates, status_word(s),
                                                                               partials, z0, z1);
  else
    tp_pair_zrun_totals_kernel<S, false><<<grid, kPairThreads, 0, s->stream>>>(f, g, s->rates, status_word(s),
                                                                                partials, z0, z1);
  return cudaGetLastError();
}

template <int D, int S>
cudaError_t launch_totals(Sim* s, int odd, float* partials) {
  using E = typename PairIO<S>::E;
  if constexpr (D == 3 && S != LBM_F32) {
    if (zrun_enabled()) return launch_zrun_totals<S>(s, odd, partials);
  }
  tp::Grid g{(int)s->nx, (int)s->ny, (int)s->nz, s->N};
  const int64_t pairs = s->nx / 2;
  dim3 block(kPairThreads);
  dim3 grid((unsigned)((pairs + kPairThreads - 1) / kPairThreads), (unsigned)s->ny, (unsigned)active_nz(s));
  const int z0 = (int)active_z0(s);
  E* f = static_cast<E*>(s->pop);
  if (odd)
    tp_pair_totals_kernel<D, S, true><<<grid, block, 0, s->stream>>>(f, g, s->rates, status_word(s), partials, z0);
  else
    tp_pair_totals_kernel<D, S, false><<<grid, block, 0, s->stream>>>(f, g, s->rates, status_word(s), partials, z0);
  return cudaGetLastError();
}

template <int D>
cudaError_t launch_totals_d(Sim* s, int odd, float* partials) {
  switch (s->storage) {
    case LBM_F32: return launch_totals<D, LBM_F32>(s, odd, partials);
    case LBM_F16: return launch_totals<D, LBM_F16>(s, odd, partials);
    case LBM_BF16: return launch_totals<D, LBM_BF16>(s, odd, partials);
  }
  return cudaErrorInvalidValue;
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

const char* tp_pair_kernel_name(const Sim* s) {
  return s->D == 3 && s->storage != LBM_F32 && zrun_enabled() ? "tp_pair_zrun_kernel" : "tp_pair_kernel";
}

cudaError_t tp_launch_pair_sweep(Sim* s, int odd) {
  return s->D == 2 ? launch_d<2>(s, odd) : launch_d<3>(s, odd);
}

int64_t tp_pair_warps(const Sim* s) {
  const int64_t nz = active_nz(s);
  const int64_t planes = s->D == 3 && s->storage != LBM_F32 && zrun_enabled() ? (nz + kZRun - 1) / kZRun : nz;
  return ((s->nx / 2 + kPairThreads - 1) / kPairThreads) * s->ny * planes * (kPairThreads / 32);
}

cudaError_t tp_launch_pair_sweep_totals(Sim* s, int odd, float* partials) {
  return s->D == 2 ? launch_totals_d<2>(s, odd, partials) : launch_totals_d<3>(s, odd, partials);
}

}  // namespace lbm
