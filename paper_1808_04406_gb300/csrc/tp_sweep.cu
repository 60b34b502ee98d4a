// Fused stream + collide sweep (one lattice Boltzmann time step) for the
// tensor-product lattices D2Q9 and D3Q27, in place with the AA pattern.
//
// One thread owns one node.  Even sweep: read the node's own slots, collide,
// write each result into the opposite slot of the same node.  Odd sweep: read
// population opp(j) from slot (x + e_j, j), collide, write population j to the
// same slot (x + e_j, j).  Both read and write exactly Q values per node, so a
// step moves 2 Q sizeof(storage) bytes per node through HBM.
//
// The collision is the CM-MRT operator of Sec. II.C (Eq. omega, final update)
// evaluated per axis in registers: populations -> raw moments -> central
// moments -> relax order by order -> raw moments -> populations.
#include "sweep_body.cuh"

namespace lbm {
namespace {

// Launch shape: threads per block along x, and the minimum resident blocks per
// SM requested from the register allocator.
#ifndef LBM_SWEEP_THREADS
#define LBM_SWEEP_THREADS 128
#endif
#ifndef LBM_SWEEP_MINB
#define LBM_SWEEP_MINB 1
#endif
constexpr int kSweepThreads = LBM_SWEEP_THREADS;

template <int D, int S, bool ODD>
__global__ void __launch_bounds__(kSweepThreads, LBM_SWEEP_MINB)
    tp_sweep_kernel(typename tp::Store<S>::type* __restrict__ f, tp::Grid g, Rates r,
                    int* __restrict__ status, int z0) {
  using T = typename tp::Store<S>::calc;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= g.nx) return;
  const int y = blockIdx.y, z = blockIdx.z + z0;  // z0: first plane of the swept range
  T om[2 * D + 1];
#pragma unroll
  for (int n = 0; n <= 2 * D; ++n) om[n] = (T)r.w[n];

  if (!tp::update_node<D, S, ODD>(f, g, om, x, y, z)) atomicOr(status, 1);
}

template <int D, int S>
cudaError_t launch(Sim* s, int odd) {
  using Tst = typename tp::Store<S>::type;
  tp::Grid g{(int)s->nx, (int)s->ny, (int)s->nz, s->N};
  dim3 block(kSweepThreads);
  dim3 grid((unsigned)((s->nx + kSweepThreads - 1) / kSweepThreads), (unsigned)s->ny, (unsigned)active_nz(s));
  Tst* f = static_cast<Tst*>(s->pop);
  const int z0 = (int)active_z0(s);
  if (odd)
    tp_sweep_kernel<D, S, true><<<grid, block, 0, s->stream>>>(f, g, s->rates, status_word(s), z0);
  else
    tp_sweep_kernel<D, S, false><<<grid, block, 0, s->stream>>>(f, g, s->rates, status_word(s), z0);
  return cudaGetLastError();
}

template <int D>
cudaError_t launch_d(Sim* s, int odd) {
  switch (s->storage) {
    case LBM_F64: return launch<D, LBM_F64>(s, odd);
    case LBM_F32: return launch<D, LBM_F32>(s, odd);
    case LBM_F16: return launch<D, LBM_F16>(s, odd);
    case LBM_BF16: return launch<D, LBM_BF16>(s, odd);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t tp_launch_sweep(Sim* s, int odd) {
  return s->D == 2 ? launch_d<2>(s, odd) : launch_d<3>(s, odd);
}

}  // namespace lbm
