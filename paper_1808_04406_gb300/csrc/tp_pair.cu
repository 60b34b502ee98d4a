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
                   int* __restrict__ status) {
  const int xp = blockIdx.x * blockDim.x + threadIdx.x;
  if (xp >= (g.nx >> 1)) return;
  const int y = blockIdx.y, z = blockIdx.z;
  f2 om[2 * D + 1];
#pragma unroll
  for (int n = 0; n <= 2 * D; ++n) om[n] = cst<f2>(r.w[n]);
  if (!tp::update_pair<D, S, ODD>(f, g, om, xp, y, z)) atomicOr(status, 1);
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
