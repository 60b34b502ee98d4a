// Block-level FP64 sums shared by the reduction kernels of every lattice:
// block partials are written to scratch, then one block adds them in a fixed
// order, so totals are deterministic.
#pragma once

#include "lbm_internal.cuh"

namespace lbm {
namespace {

constexpr int kAuxThreads = 256;

// Block-wide sum of NV doubles; result valid in thread 0.
template <int NV>
__device__ __forceinline__ void block_sum(double (&a)[NV]) {
  __shared__ double sh[kAuxThreads / 32][NV];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a[k] += __shfl_down_sync(0xffffffffu, a[k], o);
  }
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) sh[wid][k] = a[k];
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      a[k] = lane < kAuxThreads / 32 ? sh[lane][k] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) a[k] += __shfl_down_sync(0xffffffffu, a[k], o);
    }
  }
}

// Pass 2: one block sums the partials in a fixed order.
__global__ void __launch_bounds__(kAuxThreads)
    finalize_kernel(const double* __restrict__ partials, int nblocks, int nv,
                    double* __restrict__ out) {
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
    for (int k = 0; k < nv; ++k) acc[k] += partials[(size_t)b * 8 + k];
  block_sum<8>(acc);
  if (threadIdx.x == 0)
    for (int k = 0; k < nv; ++k) out[k] = acc[k];
}

}  // namespace
}  // namespace lbm
