// FP64 decay / frequency fit of a recorded single-wavenumber amplitude history
// (Sec. III.A: the time history of one Fourier component is fitted with the
// modal form A(t) = A(0) exp(omega t), Eq. modes; Re(omega) is the decay rate
// and Im(omega) the angular frequency).
#include <cmath>

#include "lbm_internal.cuh"

namespace lbm {
namespace {

constexpr int kFitThreads = 256;

__device__ __forceinline__ double block_sum_d(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double r = 0;
  if (threadIdx.x < 32) {
    r = threadIdx.x < kFitThreads / 32 ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
  }
  return r;  // valid in thread 0
}

// One block.  y_r = ln|A_r| and phi_r = arg(A_r) in parallel, phi unwrapped by
// thread 0 (consecutive records differ by less than pi), then the two
// least-squares slopes against t_r = r * stride.
__global__ void __launch_bounds__(kFitThreads)
    decay_fit_kernel(const double* __restrict__ hist, int n, double stride, double re_offset,
                     double* __restrict__ work, double* __restrict__ fit) {
  __shared__ double sh[kFitThreads / 32];
  double* y = work;
  double* ph = work + n;
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    const double re = hist[2 * r] + re_offset, im = hist[2 * r + 1];
    y[r] = 0.5 * log(re * re + im * im);
    ph[r] = atan2(im, re);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double two_pi = 6.283185307179586;
    double shift = 0;
    for (int r = 1; r < n; ++r) {
      const double raw = ph[r] + shift;
      const double d = raw - ph[r - 1];
      if (d > 0.5 * two_pi) shift -= two_pi;
      if (d < -0.5 * two_pi) shift += two_pi;
      ph[r] += shift;
    }
  }
  __syncthreads();
  const double tm = 0.5 * (double)(n - 1) * stride;
  double sy = 0, sp = 0;
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    sy += y[r];
    sp += ph[r];
  }
  const double ym = block_sum_d(sy, sh) / n;
  const double pm = block_sum_d(sp, sh) / n;
  __shared__ double means[2];
  if (threadIdx.x == 0) {
    means[0] = ym;
    means[1] = pm;
  }
  __syncthreads();
  double stt = 0, sty = 0, stp = 0;
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    const double dt = (double)r * stride - tm;
    stt += dt * dt;
    sty += dt * (y[r] - means[0]);
    stp += dt * (ph[r] - means[1]);
  }
  const double Stt = block_sum_d(stt, sh);
  const double Sty = block_sum_d(sty, sh);
  const double Stp = block_sum_d(stp, sh);
  if (threadIdx.x == 0) {
    const double gy = Stt > 0 ? Sty / Stt : 0.0;
    const double gp = Stt > 0 ? Stp / Stt : 0.0;
    fit[0] = -gy;                  // decay rate: |A| ~ exp(-fit[0] t)
    fit[1] = gp;                   // angular frequency of the phase
    fit[2] = means[0] - gy * tm;   // ln|A(0)| of the fitted line
    fit[3] = means[1] - gp * tm;   // phase at t = 0
  }
}

__global__ void fill_kernel(void* p, int dtype, int64_t n, double v) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    if (dtype == LBM_DTYPE_F64)
      static_cast<double*>(p)[k] = v;
    else
      static_cast<float*>(p)[k] = (float)v;
  }
}

}  // namespace

cudaError_t launch_fill(void* p, int dtype, int64_t n, double v, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  const int64_t blocks = (n + 255) / 256;
  fill_kernel<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, stream>>>(p, dtype, n, v);
  return cudaGetLastError();
}

cudaError_t launch_decay_fit(const double* hist, int n, double stride, double re_offset, double* fit,
                             cudaStream_t stream) {
  // scratch for y and phi: the 2n doubles right after the fit's 4 outputs
  decay_fit_kernel<<<1, kFitThreads, 0, stream>>>(hist, n, stride, re_offset, fit + 4, fit);
  return cudaGetLastError();
}

}  // namespace lbm
