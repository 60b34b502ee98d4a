// Arithmetic-throughput probes: the measured denominators of the ALU rooflines.
//
// The sweeps of the 37-velocity lattice (FP32, packed FP32x2) and the FP64
// D2Q9 sweep are bound by arithmetic, not by memory.  Their roofline fraction
// divides by what this GPU actually sustains for the same instruction kind,
// measured here: every thread runs kIlp independent chains of fused
// multiply-adds on registers (no memory traffic inside the loop), so the issue
// rate of the FMA pipe is the only limit.  The result is stored only under a
// condition no chain can meet, which keeps the compiler from removing the work.
#include "f32x2.cuh"
#include "lbm_internal.cuh"

namespace lbm {
namespace {

constexpr int kIlp = 8;  // independent chains per thread: covers the FMA latency at 4+ warps per scheduler

__global__ void probe_f32_kernel(int iters, float b, float c, float* __restrict__ sink) {
  float a[kIlp];
#pragma unroll
  for (int k = 0; k < kIlp; ++k) a[k] = (float)(threadIdx.x + k);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kIlp; ++k) a[k] = __fmaf_rn(a[k], b, c);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kIlp; ++k) s += a[k];
  if (s == -1.2345e-7f) sink[0] = s;  // never true for the probe's arguments
}

__global__ void probe_f32x2_kernel(int iters, float b, float c, float* __restrict__ sink) {
  f2 a[kIlp];
#pragma unroll
  for (int k = 0; k < kIlp; ++k) a[k] = pack2((float)(threadIdx.x + k), (float)(threadIdx.x + 2 * k));
  const f2 bb = pack2(b, b), cc = pack2(c, c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kIlp; ++k) a[k] = fma_(a[k], bb, cc);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kIlp; ++k) {
    float lo, hi;
    unpack2(a[k], lo, hi);
    s += lo + hi;
  }
  if (s == -1.2345e-7f) sink[0] = s;
}

__global__ void probe_f64_kernel(int iters, double b, double c, float* __restrict__ sink) {
  double a[kIlp];
#pragma unroll
  for (int k = 0; k < kIlp; ++k) a[k] = (double)(threadIdx.x + k);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kIlp; ++k) a[k] = __fma_rn(a[k], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kIlp; ++k) s += a[k];
  if (s == -1.2345e-7) sink[0] = (float)s;
}

}  // namespace
}  // namespace lbm

using namespace lbm;

extern "C" int lbm_alu_probe(int kind, int iters, int blocks, int threads, void* sink, void* stream,
                             double* flops) {
  if (kind < LBM_PROBE_F32 || kind > LBM_PROBE_F64) return set_error(LBM_EINVAL, "unknown probe kind %d", kind);
  if (iters < 1 || blocks < 1 || threads < 32 || threads > 1024 || (threads & 31))
    return set_error(LBM_EINVAL, "probe shape: iters %d, blocks %d, threads %d", iters, blocks, threads);
  if (!sink || !flops) return set_error(LBM_EINVAL, "NULL sink or flops pointer");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // b slightly below one and c small keep every chain finite for any iteration count
  const double b = 0.999999, c = 1e-6;
  const double lanes = kind == LBM_PROBE_F32X2 ? 2.0 : 1.0;
  *flops = 2.0 * lanes * kIlp * (double)iters * (double)blocks * (double)threads;
  float* s = static_cast<float*>(sink);
  if (kind == LBM_PROBE_F32)
    probe_f32_kernel<<<blocks, threads, 0, st>>>(iters, (float)b, (float)c, s);
  else if (kind == LBM_PROBE_F32X2)
    probe_f32x2_kernel<<<blocks, threads, 0, st>>>(iters, (float)b, (float)c, s);
  else
    probe_f64_kernel<<<blocks, threads, 0, st>>>(iters, b, c, s);
  return cuda_check(cudaGetLastError(), "probe launch");
}
