// Grid totals without any device allocation by the caller or the library.
//
// Some callers cannot call cudaMalloc: a plugin running inside a host
// application whose memory manager owns the whole device, or a time-critical
// loop that cannot afford cudaMalloc's implicit device-wide synchronisation.
// They may hold a population buffer handed to them, but no workspace.  For
// them lbm_reduce_noalloc computes the same FP64 totals as lbm_reduce with its
// scratch (block partials and result) in a fixed array that lives in this
// library's own device memory, reserved when the library is loaded.  It runs
// the same kernels on the same grid as lbm_reduce and returns the same bits.
#include <mutex>

#include "lbm_internal.cuh"

namespace lbm {
namespace {

// One row of 8 doubles per block partial (the reduction launches at most
// kRedBlocks blocks and strides over the grid, so this does not grow with the
// grid), then 8 doubles for the result: 77,888 bytes on every GPU that loads
// the library, held until the process exits.
constexpr int kNoallocBlocks = kRedBlocks;
constexpr int kNoallocResult = kNoallocBlocks * 8;
constexpr int kNoallocDoubles = kNoallocResult + 8;

static __device__ __align__(256) double g_noalloc_scratch[kNoallocDoubles];

// Device address of g_noalloc_scratch, per device, looked up by the first call
// on that device.  In host code the array's name is only a host-side stand-in;
// a kernel must be given this address.  The cache assumes the device's context
// lives as long as the process: it does not survive cudaDeviceReset.
constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
double* g_scratch_dev[kMaxDevices] = {};

int scratch_for_current_device(double** out) {
  int dev = -1;
  if (int rc = cuda_check(cudaGetDevice(&dev), "cudaGetDevice")) return rc;
  if (dev < 0 || dev >= kMaxDevices)
    return set_error(LBM_EINVAL, "device %d is beyond the %d devices supported", dev, kMaxDevices);
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    if (int rc = cuda_check(cudaGetSymbolAddress(&p, g_noalloc_scratch), "cudaGetSymbolAddress"))
      return rc;
    g_scratch_dev[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_dev[dev];
  return LBM_OK;
}

}  // namespace
}  // namespace lbm

using namespace lbm;

extern "C" int lbm_reduce_noalloc(int lattice, const int64_t dims[3], int storage, const void* pop,
                                  size_t pop_bytes, int64_t step, void* stream, double out[5]) {
  size_t need_pop = 0, need_work = 0;
  if (int rc = lbm_query_bytes(lattice, dims, storage, &need_pop, &need_work)) return rc;
  if (!pop || !out) return set_error(LBM_EINVAL, "NULL population or output pointer");
  // the same alignment lbm_create asks of a population buffer: the sweeps' and
  // the reduction's vector accesses assume it
  if ((uintptr_t)pop & 255) return set_error(LBM_EINVAL, "population buffer is not 256-byte aligned");
  if (pop_bytes < need_pop)
    return set_error(LBM_ESIZE, "population buffer too small: need %zu bytes, got %zu", need_pop,
                     pop_bytes);
  if (step < 0) return set_error(LBM_EINVAL, "negative step count");
  Sim s{};
  s.lattice = lattice;
  s.D = lattice == LBM_D3Q27 ? 3 : 2;
  s.Q = lattice == LBM_D2Q9 ? 9 : (lattice == LBM_D3Q27 ? 27 : 37);
  s.theta_ref = 1.0;  // the totals do not depend on the offset base temperature
  s.storage = storage;
  s.nx = dims[0];
  s.ny = dims[1];
  s.nz = dims[2];
  s.N = dims[0] * dims[1] * dims[2];
  s.pop = const_cast<void*>(pop);
  s.pop_bytes = pop_bytes;
  s.stream = static_cast<cudaStream_t>(stream);
  s.step = step;
  double* scratch = nullptr;
  if (int rc = scratch_for_current_device(&scratch)) return rc;
  // Every partial the finalize pass reads is written by this call's first pass
  // and the result is overwritten, so nothing has to be cleared beforehand.
  // the same grid as lbm_reduce, so both sum the block partials in the same
  // order and return the same bits
  int rc = cuda_check(launch_reduce_into(&s, scratch, kNoallocBlocks, scratch + kNoallocResult),
                      "reduction kernels");
  double tmp[5] = {0, 0, 0, 0, 0};
  if (!rc)
    rc = cuda_check(cudaMemcpyAsync(tmp, scratch + kNoallocResult, sizeof(tmp), cudaMemcpyDeviceToHost,
                                    s.stream),
                    "copy totals to host");
  if (!rc) rc = cuda_check(cudaStreamSynchronize(s.stream), "stream synchronize");
  if (!rc)
    for (int k = 0; k < 5; ++k) out[k] = tmp[k];
  return rc;
}
