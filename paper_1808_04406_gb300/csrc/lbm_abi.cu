// C ABI of the library (declarations and contracts in include/lbm.h).
// Host-side validation, the AA step loop, and chunked host <-> device
// transfers through the workspace's staging area.  No device allocation.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "lbm_internal.cuh"
#include "tc05.cuh"

namespace lbm {

// closure.cu: whether the fused learned sweep runs its network on tcgen05 (else
// on mma.sync); read from the environment at every launch.
bool closure_uses_tcgen05();
// tp_pair.cu: the kernel tp_launch_pair_sweep launches for this handle.
const char* tp_pair_kernel_name(const Sim* s);

static thread_local char g_err[512] = "";

int set_error(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

int cuda_check(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return LBM_OK;
  return set_error(LBM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

size_t storage_elem_bytes(int storage) {
  switch (storage) {
    case LBM_F64: return 8;
    case LBM_F32: return 4;
    case LBM_F16:
    case LBM_BF16: return 2;
  }
  return 0;
}

namespace {

constexpr size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

struct Shape {
  int D, Q;
  int64_t nx, ny, nz, N;
};

int check_shape(int lattice, const int64_t dims[3], int storage, Shape* sh) {
  if (!dims) return set_error(LBM_EINVAL, "dims is NULL");
  if (lattice == LBM_D2Q9) {
    sh->D = 2;
    sh->Q = 9;
  } else if (lattice == LBM_D3Q27) {
    sh->D = 3;
    sh->Q = 27;
  } else if (lattice == LBM_D2Q37) {
    sh->D = 2;
    sh->Q = 37;
  } else {
    return set_error(LBM_EINVAL, "unknown lattice %d", lattice);
  }
  if (storage_elem_bytes(storage) == 0) return set_error(LBM_EINVAL, "unknown storage %d", storage);
  sh->nx = dims[0];
  sh->ny = dims[1];
  sh->nz = dims[2];
  if (sh->nx < 1 || sh->ny < 1 || sh->nz < 1)
    return set_error(LBM_EINVAL, "dims must be >= 1, got %lld x %lld x %lld", (long long)sh->nx,
                     (long long)sh->ny, (long long)sh->nz);
  if (sh->D == 2 && sh->nz != 1) return set_error(LBM_EINVAL, "dims[2] must be 1 on a 2D lattice");
  if (lattice == LBM_D2Q37 && (sh->nx < 3 || sh->ny < 3))
    return set_error(LBM_EINVAL, "the 37-velocity lattice needs nx, ny >= 3");
  if (sh->ny > 65535 || sh->nz > 65535)
    return set_error(LBM_EINVAL, "ny and nz must be <= 65535");
  const double n = (double)sh->nx * (double)sh->ny * (double)sh->nz;
  if (n >= 2147483648.0) return set_error(LBM_EINVAL, "nx * ny * nz must be < 2^31");
  sh->N = sh->nx * sh->ny * sh->nz;
  return LBM_OK;
}

size_t staging_bytes_for(const Shape& sh) {
  const size_t want = round256((size_t)sh.N * (size_t)sh.Q * sizeof(double));
  return want < kStagingMax ? want : kStagingMax;
}

int set_rates(Sim* s, const double* tau, int n_tau) {
  if (n_tau < 0 || (n_tau > 0 && !tau)) return set_error(LBM_EINVAL, "tau_per_order is NULL");
  Rates r{};
  const int top = s->lattice == LBM_D2Q37 ? 4 : s->lattice == LBM_HERMITE ? s->hl.order : 2 * s->D;
  for (int n = 2; n <= top; ++n) {
    const double t = (n - 2 < n_tau) ? tau[n - 2] : 1.0;
    if (!(t > 0.5) || !std::isfinite(t))
      return set_error(LBM_EINVAL, "tau of order %d must be finite and > 1/2 (got %g)", n, t);
    r.w[n] = 1.0 / t;
  }
  s->rates = r;
  return LBM_OK;
}

Sim* as_sim(lbm_handle h) { return reinterpret_cast<Sim*>(h); }

int check_handle(Sim* s) {
  if (!s) return set_error(LBM_EINVAL, "NULL handle");
  return LBM_OK;
}

int sync_and_status(Sim* s, int rc) {
  if (rc) return rc;
  int st = 0;
  int e = cuda_check(cudaMemcpyAsync(&st, status_word(s), sizeof(int), cudaMemcpyDeviceToHost, s->stream),
                     "status readback");
  if (e) return e;
  e = cuda_check(cudaStreamSynchronize(s->stream), "stream synchronize");
  if (e) return e;
  if (st & 2) return set_error(LBM_ETIMEOUT, "a bounded device wait for tensor-core completion gave up");
  if (st) return set_error(LBM_EDIVERGED, "a node diverged (rho <= 0, |u| >= 1 or non-finite)");
  return LBM_OK;
}

bool is_h37(const Sim* s) { return s->lattice == LBM_D2Q37; }
bool is_hgen(const Sim* s) { return s->lattice == LBM_HERMITE; }
// the Hermite lattices carry a temperature field (37-velocity and caller-supplied)
bool hermite_family(const Sim* s) { return is_h37(s) || is_hgen(s); }

cudaError_t launch_init(Sim* s, const void* rho, const void* u, const void* th, int dtype, int64_t n0,
                        int64_t cnt, int64_t ld) {
  if (is_hgen(s)) return hgen_launch_init(s, rho, u, th, dtype, n0, cnt, ld);
  return is_h37(s) ? h37_launch_init(s, rho, u, th, dtype, n0, cnt, ld)
                   : tp_launch_init(s, rho, u, dtype, n0, cnt, ld);
}
cudaError_t launch_moments(Sim* s, void* rho, void* u, void* th, int dtype, int64_t n0, int64_t cnt,
                           int64_t ld) {
  if (is_hgen(s)) return hgen_launch_moments(s, rho, u, th, dtype, n0, cnt, ld);
  return is_h37(s) ? h37_launch_moments(s, rho, u, th, dtype, n0, cnt, ld)
                   : tp_launch_moments(s, rho, u, dtype, n0, cnt, ld);
}
cudaError_t launch_get_pops(Sim* s, double* f, int64_t n0, int64_t cnt, int64_t ld) {
  if (is_hgen(s)) return hgen_launch_get_pops(s, f, n0, cnt, ld);
  return is_h37(s) ? h37_launch_get_pops(s, f, n0, cnt, ld) : tp_launch_get_pops(s, f, n0, cnt, ld);
}
cudaError_t launch_set_pops(Sim* s, const double* f, int64_t n0, int64_t cnt, int64_t ld) {
  if (is_hgen(s)) return hgen_launch_set_pops(s, f, n0, cnt, ld);
  return is_h37(s) ? h37_launch_set_pops(s, f, n0, cnt, ld) : tp_launch_set_pops(s, f, n0, cnt, ld);
}
cudaError_t launch_mode_into(Sim* s, int field, const int64_t mode[3], double* out2) {
  if (is_hgen(s)) return hgen_launch_mode_into(s, field, mode, out2);
  return is_h37(s) ? h37_launch_mode_into(s, field, mode, out2) : tp_launch_mode_into(s, field, mode, out2);
}
int max_field(const Sim* s) { return hermite_family(s) ? 4 : s->D; }
// fields whose amplitude is accumulated from (q - 1): rho, and theta, p on the Hermite lattices
bool offset_field(const Sim* s, int field) { return field == 0 || (hermite_family(s) && field >= 3); }
// fill a host theta array with ones (temperature of models without one)
void fill_ones(void* th, int dtype, int64_t n) {
  if (dtype == LBM_DTYPE_F64)
    for (int64_t k = 0; k < n; ++k) static_cast<double*>(th)[k] = 1.0;
  else
    for (int64_t k = 0; k < n; ++k) static_cast<float*>(th)[k] = 1.0f;
}

}  // namespace

// The device address of page-locked host memory (cudaHostAlloc, a registered
// range, a pinned tensor), or nullptr for any other pointer.  Kernels read and
// write such memory directly (over NVLink-C2C on this system), so host fields
// need no staging copies.  Pageable memory keeps the staged path.  (Also used
// by the batch calls.)
void* pinned_device_view(const void* p) {
  if (!p) return nullptr;
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();  // clear the (non-sticky) error the query left
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

namespace {


// Failure-detection self-test: one warp waits, with the bounded mbarrier wait
// of the tensor-core sweeps (tc05::mbar_wait), on a barrier that nothing
// arrives at.  Nothing asynchronous (no MMA, no bulk copy) is in flight and no
// tensor memory is held, so giving up is the whole of the failure path: the
// wait returns false after `polls` polls and lane 0 sets the timeout bit of the
// status word, as a sweep does when a tensor-core completion never comes.
__global__ void selftest_wait_kernel(int polls, int* __restrict__ status) {
  __shared__ uint64_t mbar;
  if (threadIdx.x == 0) {
    tc05::mbar_init(&mbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  const bool done = tc05::mbar_wait(&mbar, 0u, polls);
  if (!done && threadIdx.x == 0) atomicOr(status, 2);
}

}  // namespace

cudaError_t launch_sweep(Sim* s) {
  const int odd = (int)(s->step & 1);
  if (is_hgen(s)) return hgen_launch_sweep(s, odd);
  if (is_h37(s)) return h37_launch_sweep(s, odd);
  if (s->closure) return closure_sweep(s, odd, closure_image(s), closure_norm(s));
  return tp_pair_supported(s) ? tp_launch_pair_sweep(s, odd) : tp_launch_sweep(s, odd);
}

cudaError_t launch_reduce_into(Sim* s, double* partials, int nblocks, double* result) {
  if (is_hgen(s)) return hgen_launch_reduce_into(s, partials, nblocks, result);
  return is_h37(s) ? h37_launch_reduce_into(s, partials, nblocks, result)
                   : tp_launch_reduce_into(s, partials, nblocks, result);
}

}  // namespace lbm

using namespace lbm;

extern "C" {

const char* lbm_last_error(void) { return g_err; }

int lbm_query_bytes(int lattice, const int64_t dims[3], int storage, size_t* pop_bytes,
                    size_t* work_bytes) {
  Shape sh;
  int rc = check_shape(lattice, dims, storage, &sh);
  if (rc) return rc;
  if (!pop_bytes || !work_bytes) return set_error(LBM_EINVAL, "NULL output pointer");
  *pop_bytes = round256((size_t)sh.Q * (size_t)sh.N * storage_elem_bytes(storage));
  *work_bytes = kWsStaging + staging_bytes_for(sh);
  return LBM_OK;
}

int lbm_create(int lattice, const int64_t dims[3], const double* tau_per_order, int n_tau,
               int storage, void* pop, size_t pop_bytes, void* work, size_t work_bytes,
               lbm_handle* out) {
  return lbm_create_ex(lattice, dims, tau_per_order, n_tau, storage, 0u, 1.0, pop, pop_bytes, work,
                       work_bytes, out);
}

int lbm_create_ex(int lattice, const int64_t dims[3], const double* tau_per_order, int n_tau,
                  int storage, unsigned flags, double theta_ref, void* pop, size_t pop_bytes,
                  void* work, size_t work_bytes, lbm_handle* out) {
  if (!out) return set_error(LBM_EINVAL, "NULL output handle pointer");
  *out = nullptr;
  Shape sh;
  int rc = check_shape(lattice, dims, storage, &sh);
  if (rc) return rc;
  if (flags & ~(LBM_THERMAL | LBM_K72 | LBM_RAW_MRT | LBM_STOCHASTIC_ROUND | LBM_FAST_TRANSFORMS))
    return set_error(LBM_EINVAL, "unknown flags 0x%x", flags);
  if (flags && lattice != LBM_D2Q37)
    return set_error(LBM_EINVAL, "model flags apply to the 37-velocity lattice only");
  if (!(theta_ref > 0.0) || !std::isfinite(theta_ref) || (lattice != LBM_D2Q37 && theta_ref != 1.0))
    return set_error(LBM_EINVAL, "theta_ref must be > 0 (and 1 on D2Q9 / D3Q27)");
  size_t need_pop = 0, need_work = 0;
  lbm_query_bytes(lattice, dims, storage, &need_pop, &need_work);
  if (!pop || !work) return set_error(LBM_EINVAL, "NULL population or workspace buffer");
  if (pop_bytes < need_pop || work_bytes < need_work)
    return set_error(LBM_ESIZE, "buffers too small: need %zu + %zu bytes, got %zu + %zu", need_pop,
                     need_work, pop_bytes, work_bytes);
  if (((uintptr_t)pop & 255) || ((uintptr_t)work & 255))
    return set_error(LBM_EINVAL, "population and workspace buffers must be 256-byte aligned");
  Sim* s = new (std::nothrow) Sim();
  if (!s) return set_error(LBM_EOOM, "host allocation of the handle failed");
  s->lattice = lattice;
  s->D = sh.D;
  s->Q = sh.Q;
  s->storage = storage;
  s->flags = flags;
  s->theta_ref = theta_ref;
  s->nx = sh.nx;
  s->ny = sh.ny;
  s->nz = sh.nz;
  s->N = sh.N;
  s->pop = pop;
  s->pop_bytes = pop_bytes;
  s->work = static_cast<unsigned char*>(work);
  s->work_bytes = work_bytes;
  s->staging_bytes = staging_bytes_for(sh);
  s->stream = nullptr;
  s->step = 0;
  s->closure = 0;
  rc = set_rates(s, tau_per_order, n_tau);
  if (!rc) rc = cuda_check(cudaMemsetAsync(status_word(s), 0, 512, s->stream), "clear status and results");
  if (!rc) rc = cuda_check(cudaStreamSynchronize(s->stream), "stream synchronize");
  if (rc) {
    delete s;
    return rc;
  }
  *out = reinterpret_cast<lbm_handle>(s);
  return LBM_OK;
}

int lbm_hermite_query_bytes(int q, const int64_t dims[3], int storage, size_t* pop_bytes, size_t* work_bytes) {
  if (q < 1 || q > kHQMax) return set_error(LBM_EINVAL, "q must be 1..%d", kHQMax);
  Shape sh;
  int rc = check_shape(LBM_D2Q37, dims, storage, &sh);  // the same 2D constraints (nx, ny >= 3)
  if (rc) return rc;
  if (!pop_bytes || !work_bytes) return set_error(LBM_EINVAL, "NULL output pointer");
  sh.Q = q;
  *pop_bytes = round256((size_t)sh.Q * (size_t)sh.N * storage_elem_bytes(storage));
  *work_bytes = kWsStaging + staging_bytes_for(sh);
  return LBM_OK;
}

int lbm_create_hermite(int q, const int* e, const double* w, double c, int order, const int64_t dims[3],
                       const double* tau_per_order, int n_tau, int storage, unsigned flags, double theta_ref,
                       void* pop, size_t pop_bytes, void* work, size_t work_bytes, lbm_handle* out) {
  if (!out) return set_error(LBM_EINVAL, "NULL output handle pointer");
  *out = nullptr;
  if (!e || !w) return set_error(LBM_EINVAL, "NULL lattice arrays");
  if (!((q == 17 && order == 3) || (q == 37 && (order == 3 || order == 4))))
    return set_error(LBM_EINVAL, "supported: 17 velocities with order 3, 37 velocities with order 3 or 4");
  if (!(c > 0.0) || !std::isfinite(c)) return set_error(LBM_EINVAL, "the scale c must be finite and > 0");
  if (storage != LBM_F64 && storage != LBM_F32) return set_error(LBM_EINVAL, "storage must be FP64 or FP32");
  if (flags & ~(LBM_THERMAL | LBM_FAST_TRANSFORMS))
    return set_error(LBM_EINVAL, "only LBM_THERMAL and LBM_FAST_TRANSFORMS apply to a caller-supplied lattice");
  if (!(theta_ref > 0.0) || !std::isfinite(theta_ref)) return set_error(LBM_EINVAL, "theta_ref must be > 0");
  HLattice L;
  L.q = q;
  L.order = order;
  L.c = c;
  for (int i = 0; i < q; ++i) {
    L.ex[i] = e[2 * i];
    L.ey[i] = e[2 * i + 1];
    L.w[i] = w[i];
    if (std::abs(L.ex[i]) > 3 || std::abs(L.ey[i]) > 3) return set_error(LBM_EINVAL, "velocity %d beyond |e| <= 3", i);
    if (!(w[i] > 0.0) || !std::isfinite(w[i])) return set_error(LBM_EINVAL, "weight %d must be > 0", i);
  }
  for (int i = 0; i < q; ++i) {
    L.opp[i] = -1;
    for (int j = 0; j < q; ++j) {
      if (j != i && L.ex[j] == L.ex[i] && L.ey[j] == L.ey[i])
        return set_error(LBM_EINVAL, "velocities %d and %d coincide", i, j);
      if (L.ex[j] == -L.ex[i] && L.ey[j] == -L.ey[i]) L.opp[i] = j;
    }
    if (L.opp[i] < 0) return set_error(LBM_EINVAL, "velocity %d has no opposite", i);
  }
  // the projection to order N needs exact Gaussian moments to degree 2N
  for (int d = 0; d <= 2 * order; ++d)
    for (int p = 0; p <= d; ++p) {
      const int qq = d - p;
      double sum = 0.0;
      for (int i = 0; i < q; ++i) sum += w[i] * std::pow(c * L.ex[i], p) * std::pow(c * L.ey[i], qq);
      auto gm = [](int a) {
        double r = (a % 2) ? 0.0 : 1.0;
        for (int k = a - 1; k > 0 && !(a % 2); k -= 2) r *= k;
        return r;
      };
      const double want = gm(p) * gm(qq);
      if (std::abs(sum - want) > 1e-10 * (1.0 + std::abs(want)))
        return set_error(LBM_EINVAL, "the rule is not exact to degree 2N = %d (moment x^%d y^%d)", 2 * order, p, qq);
    }
  size_t need_pop = 0, need_work = 0;
  int rc = lbm_hermite_query_bytes(q, dims, storage, &need_pop, &need_work);
  if (rc) return rc;
  if (!pop || !work) return set_error(LBM_EINVAL, "NULL population or workspace buffer");
  if (pop_bytes < need_pop || work_bytes < need_work)
    return set_error(LBM_ESIZE, "buffers too small: need %zu + %zu bytes, got %zu + %zu", need_pop, need_work,
                     pop_bytes, work_bytes);
  if (((uintptr_t)pop & 255) || ((uintptr_t)work & 255))
    return set_error(LBM_EINVAL, "population and workspace buffers must be 256-byte aligned");
  std::shared_ptr<HTables> tables;
  try {
    tables = std::make_shared<HTables>();
  } catch (const std::bad_alloc&) {
    return set_error(LBM_EOOM, "host allocation of the projection tables failed");
  }
  hgen_build_tables(L, theta_ref, tables.get());
  Sim* s = new (std::nothrow) Sim();
  if (!s) return set_error(LBM_EOOM, "host allocation of the handle failed");
  s->lattice = LBM_HERMITE;
  s->D = 2;
  s->Q = q;
  s->storage = storage;
  s->flags = flags;
  s->theta_ref = theta_ref;
  s->nx = dims[0];
  s->ny = dims[1];
  s->nz = 1;
  s->N = dims[0] * dims[1];
  s->pop = pop;
  s->pop_bytes = pop_bytes;
  s->work = static_cast<unsigned char*>(work);
  s->work_bytes = work_bytes;
  Shape sh{2, q, s->nx, s->ny, 1, s->N};
  s->staging_bytes = staging_bytes_for(sh);
  s->stream = nullptr;
  s->step = 0;
  s->closure = 0;
  s->hl = L;
  s->ht = tables;
  rc = set_rates(s, tau_per_order, n_tau);
  if (!rc) rc = cuda_check(cudaMemsetAsync(status_word(s), 0, 512, s->stream), "clear status and results");
  if (!rc) rc = cuda_check(cudaStreamSynchronize(s->stream), "stream synchronize");
  if (rc) {
    delete s;
    return rc;
  }
  *out = reinterpret_cast<lbm_handle>(s);
  return LBM_OK;
}

void lbm_destroy(lbm_handle h) { delete as_sim(h); }

int lbm_set_stream(lbm_handle h, void* stream) {
  Sim* s = as_sim(h);
  if (int rc = check_handle(s)) return rc;
  s->stream = static_cast<cudaStream_t>(stream);
  return LBM_OK;
}

int lbm_set_tau(lbm_handle h, const double* tau_per_order, int n_tau) {
  Sim* s = as_sim(h);
  if (int rc = check_handle(s)) return rc;
  return set_rates(s, tau_per_order, n_tau);
}

int lbm_init_fields(lbm_handle h, const void* rho, const void* u, const void* theta, int dtype,
                    int on_device) {
  Sim* s = as_sim(h);
  if (int rc = check_handle(s)) return rc;
  if (!rho || !u) return set_error(LBM_EINVAL, "NULL field pointer");
  if (dtype != LBM_DTYPE_F64 && dtype != LBM_DTYPE_F32)
    return set_error(LBM_EINVAL, "unknown field dtype %d", dtype);
  const size_t esz = dtype == LBM_DTYPE_F64 ? 8 : 4;
  const void* th = hermite_family(s) ? theta : nullptr;
  int rc = cuda_check(cudaMemsetAsync(status_word(s), 0, sizeof(int), s->stream), "clear status");
  if (rc) return rc;
  // page-locked host fields: the init kernel reads them where they are
  const void* drho = on_device ? nullptr : pinned_device_view(rho);
  const void* du = on_device ? nullptr : pinned_device_view(u);
  const void* dth = (on_device || !th) ? nullptr : pinned_device_view(th);
  if (on_device) {
    rc = cuda_check(launch_init(s, rho, u, th, dtype, 0, s->N, s->N), "init kernel");
  } else if (drho && du && (!th || dth)) {
    rc = cuda_check(launch_init(s, drho, du, dth, dtype, 0, s->N, s->N), "init kernel (page-locked host fields)");
    if (!rc) rc = cuda_check(cudaStreamSynchronize(s->stream), "stream synchronize");
  } else {
    const int nf = 1 + s->D + (th ? 1 : 0);
    const int64_t chunk = (int64_t)(s->staging_bytes / ((size_t)nf * esz));
    unsigned char* st = staging_buf(s);
    for (int64_t n0 = 0; n0 < s->N && !rc; n0 += chunk) {
      const int64_t cnt = s->N - n0 < chunk ? s->N - n0 : chunk;
      rc = cuda_check(cudaMemcpyAsync(st, static_cast<const unsigned char*>(rho) + n0 * esz, cnt * esz,
                                      cudaMemcpyHostToDevice, s->stream),
                      "copy rho to device");
      for (int d = 0; d < s->D && !rc; ++d)
        rc = cuda_check(cudaMemcpyAsync(st + (size_t)(1 + d) * cnt * esz,
                                        static_cast<const unsigned char*>(u) + ((size_t)d * s->N + n0) * esz,
                                        cnt * esz, cudaMemcpyHostToDevice, s->stream),
                        "copy u to device");
      unsigned char* st_th = st + (size_t)(1 + s->D) * cnt * esz;
      if (th && !rc)
        rc = cuda_check(cudaMemcpyAsync(st_th, static_cast<const unsigned char*>(th) + n0 * esz, cnt * esz,
                                        cudaMemcpyHostToDevice, s->stream),
                        "copy theta to device");
      if (!rc)
        rc = cuda_check(launch_init(s, st, st + cnt * esz, th ? st_th : nullptr, dtype, n0, cnt, cnt),
                        "init kernel");
    }
    if (!rc) rc = cuda_check(cudaStreamSynchronize(s->stream), "stream synchronize");
  }
  if (!rc) s->step = 0;
  return rc;
}

int lbm_step(lbm_handle h, int64_t n) {
  Sim* s = as_sim(h);
  if (int rc = check_handle(s)) return rc;
  if (n < 0) return set_error(LBM_EINVAL, "negative step count");
  for (int64_t k = 0; k < n; ++k) {
    cudaError_t e = launch_sweep(s);
    if (e != cudaSuccess) return cuda_check(e, "sweep kernel");
    ++s->step;
  }
  return LBM_OK;
}

int lbm_moments(lbm_handle h, void* rho, void* u, void* theta, int dtype, int on_device) {
  Sim* s = as_sim(h);
  if (int rc = check_handle(s)) return rc;
  if (!rho || !u) return set_error(LBM_EINVAL, "NULL field pointer");
  if (dtype != LBM_DTYPE_F64 && dtype != LBM_DTYPE_F32)
    return set_error(LBM_EINVAL, "unknown field dtype %d", dtype);
  const size_t esz = dtype == LBM_DTYPE_F64 ? 8 : 4;
  void* th = hermite_family(s) ? theta : nullptr;
  int rc = LBM_OK;
  void* drho = on_device ? nullptr : pinned_device_view(rho);
  void* du = on_device ? nullptr : pinned_device_view(u);
  void* dth = (on_device || !th) ? nullptr : pinned_device_view(th);
  if (on_device) {
    rc = cuda_check(launch_moments(s, rho, u, th, dtype, 0, s->N, s->N), "moments kernel");
    if (!rc && theta && !th)  // models without a temperature report theta = 1
      rc = cuda_check(launch_fill(theta, dtype, s->N, 1.0, s->stream), "theta fill");
  } else if (drho && du && (!th || dth)) {
    // page-locked host fields: the moments kernel writes them where they are
    rc = cuda_check(launch_moments(s, drho, du, dth, dtype, 0, s->N, s->N), "moments kernel (page-locked host)");
    if (theta && !th) fill_ones(theta, dtype, s->N);
  } else {
    const int nf = 1 + s->D + (th ? 1 : 0);
    const int64_t chunk = (int64_t)(s->staging_bytes / ((size_t)nf * esz));
    unsigned char* st = staging_buf(s);
    for (int64_t n0 = 0; n0 < s->N && !rc; n0 += chunk) {
      const int64_t cnt = s->N - n0 < chunk ? s->N - n0 : chunk;
      unsigned char* st_th = st + (size_t)(1 + s->D) * cnt * esz;
      rc = cuda_check(launch_moments(s, st, st + cnt * esz, th ? st_th : nullptr, dtype, n0, cnt, cnt),
                      "moments kernel");
      if (!rc)
        rc = cuda_check(cudaMemcpyAsync(static_cast<unsigned char*>(rho) + n0 * esz, st, cnt * esz,
                                        cudaMemcpyDeviceToHost, s->stream),
                        "copy rho to host");
      for (int d = 0; d < s->D && !rc; ++d)
        rc = cuda_check(cudaMemcpyAsync(static_cast<unsigned char*>(u) + ((size_t)d * s->N + n0) * esz,
                                        st + (size_t)(1 + d) * cnt * esz, cnt * esz,
                                        cudaMemcpyDeviceToHost, s->stream),
                        "copy u to host");
      if (th && !rc)
        rc = cuda_check(cudaMemcpyAsync(static_cast<unsigned char*>(th) + n0 * esz, st_th, cnt * esz,
                                        cudaMemcpyDeviceToHost, s->stream),
                        "copy theta to host");
    }
    if (theta && !th) fill_ones(theta, dtype, s->N);
  }
  return sync_and_status(s, rc);
}

int lbm_get_populations(lbm_handle h, double* f, int on_device) {
  Sim* s = as_sim(h);
  if (int rc = check_handle(s)) return rc;
  if (!f) return set_error(LBM_EINVAL, "NULL population pointer");
  int rc = LBM_OK;
  if (on_device) {
    rc = cuda_check(launch_get_pops(s, f, 0, s->N, s->N), "population gather kernel");
  } else {
    const int64_t chunk = (int64_t)(s->staging_bytes / ((size_t)s->Q * sizeof(double)));
    double* st = reinterpret_cast<double*>(staging_buf(s));
    for (int64_t n0 = 0; n0 < s->N && !rc; n0 += chunk) {
      const int64_t cnt = s->N - n0 < chunk ? s->N - n0 : chunk;
      rc = cuda_check(launch_get_pops(s, st, n0, cnt, cnt), "population gather kernel");
      for (int i = 0; i < s->Q && !rc; ++i)
        rc = cuda_check(cudaMemcpyAsync(f + (size_t)i * s->N + n0, st + (size_t)i * cnt,
                                        cnt * sizeof(double), cudaMemcpyDeviceToHost, s->stream),
                        "copy populations to host");
    }
  }
  if (!rc) rc = cuda_check(cudaStreamSynchronize(s->stream), "stream synchronize");
  return rc;
}

int lbm_set_populations(lbm_handle h, const double* f, int on_device) {
  Sim* s = as_sim(h);
  if (int rc = check_handle(s)) return rc;
  if (!f) return set_error(LBM_EINVAL, "NULL population pointer");
  int rc = LBM_OK;
  if (on_device) {
    rc = cuda_check(launch_set_pops(s, f, 0, s->N, s->N), "population scatter kernel");
  } else {
    const int64_t chunk = (int64_t)(s->staging_bytes / ((size_t)s->Q * sizeof(double)));
    double* st = reinterpret_cast<double*>(staging_buf(s));
    for (int64_t n0 = 0; n0 < s->N && !rc; n0 += chunk) {
      const int64_t cnt = s->N - n0 < chunk ? s->N - n0 : chunk;
      for (int i = 0; i < s->Q && !rc; ++i)
        rc = cuda_check(cudaMemcpyAsync(st + (size_t)i * cnt, f + (size_t)i * s->N + n0,
                                        cnt * sizeof(double), cudaMemcpyHostToDevice, s->stream),
                        "copy populations to device");
      if (!rc) rc = cuda_check(launch_set_pops(s, st, n0, cnt, cnt), "population scatter kernel");
    }
  }
  if (!rc) rc = cuda_check(cudaStreamSynchronize(s->stream), "stream synchronize");
  return rc;
}

int lbm_reduce(lbm_handle h, double out[5]) {
  Sim* s = as_sim(h);
  if (int rc = check_handle(s)) return rc;
  if (!out) return set_error(LBM_EINVAL, "NULL output pointer");
  int rc = cuda_check(launch_reduce_into(s, partials_buf(s), kRedBlocks, result_buf(s)), "reduction kernels");
  double tmp[5] = {0, 0, 0, 0, 0};
  if (!rc)
    rc = cuda_check(cudaMemcpyAsync(tmp, result_buf(s), sizeof(tmp), cudaMemcpyDeviceToHost, s->stream),
                    "copy totals to host");
  if (!rc) rc = cuda_check(cudaStreamSynchronize(s->stream), "stream synchronize");
  if (!rc) memcpy(out, tmp, sizeof(tmp));
  return rc;
}

// Enqueue one step whose totals of the consumed state end up in out[0..5)
// (device-accessible memory: result_buf, or a caller's page-locked host buffer).
static int enqueue_step_totals(Sim* s, double* out) {
  const size_t staging = s->staging_bytes;
  const bool fused_tp = !is_hgen(s) && !is_h37(s) && !s->closure && tp_pair_supported(s) &&
                        (size_t)tp_pair_warps(s) * 8 * sizeof(float) <= staging;
  const bool fused_h37 =
      is_h37(s) && h37_pair_supported(s) && (size_t)h37_pair_warps(s) * 8 * sizeof(float) <= staging;
  int rc = LBM_OK;
  if (fused_tp || fused_h37) {
    // one sweep: the pair kernel writes per-warp partials of the consumed state's totals
    float* warps = reinterpret_cast<float*>(staging_buf(s));
    const int odd = (int)(s->step & 1);
    rc = cuda_check(fused_tp ? tp_launch_pair_sweep_totals(s, odd, warps) : h37_launch_pair_sweep_totals(s, odd, warps),
                    "sweep kernel with totals");
    const int64_t n = fused_tp ? tp_pair_warps(s) : h37_pair_warps(s);
    if (!rc)
      rc = cuda_check(launch_sum_partials(warps, n, partials_buf(s), ticket_buf(s), out, s->stream),
                      "totals kernel");
    if (!rc) ++s->step;
  } else {
    // the same quantities from the reduction of the state before the sweep
    rc = cuda_check(launch_reduce_into(s, partials_buf(s), kRedBlocks, out), "reduction kernels");
    if (!rc) rc = cuda_check(launch_sweep(s), "sweep kernel");
    if (!rc) ++s->step;
  }
  return rc;
}

int lbm_step_totals(lbm_handle h, double out[5]) {
  Sim* s = as_sim(h);
  if (int rc = check_handle(s)) return rc;
  if (!out) return set_error(LBM_EINVAL, "NULL output pointer");
  int rc = enqueue_step_totals(s, result_buf(s));
  double tmp[5] = {0, 0, 0, 0, 0};
  if (!rc)
    rc = cuda_check(cudaMemcpyAsync(tmp, result_buf(s), sizeof(tmp), cudaMemcpyDeviceToHost, s->stream),
                    "copy totals to host");
  if (!rc) rc = cuda_check(cudaStreamSynchronize(s->stream), "stream synchronize");
  if (!rc) memcpy(out, tmp, sizeof(tmp));
  return rc;
}

int lbm_step_totals_async(lbm_handle h, double* out) {
  Sim* s = as_sim(h);
  if (int rc = check_handle(s)) return rc;
  if (!out) return set_error(LBM_EINVAL, "NULL output pointer");
  // page-locked and 8-byte aligned: the summing kernel writes the totals there
  // itself (no copy after the step); any other buffer gets a copy on the stream
  double* direct = ((uintptr_t)out & 7u) ? nullptr : static_cast<double*>(pinned_device_view(out));
  int rc = enqueue_step_totals(s, direct ? direct : result_buf(s));
  if (!rc && !direct)
    rc = cuda_check(cudaMemcpyAsync(out, result_buf(s), 5 * sizeof(double), cudaMemcpyDeviceToHost, s->stream),
                    "copy totals to host");
  return rc;
}

int lbm_mode_amplitude(lbm_handle h, int field, const int64_t mode[3], double out[2]) {
  Sim* s = as_sim(h);
  if (int rc = check_handle(s)) return rc;
  if (!out || !mode) return set_error(LBM_EINVAL, "NULL pointer");
  if (field < 0 || field > max_field(s))
    return set_error(LBM_EINVAL, "field must be 0 (rho), 1..D (u_d) or, on D2Q37, 3 (theta) / 4 (p)");
  int rc = cuda_check(launch_mode_into(s, field, mode, result_buf(s)), "mode amplitude kernels");
  double tmp[2] = {0, 0};
  if (!rc)
    rc = cuda_check(cudaMemcpyAsync(tmp, result_buf(s), sizeof(tmp), cudaMemcpyDeviceToHost, s->stream),
                    "copy amplitude to host");
  if (!rc) rc = cuda_check(cudaStreamSynchronize(s->stream), "stream synchronize");
  if (!rc) {
    // the density amplitude is accumulated from rho - 1; restore sum_x 1 * exp(0) at k = 0
    const bool k0 = (mode[0] % s->nx == 0) && (mode[1] % s->ny == 0) && (s->D == 2 || mode[2] % s->nz == 0);
    out[0] = tmp[0] + ((offset_field(s, field) && k0) ? (double)s->N : 0.0);
    out[1] = tmp[1];
  }
  return rc;
}

int lbm_mode_history(lbm_handle h, int field, const int64_t mode[3], int n_records, int64_t stride,
                     double* amplitudes, double fit[4]) {
  Sim* s = as_sim(h);
  if (int rc = check_handle(s)) return rc;
  if (!mode || !fit) return set_error(LBM_EINVAL, "NULL pointer");
  if (field < 0 || field > max_field(s))
    return set_error(LBM_EINVAL, "field must be 0 (rho), 1..D (u_d) or, on D2Q37, 3 (theta) / 4 (p)");
  if (n_records < 2 || n_records > kMaxHistory)
    return set_error(LBM_EINVAL, "n_records must be in [2, %d]", kMaxHistory);
  if (stride < 1) return set_error(LBM_EINVAL, "stride must be >= 1");
  double* hist = history_buf(s);
  int rc = LBM_OK;
  for (int r = 0; r < n_records && !rc; ++r) {
    if (r > 0) {
      for (int64_t k = 0; k < stride && !rc; ++k) {
        rc = cuda_check(launch_sweep(s), "sweep kernel");
        if (!rc) ++s->step;
      }
    }
    if (!rc) rc = cuda_check(launch_mode_into(s, field, mode, hist + 2 * r), "mode amplitude kernels");
  }
  // the density amplitude is accumulated from rho - 1; restore sum_x 1 at k = 0
  const bool k0 = (mode[0] % s->nx == 0) && (mode[1] % s->ny == 0) && (s->D == 2 || mode[2] % s->nz == 0);
  const double re_offset = (offset_field(s, field) && k0) ? (double)s->N : 0.0;
  if (!rc)
    rc = cuda_check(launch_decay_fit(hist, n_records, (double)stride, re_offset, fit_buf(s), s->stream),
                    "decay fit kernel");
  double tmp[4] = {0, 0, 0, 0};
  if (!rc)
    rc = cuda_check(cudaMemcpyAsync(tmp, fit_buf(s), sizeof(tmp), cudaMemcpyDeviceToHost, s->stream),
                    "copy fit to host");
  if (!rc && amplitudes)
    rc = cuda_check(cudaMemcpyAsync(amplitudes, hist, sizeof(double) * 2 * (size_t)n_records,
                                    cudaMemcpyDeviceToHost, s->stream),
                    "copy amplitudes to host");
  rc = sync_and_status(s, rc);
  if (rc == LBM_OK || rc == LBM_EDIVERGED) {
    for (int k = 0; k < 4; ++k) fit[k] = tmp[k];
    if (amplitudes && re_offset != 0.0)
      for (int r = 0; r < n_records; ++r) amplitudes[2 * r] += re_offset;
  }
  return rc;
}

int64_t lbm_step_count(lbm_handle h) {
  Sim* s = as_sim(h);
  return s ? s->step : -1;
}

int lbm_set_active_planes(lbm_handle h, int64_t z_lo, int64_t z_count) {
  Sim* s = as_sim(h);
  if (int rc = check_handle(s)) return rc;
  if (s->lattice != LBM_D3Q27) return set_error(LBM_EINVAL, "active plane ranges are for D3Q27 grids");
  if (z_lo < 0 || z_count < 1 || z_lo + z_count > s->nz)
    return set_error(LBM_EINVAL, "planes %lld .. %lld are not inside the grid of %lld planes", (long long)z_lo,
                     (long long)(z_lo + z_count - 1), (long long)s->nz);
  if (s->closure && !(z_lo == 0 && z_count == s->nz))
    return set_error(LBM_EINVAL, "the learned closure sweeps the whole grid");
  s->z_lo = z_lo;
  s->z_cnt = z_count == s->nz ? 0 : z_count;
  return LBM_OK;
}

const char* lbm_sweep_kernel(lbm_handle h) {
  Sim* s = as_sim(h);
  if (check_handle(s)) return nullptr;
  if (is_hgen(s)) return "hgen_sweep_kernel";
  if (is_h37(s)) return h37_pair_supported(s) ? "h37_pair_kernel" : "h37_sweep_kernel";
  if (s->closure) return closure_uses_tcgen05() ? "learned_tc_kernel" : "learned_sweep_kernel";
  return tp_pair_supported(s) ? tp_pair_kernel_name(s) : "tp_sweep_kernel";
}

int lbm_selftest_wait_timeout(lbm_handle h, int polls) {
  Sim* s = as_sim(h);
  if (int rc = check_handle(s)) return rc;
  if (polls < 1 || polls > (1 << 20)) return set_error(LBM_EINVAL, "polls must be in 1 .. 2^20");
  selftest_wait_kernel<<<1, 32, 0, s->stream>>>(polls, status_word(s));
  return cuda_check(cudaGetLastError(), "self-test wait kernel");
}

int lbm_status(lbm_handle h) {
  Sim* s = as_sim(h);
  if (int rc = check_handle(s)) return rc;
  return sync_and_status(s, LBM_OK);
}

static int check_range(double lo, double hi) {
  if (!(lo >= 0.0 && hi <= 2.0 && lo < hi)) return set_error(LBM_EINVAL, "need 0 <= omega_lo < omega_hi <= 2");
  return LBM_OK;
}

int lbm_set_closure(lbm_handle h, const float* params, const float* norm, double omega_lo, double omega_hi) {
  Sim* s = as_sim(h);
  if (int rc = check_handle(s)) return rc;
  if (!params) {
    s->closure = 0;
    return LBM_OK;
  }
  if (s->lattice != LBM_D3Q27 || s->storage != LBM_F32)
    return set_error(LBM_EINVAL, "the learned closure runs on D3Q27 with FP32 storage");
  if (s->z_cnt > 0) return set_error(LBM_EINVAL, "the learned closure sweeps the whole grid (active planes are set)");
  if (!norm) return set_error(LBM_EINVAL, "NULL feature standardisation");
  if (int rc = check_range(omega_lo, omega_hi)) return rc;
  const float range[2] = {(float)omega_lo, (float)omega_hi};
  int rc = cuda_check(cudaMemcpyAsync(closure_params(s), params, 5894 * sizeof(float), cudaMemcpyDeviceToDevice,
                                      s->stream),
                      "copy network parameters");
  if (!rc)
    rc = cuda_check(cudaMemcpyAsync(closure_norm(s), norm, 40 * sizeof(float), cudaMemcpyDeviceToDevice, s->stream),
                    "copy standardisation");
  if (!rc)
    rc = cuda_check(cudaMemcpyAsync(closure_norm(s) + 40, range, sizeof(range), cudaMemcpyHostToDevice, s->stream),
                    "copy rate range");
  if (!rc && closure_image_bytes() > kClosureImageFloats * sizeof(float))
    rc = set_error(LBM_EINVAL, "weight image larger than its workspace slot");
  if (!rc) rc = cuda_check(closure_build_image(closure_params(s), closure_image(s), s->stream), "weight image kernel");
  if (!rc) rc = cuda_check(cudaStreamSynchronize(s->stream), "stream synchronize");
  if (!rc) s->closure = 1;
  return rc;
}

int lbm_closure_filter(lbm_handle h, int m, float* coarse) {
  Sim* s = as_sim(h);
  if (int rc = check_handle(s)) return rc;
  if (s->lattice != LBM_D3Q27) return set_error(LBM_EINVAL, "the box filter works on D3Q27");
  if (!coarse) return set_error(LBM_EINVAL, "NULL output");
  if (m < 1 || s->nx % m || s->ny % m || s->nz % m)
    return set_error(LBM_EINVAL, "the filter width must divide every dimension");
  return cuda_check(closure_filter(s, m, coarse), "box filter kernel");
}

int lbm_closure_rescale(const int64_t dims[3], float* f, double scale, void* stream) {
  if (!dims || !f) return set_error(LBM_EINVAL, "NULL pointer");
  if (dims[0] < 1 || dims[1] < 1 || dims[2] < 1 || (double)dims[0] * dims[1] * dims[2] >= 2147483648.0)
    return set_error(LBM_EINVAL, "bad dims");
  if (!std::isfinite(scale)) return set_error(LBM_EINVAL, "scale must be finite");
  return cuda_check(closure_rescale(dims[0] * dims[1] * dims[2], f, scale, static_cast<cudaStream_t>(stream)),
                    "rescale kernel");
}

int lbm_closure_dataset(const int64_t dims[3], const float* f_t, const float* f_t1, double tau2, const float* norm,
                        float* X, float* abc, void* stream) {
  if (!dims || !f_t || !f_t1 || !norm || !X || !abc) return set_error(LBM_EINVAL, "NULL pointer");
  if (dims[0] < 1 || dims[1] < 1 || dims[2] < 1 || (double)dims[0] * dims[1] * dims[2] >= 2147483648.0)
    return set_error(LBM_EINVAL, "bad dims");
  return cuda_check(closure_dataset(dims, f_t, f_t1, tau2, norm, X, abc, static_cast<cudaStream_t>(stream)),
                    "dataset kernel");
}

size_t lbm_mlp_work_bytes(int64_t batch) {
  if (batch < 1) return 0;
  return closure_partials_bytes(batch) + 5904 * sizeof(float) + 256;
}

static int mlp_common(const float* X, const float* abc, int64_t n, const float* cw, const float* params,
                      int64_t batch, size_t work_bytes, void* work) {
  if (!X || !abc || !cw || !params || !work) return set_error(LBM_EINVAL, "NULL pointer");
  if (n < 1 || batch < 1) return set_error(LBM_EINVAL, "need n >= 1 and batch >= 1");
  if (work_bytes < lbm_mlp_work_bytes(batch)) return set_error(LBM_ESIZE, "workspace too small");
  if ((uintptr_t)work & 255) return set_error(LBM_EINVAL, "workspace must be 256-byte aligned");
  return LBM_OK;
}

int lbm_mlp_loss_grad(const float* X, const float* abc, int64_t n, const float* cw, double omega_lo,
                      double omega_hi, const float* params, float* grad, double* loss, void* work, size_t work_bytes,
                      void* stream) {
  if (int rc = mlp_common(X, abc, n, cw, params, n, work_bytes, work)) return rc;
  if (int rc = check_range(omega_lo, omega_hi)) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  float* partials = static_cast<float*>(work);
  float* g = reinterpret_cast<float*>(static_cast<unsigned char*>(work) + closure_partials_bytes(n));
  float* l = g + 5895;
  int rc = cuda_check(closure_grad(X, abc, n, n, 0, 0, 0, cw, omega_lo, omega_hi, params, partials, g, l, st),
                      "gradient kernels");
  if (!rc && grad)
    rc = cuda_check(cudaMemcpyAsync(grad, g, 5894 * sizeof(float), cudaMemcpyDeviceToDevice, st), "copy gradient");
  float lh = 0.0f;
  if (!rc) rc = cuda_check(cudaMemcpyAsync(&lh, l, sizeof(float), cudaMemcpyDeviceToHost, st), "copy loss");
  if (!rc) rc = cuda_check(cudaStreamSynchronize(st), "stream synchronize");
  if (!rc && loss) *loss = lh;
  return rc;
}

int lbm_mlp_train(const float* X, const float* abc, int64_t n, const float* cw, double omega_lo, double omega_hi,
                  float* params, float* adam_m, float* adam_v, int64_t iters, int64_t batch, double lr,
                  uint64_t seed, int64_t t0, float* loss_hist, void* work, size_t work_bytes, void* stream) {
  if (int rc = mlp_common(X, abc, n, cw, params, batch, work_bytes, work)) return rc;
  if (int rc = check_range(omega_lo, omega_hi)) return rc;
  if (!adam_m || !adam_v || iters < 0 || t0 < 0 || !(lr > 0.0))
    return set_error(LBM_EINVAL, "bad optimiser arguments");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  float* partials = static_cast<float*>(work);
  float* g = reinterpret_cast<float*>(static_cast<unsigned char*>(work) + closure_partials_bytes(batch));
  for (int64_t it = 0; it < iters; ++it) {
    int rc = cuda_check(closure_grad(X, abc, n, batch, 1, seed, (uint64_t)(t0 + it), cw, omega_lo, omega_hi, params,
                                     partials, g, loss_hist ? loss_hist + it : nullptr, st),
                        "gradient kernels");
    if (!rc) rc = cuda_check(closure_adam(params, adam_m, adam_v, g, lr, t0 + it + 1, st), "adam kernel");
    if (rc) return rc;
  }
  return LBM_OK;
}

}  // extern "C"
