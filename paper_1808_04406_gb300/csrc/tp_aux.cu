// Per-node auxiliary kernels for D2Q9 / D3Q27: initialisation to equilibrium,
// macroscopic fields, FP64 population exchange, FP64 grid totals and the
// single-wavenumber Fourier amplitude.  All of them are parity-aware: they read
// or write the populations of the current time whatever the AA state.
#include <type_traits>

#include "reduce.cuh"
#include "tp_common.cuh"

namespace lbm {
namespace {

// Node index -> coordinates in 32-bit arithmetic (N < 2^31).
__device__ __forceinline__ void node_xyz(const tp::Grid& g, int64_t n, int& x, int& y, int& z) {
  const uint32_t nn = (uint32_t)n, nx = (uint32_t)g.nx, ny = (uint32_t)g.ny;
  const uint32_t r = nn / nx;
  x = (int)(nn - r * nx);
  z = (int)(r / ny);
  y = (int)(r - (uint32_t)z * ny);
}

// Per-node mass excess and momentum of the offsets, in the compute type (FP64
// arithmetic is reserved for sums across nodes: it is slow on this GPU).
template <typename T, int D>
__device__ __forceinline__ void node_moments(const T (&v)[tp::qof<D>()], T& drho, T (&j)[D]) {
  drho = 0;
#pragma unroll
  for (int d = 0; d < D; ++d) j[d] = 0;
#pragma unroll
  for (int i = 0; i < tp::qof<D>(); ++i) {
    drho += v[i];
#pragma unroll
    for (int d = 0; d < D; ++d) {
      if (tp::dig(i, d) == 2) j[d] += v[i];
      if (tp::dig(i, d) == 0) j[d] -= v[i];
    }
  }
}

// f := equilibrium of (rho, u) for nodes [n0, n0 + cnt); fields indexed i - n0
// with leading dimension ld for u.  Writes the even-state layout.
template <int D, int S, typename F>
__global__ void tp_init_kernel(typename tp::Store<S>::type* __restrict__ f, tp::Grid g,
                               const F* __restrict__ rho, const F* __restrict__ u, int64_t n0,
                               int64_t cnt, int64_t ld) {
  using T = typename tp::Store<S>::calc;
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= cnt) return;
  const int64_t n = n0 + k;
  int x, y, z;
  node_xyz(g, n, x, y, z);
  T uu[D];
#pragma unroll
  for (int d = 0; d < D; ++d) uu[d] = (T)u[d * ld + k];
  const T drho = (T)((double)rho[k] - 1.0);
  T v[tp::qof<D>()];
  tp::equilibrium<T, D>(v, drho, uu);
  tp::scatter<D, S>(f, g, x, y, z, 0, v);
}

template <int D, int S, typename F>
__global__ void tp_moments_kernel(const typename tp::Store<S>::type* __restrict__ f, tp::Grid g,
                                  int odd, F* __restrict__ rho, F* __restrict__ u, int64_t n0,
                                  int64_t cnt, int64_t ld) {
  using T = typename tp::Store<S>::calc;
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= cnt) return;
  int x, y, z;
  node_xyz(g, n0 + k, x, y, z);
  T v[tp::qof<D>()];
  tp::gather<D, S>(f, g, x, y, z, odd, v);
  // the moments in the wider of the compute and the output type, so that FP64
  // fields of FP32 (or 16-bit) storage carry no FP32 rounding of their own
  using M = typename std::conditional<(sizeof(F) > sizeof(T)), F, T>::type;
  M vm[tp::qof<D>()];
#pragma unroll
  for (int i = 0; i < tp::qof<D>(); ++i) vm[i] = (M)v[i];
  M drho, j[D];
  node_moments<M, D>(vm, drho, j);
  const M r = M(1) + drho;
  rho[k] = (F)r;
#pragma unroll
  for (int d = 0; d < D; ++d) u[d * ld + k] = (F)(j[d] / r);
}

template <int D, int S>
__global__ void tp_get_pops_kernel(const typename tp::Store<S>::type* __restrict__ f, tp::Grid g,
                                   int odd, double* __restrict__ out, int64_t n0, int64_t cnt,
                                   int64_t ld) {
  using T = typename tp::Store<S>::calc;
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= cnt) return;
  int x, y, z;
  node_xyz(g, n0 + k, x, y, z);
  T v[tp::qof<D>()];
  tp::gather<D, S>(f, g, x, y, z, odd, v);
#pragma unroll
  for (int i = 0; i < tp::qof<D>(); ++i) out[i * ld + k] = tp::wq<D>(i) + (double)v[i];
}

template <int D, int S>
__global__ void tp_set_pops_kernel(typename tp::Store<S>::type* __restrict__ f, tp::Grid g, int odd,
                                   const double* __restrict__ in, int64_t n0, int64_t cnt,
                                   int64_t ld) {
  using T = typename tp::Store<S>::calc;
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= cnt) return;
  int x, y, z;
  node_xyz(g, n0 + k, x, y, z);
  T v[tp::qof<D>()];
#pragma unroll
  for (int i = 0; i < tp::qof<D>(); ++i) v[i] = (T)(in[i * ld + k] - tp::wq<D>(i));
  tp::scatter<D, S>(f, g, x, y, z, odd, v);
}

// Grid totals, pass 1: block partials of {sum drho, sum rho u_d, sum rho|u|^2/2}.
// Blocks stride over x-rows, threads over x within a row.
template <int D, int S>
__global__ void __launch_bounds__(kAuxThreads)
    tp_reduce_kernel(const typename tp::Store<S>::type* __restrict__ f, tp::Grid g, int odd, int z0, int nzr,
                     double* __restrict__ partials) {
  using T = typename tp::Store<S>::calc;
  double acc[5] = {0, 0, 0, 0, 0};
  // the rows (y, z) of planes z0 .. z0 + nzr - 1
  const uint32_t rows = (uint32_t)g.ny * (uint32_t)nzr, row0 = (uint32_t)g.ny * (uint32_t)z0;
  for (uint32_t row = blockIdx.x; row < rows; row += gridDim.x)
  for (int x = threadIdx.x; x < g.nx; x += blockDim.x) {
    const int z = (int)((row0 + row) / (uint32_t)g.ny), y = (int)(row0 + row - (uint32_t)z * (uint32_t)g.ny);
    T v[tp::qof<D>()];
    tp::gather<D, S>(f, g, x, y, z, odd, v);
    T drho, j[D];
    node_moments<T, D>(v, drho, j);
    T jj = 0;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      acc[1 + d] += (double)j[d];
      jj += j[d] * j[d];
    }
    acc[0] += (double)drho;
    acc[4] += (double)(T(0.5) * jj / (T(1) + drho));
  }
  block_sum<5>(acc);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < 5; ++k) partials[(size_t)blockIdx.x * 8 + k] = acc[k];
  }
}

// Single-wavenumber amplitude, pass 1: block partials of sum q exp(-i k.x).
// The phase factor splits as exp(-i kx x) exp(-i (ky y + kz z)): the x factors
// come from a per-block shared table (grids up to kModeTable wide), the row
// factor is computed once per row.  Phases are reduced exactly in integers.
constexpr int kModeTable = 2048;

template <int D, int S>
__global__ void __launch_bounds__(kAuxThreads)
    tp_mode_kernel(const typename tp::Store<S>::type* __restrict__ f, tp::Grid g, int odd,
                   int field, long long mx, long long my, long long mz,
                   double* __restrict__ partials) {
  using T = typename tp::Store<S>::calc;
  __shared__ double2 xt[kModeTable];
  const bool table = g.nx <= kModeTable;
  const long long ax = ((mx % g.nx) + g.nx) % g.nx, ay = ((my % g.ny) + g.ny) % g.ny,
                  az = ((mz % g.nz) + g.nz) % g.nz;
  if (table) {
    for (int x = threadIdx.x; x < g.nx; x += blockDim.x) {
      double sn, cs;
      sincospi(2.0 * (double)((ax * x) % g.nx) / g.nx, &sn, &cs);
      xt[x] = make_double2(cs, -sn);
    }
  }
  __syncthreads();
  double acc[2] = {0, 0};
  const uint32_t rows = (uint32_t)g.ny * (uint32_t)g.nz;
  for (uint32_t row = blockIdx.x; row < rows; row += gridDim.x) {
    const int z = (int)(row / (uint32_t)g.ny), y = (int)(row - (uint32_t)z * (uint32_t)g.ny);
    const double fr = (double)((ay * y) % g.ny) / g.ny + (double)((az * z) % g.nz) / g.nz;
    double sr, cr;
    sincospi(2.0 * fr, &sr, &cr);  // row factor exp(-i 2 pi fr) = (cr, -sr)
    double ar = 0, ai = 0;         // sum over the row of q * exp(-i kx x)
    for (int x = threadIdx.x; x < g.nx; x += blockDim.x) {
      T v[tp::qof<D>()];
      tp::gather<D, S>(f, g, x, y, z, odd, v);
      T drho, j[D];
      node_moments<T, D>(v, drho, j);
      const T r = T(1) + drho;
      T q = drho;  // rho - 1: the constant 1 only adds N to the k = 0 amplitude (host side)
#pragma unroll
      for (int d = 0; d < D; ++d)
        if (field == 1 + d) q = j[d] / r;
      double2 c;
      if (table) {
        c = xt[x];
      } else {
        double sn, cs;
        sincospi(2.0 * (double)((ax * x) % g.nx) / g.nx, &sn, &cs);
        c = make_double2(cs, -sn);
      }
      ar += (double)q * c.x;
      ai += (double)q * c.y;
    }
    acc[0] += ar * cr + ai * sr;  // (ar + i ai)(cr - i sr)
    acc[1] += ai * cr - ar * sr;
  }
  block_sum<2>(acc);
  if (threadIdx.x == 0) {
    partials[(size_t)blockIdx.x * 8 + 0] = acc[0];
    partials[(size_t)blockIdx.x * 8 + 1] = acc[1];
  }
}

inline unsigned blocks_for(int64_t cnt) { return (unsigned)((cnt + kAuxThreads - 1) / kAuxThreads); }

inline tp::Grid grid_of(Sim* s) { return tp::Grid{(int)s->nx, (int)s->ny, (int)s->nz, s->N}; }

template <int D, int S>
cudaError_t init_t(Sim* s, const void* rho, const void* u, int dtype, int64_t n0, int64_t cnt,
                   int64_t ld) {
  using Tst = typename tp::Store<S>::type;
  if (cnt <= 0) return cudaSuccess;
  Tst* f = static_cast<Tst*>(s->pop);
  if (dtype == LBM_DTYPE_F64)
    tp_init_kernel<D, S, double><<<blocks_for(cnt), kAuxThreads, 0, s->stream>>>(
        f, grid_of(s), static_cast<const double*>(rho), static_cast<const double*>(u), n0, cnt, ld);
  else
    tp_init_kernel<D, S, float><<<blocks_for(cnt), kAuxThreads, 0, s->stream>>>(
        f, grid_of(s), static_cast<const float*>(rho), static_cast<const float*>(u), n0, cnt, ld);
  return cudaGetLastError();
}

template <int D, int S>
cudaError_t moments_t(Sim* s, void* rho, void* u, int dtype, int64_t n0, int64_t cnt, int64_t ld) {
  using Tst = typename tp::Store<S>::type;
  if (cnt <= 0) return cudaSuccess;
  const Tst* f = static_cast<const Tst*>(s->pop);
  const int odd = (int)(s->step & 1);
  if (dtype == LBM_DTYPE_F64)
    tp_moments_kernel<D, S, double><<<blocks_for(cnt), kAuxThreads, 0, s->stream>>>(
        f, grid_of(s), odd, static_cast<double*>(rho), static_cast<double*>(u), n0, cnt, ld);
  else
    tp_moments_kernel<D, S, float><<<blocks_for(cnt), kAuxThreads, 0, s->stream>>>(
        f, grid_of(s), odd, static_cast<float*>(rho), static_cast<float*>(u), n0, cnt, ld);
  return cudaGetLastError();
}

template <int D, int S>
cudaError_t get_pops_t(Sim* s, double* out, int64_t n0, int64_t cnt, int64_t ld) {
  using Tst = typename tp::Store<S>::type;
  if (cnt <= 0) return cudaSuccess;
  tp_get_pops_kernel<D, S><<<blocks_for(cnt), kAuxThreads, 0, s->stream>>>(
      static_cast<const Tst*>(s->pop), grid_of(s), (int)(s->step & 1), out, n0, cnt, ld);
  return cudaGetLastError();
}

template <int D, int S>
cudaError_t set_pops_t(Sim* s, const double* in, int64_t n0, int64_t cnt, int64_t ld) {
  using Tst = typename tp::Store<S>::type;
  if (cnt <= 0) return cudaSuccess;
  tp_set_pops_kernel<D, S><<<blocks_for(cnt), kAuxThreads, 0, s->stream>>>(
      static_cast<Tst*>(s->pop), grid_of(s), (int)(s->step & 1), in, n0, cnt, ld);
  return cudaGetLastError();
}

template <int D, int S>
cudaError_t mode_into_t(Sim* s, int field, const int64_t m[3], double* out2) {
  using Tst = typename tp::Store<S>::type;
  tp_mode_kernel<D, S><<<kRedBlocks, kAuxThreads, 0, s->stream>>>(
      static_cast<const Tst*>(s->pop), grid_of(s), (int)(s->step & 1), field, (long long)m[0],
      (long long)m[1], (long long)(D == 3 ? m[2] : 0), partials_buf(s));
  finalize_kernel<<<1, kAuxThreads, 0, s->stream>>>(partials_buf(s), kRedBlocks, 2, out2);
  return cudaGetLastError();
}

// dispatch over (D, storage)
#define LBM_TP_DISPATCH(FN, ...)                                 \
  do {                                                           \
    if (s->D == 2) {                                             \
      switch (s->storage) {                                      \
        case LBM_F64: return FN<2, LBM_F64>(s, __VA_ARGS__);     \
        case LBM_F32: return FN<2, LBM_F32>(s, __VA_ARGS__);     \
        case LBM_F16: return FN<2, LBM_F16>(s, __VA_ARGS__);     \
        case LBM_BF16: return FN<2, LBM_BF16>(s, __VA_ARGS__);   \
      }                                                          \
    } else {                                                     \
      switch (s->storage) {                                      \
        case LBM_F64: return FN<3, LBM_F64>(s, __VA_ARGS__);     \
        case LBM_F32: return FN<3, LBM_F32>(s, __VA_ARGS__);     \
        case LBM_F16: return FN<3, LBM_F16>(s, __VA_ARGS__);     \
        case LBM_BF16: return FN<3, LBM_BF16>(s, __VA_ARGS__);   \
      }                                                          \
    }                                                            \
    return cudaErrorInvalidValue;                                \
  } while (0)

// Same two kernels, with the block partials and the result in caller-chosen
// device memory (used by the allocation-free entry point).
template <int D, int S>
cudaError_t reduce_into_t(Sim* s, double* partials, int nblocks, double* result) {
  using Tst = typename tp::Store<S>::type;
  tp_reduce_kernel<D, S><<<nblocks, kAuxThreads, 0, s->stream>>>(
      static_cast<const Tst*>(s->pop), grid_of(s), (int)(s->step & 1), (int)active_z0(s), (int)active_nz(s),
      partials);
  finalize_kernel<<<1, kAuxThreads, 0, s->stream>>>(partials, nblocks, 5, result);
  return cudaGetLastError();
}

}  // namespace

cudaError_t tp_launch_init(Sim* s, const void* rho, const void* u, int dtype, int64_t n0,
                           int64_t cnt, int64_t ld) {
  LBM_TP_DISPATCH(init_t, rho, u, dtype, n0, cnt, ld);
}
cudaError_t tp_launch_moments(Sim* s, void* rho, void* u, int dtype, int64_t n0, int64_t cnt,
                              int64_t ld) {
  LBM_TP_DISPATCH(moments_t, rho, u, dtype, n0, cnt, ld);
}
cudaError_t tp_launch_get_pops(Sim* s, double* f, int64_t n0, int64_t cnt, int64_t ld) {
  LBM_TP_DISPATCH(get_pops_t, f, n0, cnt, ld);
}
cudaError_t tp_launch_set_pops(Sim* s, const double* f, int64_t n0, int64_t cnt, int64_t ld) {
  LBM_TP_DISPATCH(set_pops_t, f, n0, cnt, ld);
}

namespace {
// Sum of n FP32 partials (stride 8, five used) in FP64: block b adds its
// contiguous chunk (threads in a fixed stride, then the block in a fixed order)
// and writes scratch[b]; the last block to finish (ticket) adds the block sums
// in index order with one warp, writes out[0..5) and resets the ticket.
__global__ void __launch_bounds__(kAuxThreads)
    sum_partials_kernel(const float* __restrict__ partials, int64_t n, int64_t chunk, double* __restrict__ scratch,
                        unsigned* __restrict__ ticket, double* __restrict__ out) {
  double acc[5] = {0, 0, 0, 0, 0};
  const int64_t b0 = (int64_t)blockIdx.x * chunk, b1 = b0 + chunk < n ? b0 + chunk : n;
  for (int64_t b = b0 + threadIdx.x; b < b1; b += blockDim.x)
#pragma unroll
    for (int k = 0; k < 5; ++k) acc[k] += (double)partials[(size_t)b * 8 + k];
  block_sum<5>(acc);
  __shared__ bool last;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < 5; ++k) scratch[(size_t)blockIdx.x * 8 + k] = acc[k];
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x < 32) {
    __threadfence();
    double t[5] = {0, 0, 0, 0, 0};
    for (unsigned b = threadIdx.x; b < gridDim.x; b += 32)
#pragma unroll
      for (int k = 0; k < 5; ++k) t[k] += __ldcg(&scratch[(size_t)b * 8 + k]);
#pragma unroll
    for (int k = 0; k < 5; ++k)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t[k] += __shfl_down_sync(0xffffffffu, t[k], o);
    if (threadIdx.x == 0) {
#pragma unroll
      for (int k = 0; k < 5; ++k) out[k] = t[k];
      *ticket = 0u;
    }
  }
}
}  // namespace

cudaError_t launch_sum_partials(const float* partials, int64_t n, double* scratch, unsigned* ticket, double* out,
                                cudaStream_t stream) {
  const int64_t first = 152;  // blocks (at most kRedBlocks: the scratch holds that many)
  const int64_t chunk = (n + first - 1) / first;
  const int nb = (int)((n + chunk - 1) / chunk);
  sum_partials_kernel<<<nb, kAuxThreads, 0, stream>>>(partials, n, chunk, scratch, ticket, out);
  return cudaGetLastError();
}
cudaError_t tp_launch_mode_into(Sim* s, int field, const int64_t mode[3], double* out2) {
  LBM_TP_DISPATCH(mode_into_t, field, mode, out2);
}

cudaError_t tp_launch_reduce_into(Sim* s, double* partials, int nblocks, double* result) {
  LBM_TP_DISPATCH(reduce_into_t, partials, nblocks, result);
}

}  // namespace lbm
