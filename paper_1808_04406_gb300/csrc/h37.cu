// Kernels of the 37-velocity degree-9 lattice: the fused stream + collide
// sweep (AA pattern, one node per thread), initialisation, macroscopic fields,
// FP64 population exchange, grid totals and mode amplitudes.
//
// Units: velocities exchanged through the C ABI are in lattice units (lattice
// spacings per step); inside, Hermite units u_H = c u are used (xi_i = c e_i),
// in which the temperature theta is the paper's dimensionless theta.
#include <cstdlib>
#include <cstring>
#include <type_traits>

#include "h37_common.cuh"
#include "pair_io.cuh"
#include "reduce.cuh"

namespace lbm {
namespace {

constexpr int kH37Threads = 128;

inline h37::Model model_of(const Sim* s) {
  h37::Model m;
  m.thermal = (s->flags & LBM_THERMAL) ? 1 : 0;
  m.raw = (s->flags & LBM_RAW_MRT) ? 1 : 0;
  m.kfac = (s->flags & LBM_K72) ? 12.0f : 1.0f;
  m.eps_ref = s->theta_ref - 1.0;
  m.sround = (s->flags & LBM_STOCHASTIC_ROUND) && (s->storage == LBM_F16 || s->storage == LBM_BF16) ? 1 : 0;
  const uint64_t st = (uint64_t)s->step * 0x9E3779B97F4A7C15ull;  // a different seed for every step
  m.seed = (uint32_t)(st >> 32) ^ (uint32_t)st;
  return m;
}

inline h37::Grid2 grid2(const Sim* s) { return h37::Grid2{(int)s->nx, (int)s->ny, s->N}; }

// LBM_H37_SWEEP=scalar keeps the one-node kernel for every storage type (read at
// every launch; used to compare the two kernels).
// FP32 storage takes the correctly rounded transforms (the one-node kernel)
// unless the caller asked for the plain FP32 ones.
inline bool h37_exact_transforms(const Sim* s) {
  return s->storage == LBM_F32 && !(s->flags & LBM_FAST_TRANSFORMS);
}

inline bool h37_scalar_only() {
  const char* e = std::getenv("LBM_H37_SWEEP");
  return e && std::strcmp(e, "scalar") == 0;
}

// EXACT: correctly rounded transforms (FP32 storage unless LBM_FAST_TRANSFORMS).
template <int S, bool ODD, bool EXACT>
__global__ void __launch_bounds__(kH37Threads)
    h37_sweep_kernel(typename h37::Store<S>::type* __restrict__ f, h37::Grid2 g, Rates r, h37::Model m,
                     int* __restrict__ status) {
  using T = typename h37::Store<S>::calc;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= g.nx) return;
  const int y = blockIdx.y;
  T om[5];
#pragma unroll
  for (int n = 0; n < 5; ++n) om[n] = (T)r.w[n];
  T v[h37::kQ];
  h37::gather<S>(f, g, x, y, ODD ? 1 : 0, v);
  const bool ok = h37::collide<T, EXACT>(v, om, m);
  if (!ok) atomicOr(status, 1);
  // even sweep: population i goes to slot (x, opp(i)); odd sweep: to slot (x + e_i, i)
  const uint32_t node = (uint32_t)x + (uint32_t)g.nx * (uint32_t)y;
  h37::SrStream rs(m.seed, node);
#pragma unroll
  for (int j = 0; j < h37::kQ; ++j) {
    const T val = ODD ? v[j] : v[h37::opp(j)];
    const auto e = m.sround ? h37::encode_sr<S>(val, j, rs.next()) : h37::encode<S>(val, j);
    if (!ODD)
      f[(size_t)j * g.N + node] = e;
    else
      f[(size_t)j * g.N + h37::nbr(g, x, y, j)] = e;
  }
}

// Two nodes per thread in packed FP32x2 (FP32 / FP16 / BF16 storage, even nx).
// Even sweep: the pair (x0, x0 + 1), x0 even, reads and writes its own slots as
// aligned 2-element accesses.  Odd sweep: x0 odd (lane 1 = x0 + 1, wrapped), so
// the slot pair (x0 + e_x, x0 + 1 + e_x) starts on an even index for the 20
// directions with odd e_x (an aligned access; the periodic wrap preserves the
// parity because nx is even) and takes two 1-element accesses for the 17 with
// even e_x.
#ifndef LBM_H37_PAIR_MINB
#define LBM_H37_PAIR_MINB 3  // 168 registers (a few words spill): 12 warps per SM
#endif
// The update of pair xp of row blockIdx.y; with TOT the pair's conserved
// moments (drho, j_x, j_y in Hermite units, both lanes) go to mom[0..2].
template <int S, bool ODD, bool TOT>
__device__ __forceinline__ void h37_pair_update(typename PairIO<S>::E* __restrict__ f, const h37::Grid2& g,
                                                const Rates& r, const h37::Model& m, int* __restrict__ status,
                                                int xp, f2* mom) {
  using IO = PairIO<S>;
  using E = typename IO::E;
  const int y = blockIdx.y;
  const int x0 = 2 * xp + (ODD ? 1 : 0);
  const int nx = g.nx;
  auto wrapx = [&](int x) { return x < 0 ? x + nx : (x >= nx ? x - nx : x); };
  auto rowof = [&](int ey) -> uint32_t {
    int yy = y + ey;
    yy = yy < 0 ? yy + g.ny : (yy >= g.ny ? yy - g.ny : yy);
    return (uint32_t)nx * (uint32_t)yy;
  };
  f2 om[5];
#pragma unroll
  for (int n = 0; n < 5; ++n) om[n] = cst<f2>(r.w[n]);
  f2 v[h37::kQ];
#pragma unroll
  for (int j = 0; j < h37::kQ; ++j) {
    const E* fj = f + (size_t)j * g.N;
    f2 val;
    if (!ODD) {
      val = IO::load2(fj + rowof(0) + x0);
    } else {
      const int ex = h37::ex_of(j);
      const uint32_t ro = rowof(h37::ey_of(j));
      if (ex & 1)
        val = IO::load2(fj + ro + wrapx(x0 + ex));
      else
        val = IO::load11(fj + ro + wrapx(x0 + ex), fj + ro + wrapx(x0 + 1 + ex));
    }
    if (IO::kScaled) val = val * cst<f2>(h37::w_of(j));
    v[ODD ? h37::opp(j) : j] = val;
  }
  const bool ok = h37::collide<f2>(v, om, m, TOT ? mom : nullptr);
  if (!ok) atomicOr(status, 1);
  // the pair's own nodes (for the stochastic-rounding bits)
  const uint32_t n0 = (uint32_t)x0 + (uint32_t)nx * (uint32_t)y, n1 = (uint32_t)wrapx(x0 + 1) + (uint32_t)nx * (uint32_t)y;
  h37::SrStream rs0(m.seed, n0), rs1(m.seed, n1);
#pragma unroll
  for (int j = 0; j < h37::kQ; ++j) {
    E* fj = f + (size_t)j * g.N;
    f2 val = ODD ? v[j] : v[h37::opp(j)];
    if (IO::kScaled) val = val * cst<f2>(1.0 / h37::w_of(j));
    E* pa;
    E* pb;
    bool adjacent;
    if (!ODD) {
      pa = fj + rowof(0) + x0;
      pb = pa + 1;
      adjacent = true;
    } else {
      const int ex = h37::ex_of(j);
      const uint32_t ro = rowof(h37::ey_of(j));
      pa = fj + ro + wrapx(x0 + ex);
      pb = fj + ro + wrapx(x0 + 1 + ex);
      adjacent = (ex & 1) != 0;
    }
    if constexpr (S == LBM_F16 || S == LBM_BF16) {
      if (m.sround) {
        float lo, hi;
        unpack2(val, lo, hi);
        const uint32_t r0 = rs0.next(), r1 = rs1.next();
        const uint32_t w = S == LBM_F16 ? h37::sr_f16x2(lo, hi, r0, r1) : h37::sr_bf16x2(lo, hi, r0, r1);
        if (adjacent) {
          *reinterpret_cast<uint32_t*>(pa) = w;
        } else {
          *reinterpret_cast<unsigned short*>(pa) = (unsigned short)(w & 0xffffu);
          *reinterpret_cast<unsigned short*>(pb) = (unsigned short)(w >> 16);
        }
        continue;
      }
    }
    if (adjacent)
      IO::store2(pa, val);
    else
      IO::store11(pa, pb, val);
  }
}

template <int S, bool ODD>
__global__ void __launch_bounds__(kH37Threads, LBM_H37_PAIR_MINB)
    h37_pair_kernel(typename PairIO<S>::E* __restrict__ f, h37::Grid2 g, Rates r, h37::Model m,
                    int* __restrict__ status) {
  const int xp = blockIdx.x * blockDim.x + threadIdx.x;
  if (2 * xp >= g.nx) return;
  h37_pair_update<S, ODD, false>(f, g, r, m, status, xp, nullptr);
}

// The same sweep, which also writes the totals of the state it consumed (the
// quantities of the grid reduction: sum (rho - 1), sum rho u_x, sum rho u_y, 0,
// sum rho |u|^2 / 2, lattice units) as one FP32 partial per warp,
// partials[warp * 8 + k]; a warp sums its 64 nodes in FP32 (fixed shuffle tree).
template <int S, bool ODD>
__global__ void __launch_bounds__(kH37Threads, LBM_H37_PAIR_MINB)
    h37_pair_totals_kernel(typename PairIO<S>::E* __restrict__ f, h37::Grid2 g, Rates r, h37::Model m,
                           int* __restrict__ status, float* __restrict__ partials) {
  const int xp = blockIdx.x * blockDim.x + threadIdx.x;
  float acc[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
  if (2 * xp < g.nx) {
    f2 mom[3];
    h37_pair_update<S, ODD, true>(f, g, r, m, status, xp, mom);
    const float ic = (float)(1.0 / h37::kC);
    float d0, d1, jx0, jx1, jy0, jy1;
    unpack2(mom[0], d0, d1);
    unpack2(mom[1], jx0, jx1);
    unpack2(mom[2], jy0, jy1);
    jx0 *= ic;
    jx1 *= ic;
    jy0 *= ic;
    jy1 *= ic;
    acc[0] = d0 + d1;
    acc[1] = jx0 + jx1;
    acc[2] = jy0 + jy1;
    acc[4] = __fdividef(0.5f * (jx0 * jx0 + jy0 * jy0), 1.0f + d0) +
             __fdividef(0.5f * (jx1 * jx1 + jy1 * jy1), 1.0f + d1);
  }
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < 5; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_down_sync(0xffffffffu, acc[k], o);
  if (lane == 0) {
    const size_t b = (size_t)blockIdx.x + (size_t)gridDim.x * blockIdx.y;
    const size_t w = b * (kH37Threads / 32) + (threadIdx.x >> 5);
#pragma unroll
    for (int k = 0; k < 5; ++k) partials[w * 8 + k] = acc[k];
  }
}

__device__ __forceinline__ void xy_of(const h37::Grid2& g, int64_t n, int& x, int& y) {
  const uint32_t nn = (uint32_t)n, nx = (uint32_t)g.nx;
  y = (int)(nn / nx);
  x = (int)(nn - (uint32_t)y * nx);
}

template <int S, typename F>
__global__ void h37_init_kernel(typename h37::Store<S>::type* __restrict__ f, h37::Grid2 g,
                                const F* __restrict__ rho, const F* __restrict__ u,
                                const F* __restrict__ theta, double eps_ref, int64_t n0, int64_t cnt,
                                int64_t ld) {
  using T = typename h37::Store<S>::calc;
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= cnt) return;
  int x, y;
  xy_of(g, n0 + k, x, y);
  const T ux = (T)((double)u[k] * h37::kC), uy = (T)((double)u[ld + k] * h37::kC);
  const T th = theta ? (T)theta[k] : T(1);
  T v[h37::kQ];
  h37::equilibrium<T>(v, (T)rho[k], ux, uy, th, eps_ref);
  h37::scatter<S>(f, g, x, y, 0, v);
}

// rho, u (Hermite units) and theta of one node from its offsets
template <typename T>
__device__ __forceinline__ void node_macro(const T (&v)[h37::kQ], double eps_ref, int thermal, T& drho, T& ux,
                                           T& uy, T& eps) {
  T a[h37::kNC];
  h37::to_hermite<T>(v, a);
  drho = a[0];
  const T irho = T(1) / (T(1) + drho);
  ux = a[h37::cidx(1, 0)] * irho;
  uy = a[h37::cidx(0, 1)] * irho;
  eps = thermal ? T(0.5) * ((T(2) * (T)eps_ref + a[h37::cidx(2, 0)] + a[h37::cidx(0, 2)]) * irho -
                            (ux * ux + uy * uy))
                : T(0);
}

template <int S, typename F>
__global__ void h37_moments_kernel(const typename h37::Store<S>::type* __restrict__ f, h37::Grid2 g, int odd,
                                   h37::Model m, F* __restrict__ rho, F* __restrict__ u,
                                   F* __restrict__ theta, int64_t n0, int64_t cnt, int64_t ld) {
  using T = typename h37::Store<S>::calc;
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= cnt) return;
  int x, y;
  xy_of(g, n0 + k, x, y);
  T v[h37::kQ];
  h37::gather<S>(f, g, x, y, odd, v);
  // the moments in the wider of the compute and the output type, so that FP64
  // fields of FP32 (or 16-bit) storage carry no FP32 rounding of their own
  using M = typename std::conditional<(sizeof(F) > sizeof(T)), F, T>::type;
  M vm[h37::kQ];
#pragma unroll
  for (int i = 0; i < h37::kQ; ++i) vm[i] = (M)v[i];
  M drho, ux, uy, eps;
  node_macro<M>(vm, m.eps_ref, m.thermal, drho, ux, uy, eps);
  rho[k] = (F)(M(1) + drho);
  u[k] = (F)(ux * (M)(1.0 / h37::kC));
  u[ld + k] = (F)(uy * (M)(1.0 / h37::kC));
  if (theta) theta[k] = (F)(M(1) + eps);
}

template <int S>
__global__ void h37_get_pops_kernel(const typename h37::Store<S>::type* __restrict__ f, h37::Grid2 g, int odd,
                                    double eps_ref, double* __restrict__ out, int64_t n0, int64_t cnt,
                                    int64_t ld) {
  using T = typename h37::Store<S>::calc;
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= cnt) return;
  int x, y;
  xy_of(g, n0 + k, x, y);
  T v[h37::kQ];
  h37::gather<S>(f, g, x, y, odd, v);
#pragma unroll
  for (int i = 0; i < h37::kQ; ++i) out[i * ld + k] = h37::fref(i, eps_ref) + (double)v[i];
}

template <int S>
__global__ void h37_set_pops_kernel(typename h37::Store<S>::type* __restrict__ f, h37::Grid2 g, int odd,
                                    double eps_ref, const double* __restrict__ in, int64_t n0, int64_t cnt,
                                    int64_t ld) {
  using T = typename h37::Store<S>::calc;
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= cnt) return;
  int x, y;
  xy_of(g, n0 + k, x, y);
  T v[h37::kQ];
#pragma unroll
  for (int i = 0; i < h37::kQ; ++i) v[i] = (T)(in[i * ld + k] - h37::fref(i, eps_ref));
  h37::scatter<S>(f, g, x, y, odd, v);
}

// Grid totals: {sum (rho - 1), sum rho u_x, sum rho u_y, 0, sum rho |u|^2 / 2}, lattice units.
template <int S>
__global__ void __launch_bounds__(kAuxThreads)
    h37_reduce_kernel(const typename h37::Store<S>::type* __restrict__ f, h37::Grid2 g, int odd, h37::Model m,
                      double* __restrict__ partials) {
  using T = typename h37::Store<S>::calc;
  double acc[5] = {0, 0, 0, 0, 0};
  const T ic = (T)(1.0 / h37::kC);
  for (int y = blockIdx.x; y < g.ny; y += gridDim.x)
    for (int x = threadIdx.x; x < g.nx; x += blockDim.x) {
      T v[h37::kQ];
      h37::gather<S>(f, g, x, y, odd, v);
      T drho, ux, uy, eps;
      node_macro<T>(v, m.eps_ref, 0, drho, ux, uy, eps);
      const T r = T(1) + drho;
      ux = ux * ic;
      uy = uy * ic;
      acc[0] += (double)drho;
      acc[1] += (double)(r * ux);
      acc[2] += (double)(r * uy);
      acc[4] += (double)(T(0.5) * r * (ux * ux + uy * uy));
    }
  block_sum<5>(acc);
  if (threadIdx.x == 0)
    for (int k = 0; k < 5; ++k) partials[(size_t)blockIdx.x * 8 + k] = acc[k];
}

// Mode amplitude of field 0 = rho - 1, 1/2 = u_x/u_y (lattice units),
// 3 = theta - 1, 4 = rho theta - 1 (the constant adds N at k = 0, host side).
template <int S>
__global__ void __launch_bounds__(kAuxThreads)
    h37_mode_kernel(const typename h37::Store<S>::type* __restrict__ f, h37::Grid2 g, int odd, h37::Model m,
                    int field, long long mx, long long my, double* __restrict__ partials) {
  using T = typename h37::Store<S>::calc;
  double acc[2] = {0, 0};
  const long long ax = ((mx % g.nx) + g.nx) % g.nx, ay = ((my % g.ny) + g.ny) % g.ny;
  for (int y = blockIdx.x; y < g.ny; y += gridDim.x) {
    double sr, cr;
    sincospi(2.0 * (double)((ay * y) % g.ny) / g.ny, &sr, &cr);
    double ar = 0, ai = 0;
    for (int x = threadIdx.x; x < g.nx; x += blockDim.x) {
      T v[h37::kQ];
      h37::gather<S>(f, g, x, y, odd, v);
      T drho, ux, uy, eps;
      node_macro<T>(v, m.eps_ref, m.thermal, drho, ux, uy, eps);
      T q;
      if (field == 0) q = drho;
      else if (field == 1) q = ux * (T)(1.0 / h37::kC);
      else if (field == 2) q = uy * (T)(1.0 / h37::kC);
      else if (field == 3) q = eps;
      else q = drho + eps + drho * eps;  // (1 + drho)(1 + eps) - 1
      double sn, cs;
      sincospi(2.0 * (double)((ax * x) % g.nx) / g.nx, &sn, &cs);
      ar += (double)q * cs;
      ai -= (double)q * sn;
    }
    acc[0] += ar * cr + ai * sr;
    acc[1] += ai * cr - ar * sr;
  }
  block_sum<2>(acc);
  if (threadIdx.x == 0) {
    partials[(size_t)blockIdx.x * 8 + 0] = acc[0];
    partials[(size_t)blockIdx.x * 8 + 1] = acc[1];
  }
}

inline unsigned blocks_for(int64_t cnt) { return (unsigned)((cnt + kAuxThreads - 1) / kAuxThreads); }

template <int S>
cudaError_t pair_t(Sim* s, int odd) {
  using E = typename PairIO<S>::E;
  dim3 grid((unsigned)((s->nx / 2 + kH37Threads - 1) / kH37Threads), (unsigned)s->ny);
  E* f = static_cast<E*>(s->pop);
  if (odd)
    h37_pair_kernel<S, true><<<grid, kH37Threads, 0, s->stream>>>(f, grid2(s), s->rates, model_of(s),
                                                                    status_word(s));
  else
    h37_pair_kernel<S, false><<<grid, kH37Threads, 0, s->stream>>>(f, grid2(s), s->rates, model_of(s),
                                                                     status_word(s));
  return cudaGetLastError();
}

template <int S>
cudaError_t pair_totals_t(Sim* s, int odd, float* partials) {
  using E = typename PairIO<S>::E;
  dim3 grid((unsigned)((s->nx / 2 + kH37Threads - 1) / kH37Threads), (unsigned)s->ny);
  E* f = static_cast<E*>(s->pop);
  if (odd)
    h37_pair_totals_kernel<S, true><<<grid, kH37Threads, 0, s->stream>>>(f, grid2(s), s->rates, model_of(s),
                                                                           status_word(s), partials);
  else
    h37_pair_totals_kernel<S, false><<<grid, kH37Threads, 0, s->stream>>>(f, grid2(s), s->rates, model_of(s),
                                                                            status_word(s), partials);
  return cudaGetLastError();
}

template <int S>
cudaError_t sweep_t(Sim* s, int odd) {
  using E = typename h37::Store<S>::type;
  if constexpr (S != LBM_F64) {
    if (h37_pair_supported(s)) return pair_t<S>(s, odd);
  }
  dim3 grid((unsigned)((s->nx + kH37Threads - 1) / kH37Threads), (unsigned)s->ny);
  E* f = static_cast<E*>(s->pop);
  if constexpr (S == LBM_F32) {
    if (h37_exact_transforms(s)) {
      if (odd)
        h37_sweep_kernel<S, true, true><<<grid, kH37Threads, 0, s->stream>>>(f, grid2(s), s->rates, model_of(s),
                                                                           status_word(s));
      else
        h37_sweep_kernel<S, false, true><<<grid, kH37Threads, 0, s->stream>>>(f, grid2(s), s->rates, model_of(s),
                                                                            status_word(s));
      return cudaGetLastError();
    }
  }
  if (odd)
    h37_sweep_kernel<S, true, false><<<grid, kH37Threads, 0, s->stream>>>(f, grid2(s), s->rates, model_of(s),
                                                                          status_word(s));
  else
    h37_sweep_kernel<S, false, false><<<grid, kH37Threads, 0, s->stream>>>(f, grid2(s), s->rates, model_of(s),
                                                                           status_word(s));
  return cudaGetLastError();
}

template <int S>
cudaError_t init_t(Sim* s, const void* rho, const void* u, const void* th, int dtype, int64_t n0, int64_t cnt,
                   int64_t ld) {
  using E = typename h37::Store<S>::type;
  if (cnt <= 0) return cudaSuccess;
  E* f = static_cast<E*>(s->pop);
  const double er = s->theta_ref - 1.0;
  if (dtype == LBM_DTYPE_F64)
    h37_init_kernel<S, double><<<blocks_for(cnt), kAuxThreads, 0, s->stream>>>(
        f, grid2(s), static_cast<const double*>(rho), static_cast<const double*>(u),
        static_cast<const double*>(th), er, n0, cnt, ld);
  else
    h37_init_kernel<S, float><<<blocks_for(cnt), kAuxThreads, 0, s->stream>>>(
        f, grid2(s), static_cast<const float*>(rho), static_cast<const float*>(u), static_cast<const float*>(th),
        er, n0, cnt, ld);
  return cudaGetLastError();
}

template <int S>
cudaError_t moments_t(Sim* s, void* rho, void* u, void* th, int dtype, int64_t n0, int64_t cnt, int64_t ld) {
  using E = typename h37::Store<S>::type;
  if (cnt <= 0) return cudaSuccess;
  const E* f = static_cast<const E*>(s->pop);
  const int odd = (int)(s->step & 1);
  if (dtype == LBM_DTYPE_F64)
    h37_moments_kernel<S, double><<<blocks_for(cnt), kAuxThreads, 0, s->stream>>>(
        f, grid2(s), odd, model_of(s), static_cast<double*>(rho), static_cast<double*>(u),
        static_cast<double*>(th), n0, cnt, ld);
  else
    h37_moments_kernel<S, float><<<blocks_for(cnt), kAuxThreads, 0, s->stream>>>(
        f, grid2(s), odd, model_of(s), static_cast<float*>(rho), static_cast<float*>(u), static_cast<float*>(th),
        n0, cnt, ld);
  return cudaGetLastError();
}

template <int S>
cudaError_t get_pops_t(Sim* s, double* out, int64_t n0, int64_t cnt, int64_t ld) {
  using E = typename h37::Store<S>::type;
  if (cnt <= 0) return cudaSuccess;
  h37_get_pops_kernel<S><<<blocks_for(cnt), kAuxThreads, 0, s->stream>>>(
      static_cast<const E*>(s->pop), grid2(s), (int)(s->step & 1), s->theta_ref - 1.0, out, n0, cnt, ld);
  return cudaGetLastError();
}

template <int S>
cudaError_t set_pops_t(Sim* s, const double* in, int64_t n0, int64_t cnt, int64_t ld) {
  using E = typename h37::Store<S>::type;
  if (cnt <= 0) return cudaSuccess;
  h37_set_pops_kernel<S><<<blocks_for(cnt), kAuxThreads, 0, s->stream>>>(
      static_cast<E*>(s->pop), grid2(s), (int)(s->step & 1), s->theta_ref - 1.0, in, n0, cnt, ld);
  return cudaGetLastError();
}

template <int S>
cudaError_t reduce_into_t(Sim* s, double* partials, int nblocks, double* result) {
  using E = typename h37::Store<S>::type;
  h37_reduce_kernel<S><<<nblocks, kAuxThreads, 0, s->stream>>>(static_cast<const E*>(s->pop), grid2(s),
                                                               (int)(s->step & 1), model_of(s), partials);
  finalize_kernel<<<1, kAuxThreads, 0, s->stream>>>(partials, nblocks, 5, result);
  return cudaGetLastError();
}

template <int S>
cudaError_t mode_into_t(Sim* s, int field, const int64_t m[3], double* out2) {
  using E = typename h37::Store<S>::type;
  h37_mode_kernel<S><<<kRedBlocks, kAuxThreads, 0, s->stream>>>(static_cast<const E*>(s->pop), grid2(s),
                                                                (int)(s->step & 1), model_of(s), field,
                                                                (long long)m[0], (long long)m[1], partials_buf(s));
  finalize_kernel<<<1, kAuxThreads, 0, s->stream>>>(partials_buf(s), kRedBlocks, 2, out2);
  return cudaGetLastError();
}

#define LBM_H37_DISPATCH(FN, ...)                          \
  do {                                                     \
    switch (s->storage) {                                  \
      case LBM_F64: return FN<LBM_F64>(s, __VA_ARGS__);    \
      case LBM_F32: return FN<LBM_F32>(s, __VA_ARGS__);    \
      case LBM_F16: return FN<LBM_F16>(s, __VA_ARGS__);    \
      case LBM_BF16: return FN<LBM_BF16>(s, __VA_ARGS__);  \
    }                                                      \
    return cudaErrorInvalidValue;                          \
  } while (0)

}  // namespace

cudaError_t h37_launch_sweep(Sim* s, int odd) { LBM_H37_DISPATCH(sweep_t, odd); }

bool h37_pair_supported(const Sim* s) {
  return s->storage != LBM_F64 && (s->nx & 1) == 0 && !h37_scalar_only() && !h37_exact_transforms(s);
}
int64_t h37_pair_warps(const Sim* s) {
  return ((s->nx / 2 + kH37Threads - 1) / kH37Threads) * s->ny * (kH37Threads / 32);
}
cudaError_t h37_launch_pair_sweep_totals(Sim* s, int odd, float* partials) {
  switch (s->storage) {
    case LBM_F32: return pair_totals_t<LBM_F32>(s, odd, partials);
    case LBM_F16: return pair_totals_t<LBM_F16>(s, odd, partials);
    case LBM_BF16: return pair_totals_t<LBM_BF16>(s, odd, partials);
  }
  return cudaErrorInvalidValue;
}
cudaError_t h37_launch_init(Sim* s, const void* rho, const void* u, const void* theta, int dtype, int64_t n0,
                            int64_t cnt, int64_t ld) {
  LBM_H37_DISPATCH(init_t, rho, u, theta, dtype, n0, cnt, ld);
}
cudaError_t h37_launch_moments(Sim* s, void* rho, void* u, void* theta, int dtype, int64_t n0, int64_t cnt,
                               int64_t ld) {
  LBM_H37_DISPATCH(moments_t, rho, u, theta, dtype, n0, cnt, ld);
}
cudaError_t h37_launch_get_pops(Sim* s, double* f, int64_t n0, int64_t cnt, int64_t ld) {
  LBM_H37_DISPATCH(get_pops_t, f, n0, cnt, ld);
}
cudaError_t h37_launch_set_pops(Sim* s, const double* f, int64_t n0, int64_t cnt, int64_t ld) {
  LBM_H37_DISPATCH(set_pops_t, f, n0, cnt, ld);
}
cudaError_t h37_launch_reduce_into(Sim* s, double* partials, int nblocks, double* result) {
  LBM_H37_DISPATCH(reduce_into_t, partials, nblocks, result);
}
cudaError_t h37_launch_mode_into(Sim* s, int field, const int64_t mode[3], double* out2) {
  LBM_H37_DISPATCH(mode_into_t, field, mode, out2);
}

}  // namespace lbm
