// Kernels for a caller-supplied two-dimensional Hermite lattice (LBM_HERMITE):
// the minimal square-symmetric rules of Sec. III.A (17 velocities, degree 7,
// truncation N = 3; 37 velocities, degree 9, N = 3 or 4) or any other such
// rule that integrates the Gaussian exactly to degree 2N.  The collision is the
// same Hermite-space CM-MRT as on the built-in 37-velocity lattice
// (h37::collide_coeffs: Eq. omega in the relative frame, K = 6 at order 4);
// only the projection onto and from the Hermite coefficients differs: it uses
// per-simulation tables (HTables) passed by value instead of compiled-in
// constants.  One node per thread, AA pattern, FP64 or FP32 offsets from
// f_eq(1, 0, theta_ref).  Velocities crossing the C ABI are in lattice units.
#include <cmath>
#include <type_traits>

#include "h37_common.cuh"
#include "reduce.cuh"

namespace lbm {

void hgen_build_tables(const HLattice& L, double theta_ref, HTables* t) {
  auto he = [](int n, double x) {
    return n == 0 ? 1.0 : n == 1 ? x : n == 2 ? x * x - 1.0 : n == 3 ? x * x * x - 3.0 * x
                                                                       : x * x * x * x - 6.0 * x * x + 3.0;
  };
  auto fct = [](int n) { return n <= 1 ? 1.0 : n == 2 ? 2.0 : n == 3 ? 6.0 : 24.0; };
  const double er = theta_ref - 1.0;
  auto aref = [&](int p, int q) {  // Hermite coefficients of f_eq(1, 0, theta_ref)
    auto g = [&](int n) { return n == 0 ? 1.0 : n == 2 ? er : n == 4 ? 3.0 * er * er : 0.0; };
    return g(p) * g(q);
  };
  const int nc = (L.order + 1) * (L.order + 2) / 2;
  t->q = L.q;
  t->nc = nc;
  t->c = L.c;
  for (int i = 0; i < L.q; ++i) {
    t->ex[i] = L.ex[i];
    t->ey[i] = L.ey[i];
    t->opp[i] = L.opp[i];
    const double x = L.c * L.ex[i], y = L.c * L.ey[i];
    double fr = 0.0;
    for (int k = 0; k < 15; ++k) {
      const int p = h37::cp(k), q = h37::cq(k);
      const double h = k < nc ? he(p, x) * he(q, y) : 0.0;
      t->H[k][i] = h;
      t->R[i][k] = k < nc ? L.w[i] * h / (fct(p) * fct(q)) : 0.0;
      if (k < nc) fr += aref(p, q) * t->R[i][k];
    }
    t->fref[i] = fr;
  }
}

namespace {

constexpr int kHgThreads = 128;

template <int S>
struct HStore;
template <>
struct HStore<LBM_F64> {
  using type = double;
};
template <>
struct HStore<LBM_F32> {
  using type = float;
};

struct HGrid {
  int nx, ny;
  int64_t N;
};

__device__ __forceinline__ uint32_t hnbr(const HGrid& g, int x, int y, int dx, int dy) {
  int xn = x + dx, yn = y + dy;
  xn = xn < 0 ? xn + g.nx : (xn >= g.nx ? xn - g.nx : xn);
  yn = yn < 0 ? yn + g.ny : (yn >= g.ny ? yn - g.ny : yn);
  return (uint32_t)xn + (uint32_t)g.nx * (uint32_t)yn;
}

// Offsets of node (x, y) in the state of the given parity.  Odd state: the
// population i of node x sits in slot (x - e_i, opp(i)).
template <typename T, int Q>
__device__ __forceinline__ void hgather(const T* __restrict__ f, const HGrid& g, const HTables& t, int x, int y,
                                        int odd, T (&v)[Q]) {
  const uint32_t node = (uint32_t)x + (uint32_t)g.nx * (uint32_t)y;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    if (!odd)
      v[i] = f[(size_t)i * g.N + node];
    else
      v[i] = f[(size_t)t.opp[i] * g.N + hnbr(g, x, y, -t.ex[i], -t.ey[i])];
  }
}

// Write the offsets of node (x, y) as the state of the given parity.
template <typename T, int Q>
__device__ __forceinline__ void hscatter(T* __restrict__ f, const HGrid& g, const HTables& t, int x, int y, int odd,
                                         const T (&v)[Q]) {
  const uint32_t node = (uint32_t)x + (uint32_t)g.nx * (uint32_t)y;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    if (!odd)
      f[(size_t)i * g.N + node] = v[i];
    else
      f[(size_t)t.opp[i] * g.N + hnbr(g, x, y, -t.ex[i], -t.ey[i])] = v[i];
  }
}

template <typename T, int Q, int NC>
__device__ __forceinline__ void to_coeffs(const HTables& t, const T (&v)[Q], T (&a)[NC]) {
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    T s = cst<T>(0.0);
#pragma unroll
    for (int i = 0; i < Q; ++i) s = fma_(v[i], (T)t.H[k][i], s);
    a[k] = s;
  }
}

template <typename T, int Q, int NC>
__device__ __forceinline__ void from_coeffs(const HTables& t, const T (&a)[NC], T (&v)[Q]) {
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    T s = cst<T>(0.0);
#pragma unroll
    for (int k = 0; k < NC; ++k) s = fma_(a[k], (T)t.R[i][k], s);
    v[i] = s;
  }
}

// The projection tables as FP32 pairs hi + lo (hi = the FP32 rounding, lo = the
// FP32 rounding of the rest), for the correctly rounded FP32 transforms (see
// h37_common.cuh): built on the host from the FP64 tables at each launch.
struct HSplit {
  float Hh[15][kHQMax], Hl[15][kHQMax];
  float Rh[kHQMax][15], Rl[kHQMax][15];
};

void split_tables(const HTables& t, HSplit* out) {
  for (int k = 0; k < 15; ++k)
    for (int i = 0; i < kHQMax; ++i) {
      const double h = i < t.q ? t.H[k][i] : 0.0, r = i < t.q ? t.R[i][k] : 0.0;
      out->Hh[k][i] = (float)h;
      out->Hl[k][i] = (float)(h - (double)out->Hh[k][i]);
      out->Rh[i][k] = (float)r;
      out->Rl[i][k] = (float)(r - (double)out->Rh[i][k]);
    }
}

template <int Q, int NC>
__device__ __forceinline__ void to_coeffs_exact(const HSplit& t, const float (&v)[Q], float (&a)[NC]) {
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    float s = 0.f, c = 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) h37::dot2_add_split(s, c, v[i], t.Hh[k][i], t.Hl[k][i]);
    a[k] = s + c;
  }
}

template <int Q, int NC>
__device__ __forceinline__ void from_coeffs_exact(const HSplit& t, const float (&a)[NC], float (&v)[Q]) {
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    float s = 0.f, c = 0.f;
#pragma unroll
    for (int k = 0; k < NC; ++k) h37::dot2_add_split(s, c, a[k], t.Rh[i][k], t.Rl[i][k]);
    v[i] = s + c;
  }
}

// EXACT: FP32 storage with the correctly rounded transforms (tables in sp).
template <int S, int Q, int NC, bool ODD, bool EXACT>
__global__ void __launch_bounds__(kHgThreads)
    hgen_sweep_kernel(typename HStore<S>::type* __restrict__ f, HGrid g, const HTables t, Rates r, h37::Model m,
                      int* __restrict__ status, const HSplit sp) {
  using T = typename HStore<S>::type;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= g.nx) return;
  const int y = blockIdx.y;
  T om[5];
#pragma unroll
  for (int n = 0; n < 5; ++n) om[n] = (T)r.w[n];
  T v[Q];
  const uint32_t node = (uint32_t)x + (uint32_t)g.nx * (uint32_t)y;
  // even state: population i of node x in slot (x, i); odd state: in slot (x - e_i, opp(i))
#pragma unroll
  for (int i = 0; i < Q; ++i)
    v[i] = ODD ? f[(size_t)t.opp[i] * g.N + hnbr(g, x, y, -t.ex[i], -t.ey[i])] : f[(size_t)i * g.N + node];
  T a[NC];
  if constexpr (EXACT)
    to_coeffs_exact<Q, NC>(sp, v, a);
  else
    to_coeffs<T, Q, NC>(t, v, a);
  if (!h37::collide_coeffs<T, NC>(a, om, m)) atomicOr(status, 1);
  if constexpr (EXACT)
    from_coeffs_exact<Q, NC>(sp, a, v);
  else
    from_coeffs<T, Q, NC>(t, a, v);
  // even sweep: population i to slot (x, opp(i)); odd sweep: to slot (x + e_i, i)
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    if (!ODD)
      f[(size_t)t.opp[i] * g.N + node] = v[i];
    else
      f[(size_t)i * g.N + hnbr(g, x, y, t.ex[i], t.ey[i])] = v[i];
  }
}

__device__ __forceinline__ void hxy_of(const HGrid& g, int64_t n, int& x, int& y) {
  const uint32_t nn = (uint32_t)n, nx = (uint32_t)g.nx;
  y = (int)(nn / nx);
  x = (int)(nn - (uint32_t)y * nx);
}

template <int S, int Q, int NC, typename F>
__global__ void hgen_init_kernel(typename HStore<S>::type* __restrict__ f, HGrid g, const HTables t, double eps_ref,
                                 const F* __restrict__ rho, const F* __restrict__ u, const F* __restrict__ theta,
                                 int64_t n0, int64_t cnt, int64_t ld) {
  using T = typename HStore<S>::type;
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= cnt) return;
  int x, y;
  hxy_of(g, n0 + k, x, y);
  const T ux = (T)((double)u[k] * t.c), uy = (T)((double)u[ld + k] * t.c);
  const T eps = theta ? (T)((double)theta[k] - 1.0) : cst<T>(0.0);
  T gx[5], gy[5];
  h37::g_forms<T>(ux, eps, gx);
  h37::g_forms<T>(uy, eps, gy);
  T a[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c)
    a[c] = (T)rho[k] * gx[h37::cp(c)] * gy[h37::cq(c)] - h37::aref<T>(c, (T)eps_ref);
  T v[Q];
  from_coeffs<T, Q, NC>(t, a, v);
  hscatter<T, Q>(f, g, t, x, y, 0, v);
}

// rho - 1, u (Hermite units) and theta - 1 of one node from its offsets
template <typename T, int Q, int NC>
__device__ __forceinline__ void hnode_macro(const HTables& t, const T (&v)[Q], double eps_ref, int thermal, T& drho,
                                            T& ux, T& uy, T& eps) {
  T a[NC];
  to_coeffs<T, Q, NC>(t, v, a);
  drho = a[0];
  const T irho = cst<T>(1.0) / (cst<T>(1.0) + drho);
  ux = a[h37::cidx(1, 0)] * irho;
  uy = a[h37::cidx(0, 1)] * irho;
  eps = thermal ? cst<T>(0.5) * ((cst<T>(2.0 * eps_ref) + a[h37::cidx(2, 0)] + a[h37::cidx(0, 2)]) * irho -
                                 (ux * ux + uy * uy))
                : cst<T>(0.0);
}

template <int S, int Q, int NC, typename F>
__global__ void hgen_moments_kernel(const typename HStore<S>::type* __restrict__ f, HGrid g, const HTables t, int odd,
                                    double eps_ref, int thermal, F* __restrict__ rho, F* __restrict__ u,
                                    F* __restrict__ theta, int64_t n0, int64_t cnt, int64_t ld) {
  using T = typename HStore<S>::type;
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= cnt) return;
  int x, y;
  hxy_of(g, n0 + k, x, y);
  T v[Q];
  hgather<T, Q>(f, g, t, x, y, odd, v);
  // the moments in the wider of the storage and the output type, so that FP64
  // fields of FP32 storage carry no FP32 rounding of their own
  using M = typename std::conditional<(sizeof(F) > sizeof(T)), F, T>::type;
  M vm[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) vm[i] = (M)v[i];
  M drho, ux, uy, eps;
  hnode_macro<M, Q, NC>(t, vm, eps_ref, thermal, drho, ux, uy, eps);
  rho[k] = (F)(cst<M>(1.0) + drho);
  u[k] = (F)((double)ux / t.c);
  u[ld + k] = (F)((double)uy / t.c);
  if (theta) theta[k] = (F)(cst<M>(1.0) + eps);
}

template <int S, int Q>
__global__ void hgen_get_pops_kernel(const typename HStore<S>::type* __restrict__ f, HGrid g, const HTables t, int odd,
                                     double* __restrict__ out, int64_t n0, int64_t cnt, int64_t ld) {
  using T = typename HStore<S>::type;
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= cnt) return;
  int x, y;
  hxy_of(g, n0 + k, x, y);
  T v[Q];
  hgather<T, Q>(f, g, t, x, y, odd, v);
#pragma unroll
  for (int i = 0; i < Q; ++i) out[i * ld + k] = t.fref[i] + (double)v[i];
}

template <int S, int Q>
__global__ void hgen_set_pops_kernel(typename HStore<S>::type* __restrict__ f, HGrid g, const HTables t, int odd,
                                     const double* __restrict__ in, int64_t n0, int64_t cnt, int64_t ld) {
  using T = typename HStore<S>::type;
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= cnt) return;
  int x, y;
  hxy_of(g, n0 + k, x, y);
  T v[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) v[i] = (T)(in[i * ld + k] - t.fref[i]);
  hscatter<T, Q>(f, g, t, x, y, odd, v);
}

// Grid totals {sum (rho - 1), sum rho u_x, sum rho u_y, 0, sum rho |u|^2 / 2}, lattice units.
template <int S, int Q, int NC>
__global__ void __launch_bounds__(kAuxThreads)
    hgen_reduce_kernel(const typename HStore<S>::type* __restrict__ f, HGrid g, const HTables t, int odd,
                       double eps_ref, double* __restrict__ partials) {
  using T = typename HStore<S>::type;
  double acc[5] = {0, 0, 0, 0, 0};
  for (int y = blockIdx.x; y < g.ny; y += gridDim.x)
    for (int x = threadIdx.x; x < g.nx; x += blockDim.x) {
      T v[Q];
      hgather<T, Q>(f, g, t, x, y, odd, v);
      T drho, ux, uy, eps;
      hnode_macro<T, Q, NC>(t, v, eps_ref, 0, drho, ux, uy, eps);
      const double r = 1.0 + (double)drho, vx = (double)ux / t.c, vy = (double)uy / t.c;
      acc[0] += (double)drho;
      acc[1] += r * vx;
      acc[2] += r * vy;
      acc[4] += 0.5 * r * (vx * vx + vy * vy);
    }
  block_sum<5>(acc);
  if (threadIdx.x == 0)
    for (int k = 0; k < 5; ++k) partials[(size_t)blockIdx.x * 8 + k] = acc[k];
}

// Mode amplitude of field 0 = rho - 1, 1/2 = u_x/u_y (lattice units), 3 = theta - 1,
// 4 = rho theta - 1.
template <int S, int Q, int NC>
__global__ void __launch_bounds__(kAuxThreads)
    hgen_mode_kernel(const typename HStore<S>::type* __restrict__ f, HGrid g, const HTables t, int odd, double eps_ref,
                     int thermal, int field, long long mx, long long my, double* __restrict__ partials) {
  using T = typename HStore<S>::type;
  double acc[2] = {0, 0};
  const long long ax = ((mx % g.nx) + g.nx) % g.nx, ay = ((my % g.ny) + g.ny) % g.ny;
  for (int y = blockIdx.x; y < g.ny; y += gridDim.x) {
    double sr, cr;
    sincospi(2.0 * (double)((ay * y) % g.ny) / g.ny, &sr, &cr);
    double ar = 0, ai = 0;
    for (int x = threadIdx.x; x < g.nx; x += blockDim.x) {
      T v[Q];
      hgather<T, Q>(f, g, t, x, y, odd, v);
      T drho, ux, uy, eps;
      hnode_macro<T, Q, NC>(t, v, eps_ref, thermal, drho, ux, uy, eps);
      double q;
      if (field == 0) q = (double)drho;
      else if (field == 1) q = (double)ux / t.c;
      else if (field == 2) q = (double)uy / t.c;
      else if (field == 3) q = (double)eps;
      else q = (double)drho + (double)eps + (double)drho * (double)eps;  // (1 + drho)(1 + eps) - 1
      double sn, cs;
      sincospi(2.0 * (double)((ax * x) % g.nx) / g.nx, &sn, &cs);
      ar += q * cs;
      ai -= q * sn;
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

inline HGrid hgrid(const Sim* s) { return HGrid{(int)s->nx, (int)s->ny, s->N}; }
inline unsigned hblocks(int64_t cnt) { return (unsigned)((cnt + kAuxThreads - 1) / kAuxThreads); }

inline h37::Model hmodel(const Sim* s) {
  h37::Model m;
  m.thermal = (s->flags & LBM_THERMAL) ? 1 : 0;
  m.raw = 0;
  m.kfac = 1.0f;
  m.eps_ref = s->theta_ref - 1.0;
  m.sround = 0;
  m.seed = 0;
  return m;
}

template <int S, int Q, int NC, bool EXACT>
cudaError_t sweep_e(Sim* s, int odd, const HSplit& sp) {
  using E = typename HStore<S>::type;
  dim3 grid((unsigned)((s->nx + kHgThreads - 1) / kHgThreads), (unsigned)s->ny);
  E* f = static_cast<E*>(s->pop);
  if (odd)
    hgen_sweep_kernel<S, Q, NC, true, EXACT><<<grid, kHgThreads, 0, s->stream>>>(f, hgrid(s), *s->ht, s->rates,
                                                                                 hmodel(s), status_word(s), sp);
  else
    hgen_sweep_kernel<S, Q, NC, false, EXACT><<<grid, kHgThreads, 0, s->stream>>>(f, hgrid(s), *s->ht, s->rates,
                                                                                  hmodel(s), status_word(s), sp);
  return cudaGetLastError();
}

// FP32 storage takes the correctly rounded transforms unless LBM_FAST_TRANSFORMS.
template <int S, int Q, int NC>
cudaError_t sweep_t(Sim* s, int odd) {
  // host staging of the split tables, one per host thread (the launch copies its parameters)
  thread_local static HSplit sp;
  if constexpr (S == LBM_F32) {
    if (!(s->flags & LBM_FAST_TRANSFORMS)) {
      split_tables(*s->ht, &sp);
      return sweep_e<S, Q, NC, true>(s, odd, sp);
    }
  }
  return sweep_e<S, Q, NC, false>(s, odd, sp);
}

template <int S, int Q, int NC>
cudaError_t init_t(Sim* s, const void* rho, const void* u, const void* th, int dtype, int64_t n0, int64_t cnt,
                   int64_t ld) {
  using E = typename HStore<S>::type;
  if (cnt <= 0) return cudaSuccess;
  E* f = static_cast<E*>(s->pop);
  const double er = s->theta_ref - 1.0;
  if (dtype == LBM_DTYPE_F64)
    hgen_init_kernel<S, Q, NC, double><<<hblocks(cnt), kAuxThreads, 0, s->stream>>>(
        f, hgrid(s), *s->ht, er, static_cast<const double*>(rho), static_cast<const double*>(u),
        static_cast<const double*>(th), n0, cnt, ld);
  else
    hgen_init_kernel<S, Q, NC, float><<<hblocks(cnt), kAuxThreads, 0, s->stream>>>(
        f, hgrid(s), *s->ht, er, static_cast<const float*>(rho), static_cast<const float*>(u),
        static_cast<const float*>(th), n0, cnt, ld);
  return cudaGetLastError();
}

template <int S, int Q, int NC>
cudaError_t moments_t(Sim* s, void* rho, void* u, void* th, int dtype, int64_t n0, int64_t cnt, int64_t ld) {
  using E = typename HStore<S>::type;
  if (cnt <= 0) return cudaSuccess;
  const E* f = static_cast<const E*>(s->pop);
  const int odd = (int)(s->step & 1);
  const int thermal = (s->flags & LBM_THERMAL) ? 1 : 0;
  if (dtype == LBM_DTYPE_F64)
    hgen_moments_kernel<S, Q, NC, double><<<hblocks(cnt), kAuxThreads, 0, s->stream>>>(
        f, hgrid(s), *s->ht, odd, s->theta_ref - 1.0, thermal, static_cast<double*>(rho), static_cast<double*>(u),
        static_cast<double*>(th), n0, cnt, ld);
  else
    hgen_moments_kernel<S, Q, NC, float><<<hblocks(cnt), kAuxThreads, 0, s->stream>>>(
        f, hgrid(s), *s->ht, odd, s->theta_ref - 1.0, thermal, static_cast<float*>(rho), static_cast<float*>(u),
        static_cast<float*>(th), n0, cnt, ld);
  return cudaGetLastError();
}

template <int S, int Q, int NC>
cudaError_t get_pops_t(Sim* s, double* out, int64_t n0, int64_t cnt, int64_t ld) {
  using E = typename HStore<S>::type;
  if (cnt <= 0) return cudaSuccess;
  hgen_get_pops_kernel<S, Q><<<hblocks(cnt), kAuxThreads, 0, s->stream>>>(
      static_cast<const E*>(s->pop), hgrid(s), *s->ht, (int)(s->step & 1), out, n0, cnt, ld);
  return cudaGetLastError();
}

template <int S, int Q, int NC>
cudaError_t set_pops_t(Sim* s, const double* in, int64_t n0, int64_t cnt, int64_t ld) {
  using E = typename HStore<S>::type;
  if (cnt <= 0) return cudaSuccess;
  hgen_set_pops_kernel<S, Q><<<hblocks(cnt), kAuxThreads, 0, s->stream>>>(
      static_cast<E*>(s->pop), hgrid(s), *s->ht, (int)(s->step & 1), in, n0, cnt, ld);
  return cudaGetLastError();
}

template <int S, int Q, int NC>
cudaError_t reduce_into_t(Sim* s, double* partials, int nblocks, double* result) {
  using E = typename HStore<S>::type;
  hgen_reduce_kernel<S, Q, NC><<<nblocks, kAuxThreads, 0, s->stream>>>(
      static_cast<const E*>(s->pop), hgrid(s), *s->ht, (int)(s->step & 1), s->theta_ref - 1.0, partials);
  finalize_kernel<<<1, kAuxThreads, 0, s->stream>>>(partials, nblocks, 5, result);
  return cudaGetLastError();
}

template <int S, int Q, int NC>
cudaError_t mode_into_t(Sim* s, int field, const int64_t m[3], double* out2) {
  using E = typename HStore<S>::type;
  hgen_mode_kernel<S, Q, NC><<<kRedBlocks, kAuxThreads, 0, s->stream>>>(
      static_cast<const E*>(s->pop), hgrid(s), *s->ht, (int)(s->step & 1), s->theta_ref - 1.0,
      (s->flags & LBM_THERMAL) ? 1 : 0, field, (long long)m[0], (long long)m[1], partials_buf(s));
  finalize_kernel<<<1, kAuxThreads, 0, s->stream>>>(partials_buf(s), kRedBlocks, 2, out2);
  return cudaGetLastError();
}

// storage (FP64 / FP32) x (Q, NC) in {(17, 10), (37, 10), (37, 15)}
#define LBM_HGEN_DISPATCH(FN, ...)                                                        \
  do {                                                                                    \
    const int key = s->hl.q * 100 + s->ht->nc;                                            \
    if (s->storage == LBM_F64) {                                                          \
      if (key == 1710) return FN<LBM_F64, 17, 10>(s, __VA_ARGS__);                        \
      if (key == 3710) return FN<LBM_F64, 37, 10>(s, __VA_ARGS__);                        \
      if (key == 3715) return FN<LBM_F64, 37, 15>(s, __VA_ARGS__);                        \
    } else if (s->storage == LBM_F32) {                                                   \
      if (key == 1710) return FN<LBM_F32, 17, 10>(s, __VA_ARGS__);                        \
      if (key == 3710) return FN<LBM_F32, 37, 10>(s, __VA_ARGS__);                        \
      if (key == 3715) return FN<LBM_F32, 37, 15>(s, __VA_ARGS__);                        \
    }                                                                                     \
    return cudaErrorInvalidValue;                                                         \
  } while (0)

}  // namespace

cudaError_t hgen_launch_sweep(Sim* s, int odd) { LBM_HGEN_DISPATCH(sweep_t, odd); }
cudaError_t hgen_launch_init(Sim* s, const void* rho, const void* u, const void* theta, int dtype, int64_t n0,
                             int64_t cnt, int64_t ld) {
  LBM_HGEN_DISPATCH(init_t, rho, u, theta, dtype, n0, cnt, ld);
}
cudaError_t hgen_launch_moments(Sim* s, void* rho, void* u, void* theta, int dtype, int64_t n0, int64_t cnt,
                                int64_t ld) {
  LBM_HGEN_DISPATCH(moments_t, rho, u, theta, dtype, n0, cnt, ld);
}
cudaError_t hgen_launch_get_pops(Sim* s, double* f, int64_t n0, int64_t cnt, int64_t ld) {
  LBM_HGEN_DISPATCH(get_pops_t, f, n0, cnt, ld);
}
cudaError_t hgen_launch_set_pops(Sim* s, const double* f, int64_t n0, int64_t cnt, int64_t ld) {
  LBM_HGEN_DISPATCH(set_pops_t, f, n0, cnt, ld);
}
cudaError_t hgen_launch_reduce_into(Sim* s, double* partials, int nblocks, double* result) {
  LBM_HGEN_DISPATCH(reduce_into_t, partials, nblocks, result);
}
cudaError_t hgen_launch_mode_into(Sim* s, int field, const int64_t mode[3], double* out2) {
  LBM_HGEN_DISPATCH(mode_into_t, field, mode, out2);
}

}  // namespace lbm
