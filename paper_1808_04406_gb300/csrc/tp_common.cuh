// Device-side building blocks for the tensor-product lattices D2Q9 / D3Q27:
// compile-time lattice constants, the storage codecs, the CM-MRT collision in
// deviation form and the AA-pattern gather / scatter of one node.
//
// Velocity index i = sum_d (e_id + 1) 3^d, e_id in {-1, 0, 1}; moment index
// a = sum_d alpha_d 3^d with alpha_d in {0, 1, 2} and order |a| = sum_d alpha_d.
// Population storage holds offsets from the rest equilibrium w_i.
#pragma once

#include "f32x2.cuh"
#include "lbm_internal.cuh"

namespace lbm {
namespace tp {

__host__ __device__ constexpr int p3(int d) { return d == 0 ? 1 : (d == 1 ? 3 : 9); }
__host__ __device__ constexpr int dig(int i, int d) { return (i / p3(d)) % 3; }
template <int D>
__host__ __device__ constexpr int qof() { return D == 2 ? 9 : 27; }
template <int D>
__host__ __device__ constexpr int opp(int i) { return qof<D>() - 1 - i; }
template <int D>
__host__ __device__ constexpr int order_of(int a) {
  return dig(a, 0) + dig(a, 1) + (D == 3 ? dig(a, 2) : 0);
}
// Three-point Gauss-Hermite weights per axis: 2/3 at rest, 1/6 for e = +-1.
__host__ __device__ constexpr double w1(int digit) { return digit == 1 ? 2.0 / 3.0 : 1.0 / 6.0; }
__host__ __device__ constexpr double iw1(int digit) { return digit == 1 ? 1.5 : 6.0; }
template <int D>
__host__ __device__ constexpr double wq(int i) {
  return w1(dig(i, 0)) * w1(dig(i, 1)) * (D == 3 ? w1(dig(i, 2)) : 1.0);
}
template <int D>
__host__ __device__ constexpr double iwq(int i) {  // exact: products of 1.5 and 6
  return iw1(dig(i, 0)) * iw1(dig(i, 1)) * (D == 3 ? iw1(dig(i, 2)) : 1.0);
}

// ---- storage codecs ---------------------------------------------------------
template <int S>
struct Store;
template <>
struct Store<LBM_F64> {
  using type = double;
  using calc = double;
};
template <>
struct Store<LBM_F32> {
  using type = float;
  using calc = float;
};
template <>
struct Store<LBM_F16> {
  using type = __half;
  using calc = float;
};
template <>
struct Store<LBM_BF16> {
  using type = __nv_bfloat16;
  using calc = float;
};

template <int S, int D>
__device__ __forceinline__ typename Store<S>::calc decode(typename Store<S>::type s, int i) {
  if constexpr (S == LBM_F64 || S == LBM_F32) {
    return s;
  } else if constexpr (S == LBM_F16) {
    return __half2float(s) * (float)wq<D>(i);
  } else {
    return __bfloat162float(s) * (float)wq<D>(i);
  }
}

template <int S, int D>
__device__ __forceinline__ typename Store<S>::type encode(typename Store<S>::calc v, int i) {
  if constexpr (S == LBM_F64 || S == LBM_F32) {
    return v;
  } else if constexpr (S == LBM_F16) {
    return __float2half_rn(v * (float)iwq<D>(i));
  } else {
    return __float2bfloat16_rn(v * (float)iwq<D>(i));
  }
}

// ---- collision --------------------------------------------------------------
// Written once for every compute type T: float, double, or f2 (two nodes per
// thread in packed FP32x2 arithmetic).  Per-axis triplet transforms act on
// v[Q] in place; axis d pairs indices (b, b + 3^d, b + 2 * 3^d) for every b
// whose digit d is 0.  All branches on moment indices resolve at compile time.

// populations (e = -1, 0, +1) -> raw moments (M0, M1, M2) = (sum, sum e, sum e^2)
template <typename T, int D>
__device__ __forceinline__ void pops_to_raw(T (&v)[qof<D>()]) {
#pragma unroll
  for (int d = 0; d < D; ++d) {
#pragma unroll
    for (int b = 0; b < qof<D>(); ++b) {
      if (dig(b, d) != 0) continue;
      const int s = p3(d);
      const T fm = v[b], f0 = v[b + s], fp = v[b + 2 * s];
      const T sum = fm + fp;
      v[b] = sum + f0;
      v[b + s] = fp - fm;
      v[b + 2 * s] = sum;
    }
  }
}

// raw moments -> central moments about u (binomial transform, Appendix Eq. trans-a):
// k1 = m1 - u m0, k2 = m2 - 2 u m1 + u^2 m0 = m2 - u (m1 + k1).  nu = -u.
template <typename T, int D>
__device__ __forceinline__ void raw_to_central(T (&v)[qof<D>()], const T (&nu)[D]) {
#pragma unroll
  for (int d = 0; d < D; ++d) {
#pragma unroll
    for (int b = 0; b < qof<D>(); ++b) {
      if (dig(b, d) != 0) continue;
      const int s = p3(d);
      const T m0 = v[b], m1 = v[b + s], m2 = v[b + 2 * s];
      const T k1 = fma_(nu[d], m0, m1);
      v[b + s] = k1;
      v[b + 2 * s] = fma_(nu[d], m1 + k1, m2);
    }
  }
}

// central moments about u -> raw moments: m1 = k1 + u k0, m2 = k2 + u (k1 + m1)
template <typename T, int D>
__device__ __forceinline__ void central_to_raw(T (&v)[qof<D>()], const T (&u)[D]) {
#pragma unroll
  for (int d = 0; d < D; ++d) {
#pragma unroll
    for (int b = 0; b < qof<D>(); ++b) {
      if (dig(b, d) != 0) continue;
      const int s = p3(d);
      const T k0 = v[b], k1 = v[b + s], k2 = v[b + 2 * s];
      const T m1 = fma_(u[d], k0, k1);
      v[b + s] = m1;
      v[b + 2 * s] = fma_(u[d], k1 + m1, k2);
    }
  }
}

// raw moments -> populations: f(-1) = (M2 - M1)/2, f(0) = M0 - M2, f(+1) = (M2 + M1)/2
template <typename T, int D>
__device__ __forceinline__ void raw_to_pops(T (&v)[qof<D>()]) {
  const T half = cst<T>(0.5), mhalf = cst<T>(-0.5);
#pragma unroll
  for (int d = 0; d < D; ++d) {
#pragma unroll
    for (int b = 0; b < qof<D>(); ++b) {
      if (dig(b, d) != 0) continue;
      const int s = p3(d);
      const T m0 = v[b], m1 = v[b + s], m2 = v[b + 2 * s];
      const T h = half * m2;
      v[b] = fma_(m1, mhalf, h);
      v[b + s] = m0 - m2;
      v[b + 2 * s] = fma_(m1, half, h);
    }
  }
}

// Per-node velocity terms used by the equilibrium deviation.
template <typename T, int D>
struct Vel {
  T u[D], nu[D], usq[D], nusq[D], kk2[D];  // u, -u, u^2, -u^2, 1/3 + u^2
};

// Dev_a = rho prod_d m_{alpha_d} - prod_d k_{alpha_d}(u_d): the equilibrium
// central moment minus the central moment of the weights (one-axis factors
// m = (1, 0, 1/3), k(u) = (1, -u, 1/3 + u^2)), in closed forms that never
// subtract nearly equal large terms:
//   some alpha_d = 1:  Dev = -prod_{alpha_d=1} (-u_d) prod_{alpha_d=2} (1/3 + u_d^2)
//   otherwise, with a_d = u_d^2 over the n2 axes with alpha_d = 2:
//     n2 = 0: drho;  n2 = 1: drho/3 - a;  n2 = 2: drho/9 - (a + b)/3 - ab;
//     n2 = 3: drho/27 - (a + b + c)/9 - (ab + ac + bc)/3 - abc.
template <typename T, int D>
__device__ __forceinline__ T eq_deviation(int a, T drho, const Vel<T, D>& w) {
  int n1 = 0, n2 = 0, i2[3] = {0, 0, 0};
#pragma unroll
  for (int d = 0; d < D; ++d) {
    if (dig(a, d) == 1) ++n1;
    if (dig(a, d) == 2) i2[n2++] = d;
  }
  if (n1 > 0) {
    T p = drho;  // placeholder, overwritten by the first factor
    bool have = false, first1 = true;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const int al = dig(a, d);
      if (al == 0) continue;
      T fac;
      if (al == 1) {
        // an even number of (-u) factors needs one extra sign: use -u once
        fac = (first1 && (n1 % 2 == 0)) ? w.nu[d] : w.u[d];
        first1 = false;
      } else {
        fac = w.kk2[d];
      }
      p = have ? p * fac : fac;
      have = true;
    }
    return p;
  }
  if (n2 == 0) return drho;
  if (n2 == 1) return fma_(drho, cst<T>(1.0 / 3.0), w.nusq[i2[0]]);
  if (n2 == 2) {
    const T s = w.usq[i2[0]] + w.usq[i2[1]];
    const T t = fma_(s, cst<T>(-1.0 / 3.0), drho * cst<T>(1.0 / 9.0));
    return fma_(w.nusq[i2[0]], w.usq[i2[1]], t);
  }
  const T a0 = w.usq[0], a1 = w.usq[1], a2 = w.usq[2];
  const T p01 = a0 * a1;
  const T e1 = a0 + a1 + a2;
  const T e2 = fma_(a2, a0 + a1, p01);
  T t = fma_(e1, cst<T>(-1.0 / 9.0), drho * cst<T>(1.0 / 27.0));
  t = fma_(e2, cst<T>(-1.0 / 3.0), t);
  return fma_(p01, w.nusq[2], t);
}

// CM-MRT collision of one node (or node pair) in deviation form.  v holds
// f_i - w_i on entry and f*_i - w_i on exit.  With kappa = central moments of f
// about u, kappa_w those of the weights and kappa_eq = rho prod m, Eq. omega
// gives kappa* = kappa_eq + (1 - omega_n)(kappa - kappa_eq), so
//   kappa* - kappa_w = K + omega_n (Dev - K),
// K = central moments of (f - w), Dev = kappa_eq - kappa_w.  Orders 0 and 1 are
// left unchanged.  Returns false when a node is unphysical (rho <= 0, |u| >= 1,
// NaN).
// The node's conserved moments as the collision computes them: drho = sum (f - w),
// j_d = sum (f - w) e_d (the same on both sides of the collision).
template <typename T, int D>
struct NodeMoments {
  T drho, j[D];
};

template <typename T, int D, bool MOM = false>
__device__ __forceinline__ bool collide(T (&v)[qof<D>()], const T (&om)[2 * D + 1],
                                        NodeMoments<T, D>* mom = nullptr) {
  pops_to_raw<T, D>(v);
  const T drho = v[0];
  if constexpr (MOM) {
    mom->drho = drho;
#pragma unroll
    for (int d = 0; d < D; ++d) mom->j[d] = v[p3(d)];
  }
  const T rho = cst<T>(1.0) + drho;
  const T irho = rcp_(rho);
  Vel<T, D> w;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    w.u[d] = v[p3(d)] * irho;
    w.nu[d] = neg_(w.u[d]);
    w.usq[d] = w.u[d] * w.u[d];
    w.nusq[d] = neg_sq(w.nu[d], w.u[d], w.usq[d]);
    w.kk2[d] = w.usq[d] + cst<T>(1.0 / 3.0);
  }
  raw_to_central<T, D>(v, w.nu);
#pragma unroll
  for (int a = 0; a < qof<D>(); ++a) {
    const int n = order_of<D>(a);
    if (n <= 1) continue;
    const T dev = eq_deviation<T, D>(a, drho, w);
    v[a] = fma_(om[n], dev - v[a], v[a]);
  }
  central_to_raw<T, D>(v, w.u);
  raw_to_pops<T, D>(v);
  T usq = w.usq[0];
#pragma unroll
  for (int d = 1; d < D; ++d) usq = usq + w.usq[d];
  return sane(rho, usq);
}

// Equilibrium deviation f_eq_i - w_i of (rho, u): its central moments about u
// minus the weights' are exactly Dev_a for every a.
template <typename T, int D>
__device__ __forceinline__ void equilibrium(T (&v)[qof<D>()], T drho, const T (&u)[D]) {
  Vel<T, D> w;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    w.u[d] = u[d];
    w.nu[d] = cst<T>(0.0) - u[d];
    w.usq[d] = u[d] * u[d];
    w.nusq[d] = w.nu[d] * u[d];
    w.kk2[d] = w.usq[d] + cst<T>(1.0 / 3.0);
  }
#pragma unroll
  for (int a = 0; a < qof<D>(); ++a) v[a] = eq_deviation<T, D>(a, drho, w);
  central_to_raw<T, D>(v, w.u);
  raw_to_pops<T, D>(v);
}

// ---- AA-pattern addressing ---------------------------------------------------
// Even state (after an even number of steps): f_i(x) is in slot (x, i).
// Odd state: f_i(x) is in slot (x - e_i, opp(i)).  Neighbour node of x along
// velocity j: nb_j = x + e_j (periodic).  In the odd state population opp(j) of
// node x is found in slot (nb_j, j), and a sweep writes its result for
// population j to the same slot (nb_j, j): each node reads and writes one set.
struct Grid {
  int nx, ny, nz;
  int64_t N;
};

template <int D>
__device__ __forceinline__ uint32_t neighbour(const Grid& g, int x, int y, int z, int j) {
  const int ex = dig(j, 0) - 1, ey = dig(j, 1) - 1;
  int xn = x + ex, yn = y + ey;
  xn = xn < 0 ? g.nx - 1 : (xn >= g.nx ? 0 : xn);
  yn = yn < 0 ? g.ny - 1 : (yn >= g.ny ? 0 : yn);
  int zn = z;
  if (D == 3) {
    const int ez = dig(j, 2) - 1;
    zn = z + ez;
    zn = zn < 0 ? g.nz - 1 : (zn >= g.nz ? 0 : zn);
  }
  return (uint32_t)xn + (uint32_t)g.nx * ((uint32_t)yn + (uint32_t)g.ny * (uint32_t)zn);
}

// Read the populations (deviations) of node (x, y, z) in the given state parity.
template <int D, int S>
__device__ __forceinline__ void gather(const typename Store<S>::type* __restrict__ f, const Grid& g,
                                       int x, int y, int z, int odd,
                                       typename Store<S>::calc (&v)[qof<D>()]) {
  const uint32_t node = (uint32_t)x + (uint32_t)g.nx * ((uint32_t)y + (uint32_t)g.ny * (uint32_t)z);
  if (!odd) {
#pragma unroll
    for (int j = 0; j < qof<D>(); ++j) v[j] = decode<S, D>(f[(size_t)j * g.N + node], j);
  } else {
#pragma unroll
    for (int j = 0; j < qof<D>(); ++j)
      v[opp<D>(j)] = decode<S, D>(f[(size_t)j * g.N + neighbour<D>(g, x, y, z, j)], j);
  }
}

// Write populations (deviations) of node (x, y, z) in the given state parity.
template <int D, int S>
__device__ __forceinline__ void scatter(typename Store<S>::type* __restrict__ f, const Grid& g, int x,
                                        int y, int z, int odd,
                                        const typename Store<S>::calc (&v)[qof<D>()]) {
  const uint32_t node = (uint32_t)x + (uint32_t)g.nx * ((uint32_t)y + (uint32_t)g.ny * (uint32_t)z);
  if (!odd) {
#pragma unroll
    for (int j = 0; j < qof<D>(); ++j) f[(size_t)j * g.N + node] = encode<S, D>(v[j], j);
  } else {
#pragma unroll
    for (int j = 0; j < qof<D>(); ++j)
      f[(size_t)j * g.N + neighbour<D>(g, x, y, z, j)] = encode<S, D>(v[opp<D>(j)], j);
  }
}

}  // namespace tp
}  // namespace lbm
