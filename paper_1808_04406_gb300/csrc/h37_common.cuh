// Device building blocks for the 37-velocity degree-9 lattice (Hermite
// projection order N = 4, equilibrium order M = 4): Hermite constants, the
// CM-MRT collision of Sec. II.C in Hermite coefficients, and the AA addressing.
//
// Hermite coefficients are kept as the 15 independent components of the
// symmetric tensors a^(n), n <= 4: component (p, q) has p x-indices and q
// y-indices, index cidx(p, q) = n(n+1)/2 + (n - p).  The tensor Hermite
// polynomial component is He_p(xi_x) He_q(xi_y), and (1/n!) a^(n) : H^(n)
// = sum_(p,q) a_(p,q) He_p He_q / (p! q!) (Eqs. an, fi).
#pragma once

#include <type_traits>

#include "d2q37_lattice.cuh"
#include "f32x2.cuh"
#include "lbm_internal.cuh"

namespace lbm {
namespace h37 {

constexpr int kNC = 15;
__host__ __device__ constexpr int cidx(int p, int q) { return (p + q) * (p + q + 1) / 2 + q; }
__host__ __device__ constexpr int cp(int c) {  // p of component c
  return c == 0 ? 0 : c < 3 ? 2 - c : c < 6 ? 5 - c : c < 10 ? 9 - c : 14 - c;
}
__host__ __device__ constexpr int cq(int c) {
  return c == 0 ? 0 : c < 3 ? c - 1 : c < 6 ? c - 3 : c < 10 ? c - 6 : c - 10;
}
__host__ __device__ constexpr int corder(int c) { return cp(c) + cq(c); }
__host__ __device__ constexpr double he(int n, double x) {  // probabilists' Hermite
  return n == 0 ? 1.0 : n == 1 ? x : n == 2 ? x * x - 1.0 : n == 3 ? x * x * x - 3.0 * x
                                                          : x * x * x * x - 6.0 * x * x + 3.0;
}
__host__ __device__ constexpr double fct(int n) { return n <= 1 ? 1.0 : n == 2 ? 2.0 : n == 3 ? 6.0 : 24.0; }
// He_p(xi_x) He_q(xi_y) at velocity i
__host__ __device__ constexpr double hval(int i, int c) {
  return he(cp(c), kC * ex_of(i)) * he(cq(c), kC * ey_of(i));
}
// reconstruction weight w_i He_p He_q / (p! q!)
__host__ __device__ constexpr double rval(int i, int c) {
  return w_of(i) * hval(i, c) / (fct(cp(c)) * fct(cq(c)));
}
__host__ __device__ constexpr int opp(int i) { return kQ - 1 - i; }
constexpr int kHalf = 18;  // velocities 0..17 pair with 36..19; 18 is the rest velocity

// Model flags (mirror include/lbm.h)
struct Model {
  int thermal;   // theta from the moments (else theta = 1)
  int raw;       // absolute-frame relaxation of each Hermite order (Sec. II.B MRT)
  float kfac;    // 4th-order coupling K / 6 (1 for K = 6, 12 for the printed 72)
  double eps_ref;  // theta_ref - 1: the offsets are taken from f_eq(1, 0, theta_ref)
  int sround;      // stochastic rounding of FP16 / BF16 stores
  uint32_t seed;   // per-step seed of the rounding bits
};

// ---- stochastic rounding of FP16 / BF16 stores ----
// Random bits per node: a 32-bit integer avalanche hash of (node, step seed)
// starts a linear congruential stream (multiplier 747796405, increment
// 2891336453, modulus 2^32) that gives one value per stored population; only
// its high bits are used.
__device__ __forceinline__ uint32_t hash32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}
struct SrStream {
  uint32_t s;
  __device__ __forceinline__ SrStream(uint32_t seed, uint32_t node) : s(hash32(seed ^ (node * 0x9E3779B9u))) {}
  __device__ __forceinline__ uint32_t next() {
    s = s * 747796405u + 2891336453u;
    return s;
  }
};
// Add `drop` random bits below the kept mantissa (13 for FP16, 16 for BF16); a
// conversion toward zero then rounds up in magnitude with probability equal to
// the dropped fraction.
__device__ __forceinline__ float dither(float x, uint32_t r, int drop) {
  return __uint_as_float(__float_as_uint(x) + (r >> (32 - drop)));
}
__device__ __forceinline__ uint32_t sr_f16x2(float lo, float hi, uint32_t rlo, uint32_t rhi) {
  uint32_t d;
  asm("cvt.rz.f16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(dither(hi, rhi, 13)), "f"(dither(lo, rlo, 13)));
  return d;
}
__device__ __forceinline__ uint32_t sr_bf16x2(float lo, float hi, uint32_t rlo, uint32_t rhi) {
  uint32_t d;
  asm("cvt.rz.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(dither(hi, rhi, 16)), "f"(dither(lo, rlo, 16)));
  return d;
}

// Hermite coefficients of the reference state f_eq(rho = 1, u = 0, theta_ref):
// the one-axis forms g_0 = 1, g_2 = eps, g_4 = 3 eps^2 multiplied per axis.
template <typename T>
__device__ __forceinline__ T aref(int c, T eps) {
  const int p = cp(c), q = cq(c);
  if ((p & 1) || (q & 1)) return T(0);
  auto g = [&](int n) -> T { return n == 0 ? T(1) : n == 2 ? eps : T(3) * eps * eps; };
  return g(p) * g(q);
}

// 15 Hermite coefficients of the offsets v (37 values), using +- pairs.
template <typename T>
__device__ __forceinline__ void to_hermite(const T (&v)[kQ], T (&a)[kNC]) {
  T sp[kHalf], dm[kHalf];
#pragma unroll
  for (int i = 0; i < kHalf; ++i) {
    sp[i] = v[i] + v[opp(i)];
    dm[i] = v[i] - v[opp(i)];
  }
#pragma unroll
  for (int c = 0; c < kNC; ++c) {
    const bool even = (corder(c) & 1) == 0;
    T s = even ? v[kHalf] * cst<T>(hval(kHalf, c)) : cst<T>(0.0);
#pragma unroll
    for (int i = 0; i < kHalf; ++i) {
      const double h = hval(i, c);
      if (h != 0.0) s = fma_(even ? sp[i] : dm[i], cst<T>(h), s);
    }
    a[c] = s;
  }
}

// offsets from 15 coefficients: v_i = sum_c a_c w_i He_p He_q / (p! q!)
template <typename T>
__device__ __forceinline__ void from_hermite(const T (&a)[kNC], T (&v)[kQ]) {
  T rest = cst<T>(0.0);
#pragma unroll
  for (int c = 0; c < kNC; ++c)
    if ((corder(c) & 1) == 0 && rval(kHalf, c) != 0.0) rest = fma_(a[c], cst<T>(rval(kHalf, c)), rest);
  v[kHalf] = rest;
#pragma unroll
  for (int i = 0; i < kHalf; ++i) {
    T ev = cst<T>(0.0), od = cst<T>(0.0);
#pragma unroll
    for (int c = 0; c < kNC; ++c) {
      const double r = rval(i, c);
      if (r == 0.0) continue;
      if ((corder(c) & 1) == 0)
        ev = fma_(a[c], cst<T>(r), ev);
      else
        od = fma_(a[c], cst<T>(r), od);
    }
    v[i] = ev + od;
    v[opp(i)] = ev - od;
  }
}

// ---- correctly rounded transforms (FP32 storage) ----------------------------
// In FP32 both transforms drift: the constants He_p He_q and w_i He_p He_q /
// (p! q!) round to FP32, so the two tables are not exact inverses (the momentum
// row of the round trip is off by ~8e-9 per step), and the 15 - 19 term sums
// round at every addition.  Each error is below an ulp, but it recurs at every
// step on a slowly varying state and the conserved moments accumulate it
// linearly (1e-5 relative on the velocity after 1000 steps).  These versions
// compute each coefficient and each offset as if in twice the working precision
// and round once: every constant is carried as an FP32 pair hi + lo, every
// product's rounding error is recovered with an FMA and every partial sum's
// with Knuth's two-sum, and the errors are summed in a second accumulator (the
// compensated dot product of Ogita, Rump and Oishi, SIAM J. Sci. Comput. 26,
// 2005).  About 11 flops per term instead of 1.

// s + c += x (hh + hl)
__device__ __forceinline__ void dot2_add_split(float& s, float& c, float x, float hh, float hl) {
  const float p = x * hh;
  const float t = s + p;
  const float z = t - s;
  const float es = (s - (t - z)) + (p - z);
  s = t;
  c = c + __fmaf_rn(x, hl, __fmaf_rn(x, hh, -p) + es);
}
// s + c += x h, h given in FP64 (a compile-time constant here) and split into hi + lo
__device__ __forceinline__ void dot2_add(float& s, float& c, float x, double h) {
  const float hh = (float)h;
  dot2_add_split(s, c, x, hh, (float)(h - (double)hh));
}
// a + b = s + e exactly
__device__ __forceinline__ float two_sum_err(float a, float b, float s) {
  const float z = s - a;
  return (a - (s - z)) + (b - z);
}

__device__ __forceinline__ void to_hermite_exact(const float (&v)[kQ], float (&a)[kNC]) {
  float sp[kHalf], dm[kHalf], spe[kHalf], dme[kHalf];
#pragma unroll
  for (int i = 0; i < kHalf; ++i) {
    sp[i] = v[i] + v[opp(i)];
    dm[i] = v[i] - v[opp(i)];
    spe[i] = two_sum_err(v[i], v[opp(i)], sp[i]);
    dme[i] = two_sum_err(v[i], -v[opp(i)], dm[i]);
  }
#pragma unroll
  for (int c = 0; c < kNC; ++c) {
    const bool even = (corder(c) & 1) == 0;
    float s = 0.f, cc = 0.f;
    if (even) dot2_add(s, cc, v[kHalf], hval(kHalf, c));
#pragma unroll
    for (int i = 0; i < kHalf; ++i) {
      const double h = hval(i, c);
      if (h == 0.0) continue;
      dot2_add(s, cc, even ? sp[i] : dm[i], h);
      cc = __fmaf_rn(even ? spe[i] : dme[i], (float)h, cc);  // the pair sum's own rounding
    }
    a[c] = s + cc;
  }
}

__device__ __forceinline__ void from_hermite_exact(const float (&a)[kNC], float (&v)[kQ]) {
  {
    float s = 0.f, cc = 0.f;
#pragma unroll
    for (int c = 0; c < kNC; ++c)
      if ((corder(c) & 1) == 0 && rval(kHalf, c) != 0.0) dot2_add(s, cc, a[c], rval(kHalf, c));
    v[kHalf] = s + cc;
  }
#pragma unroll
  for (int i = 0; i < kHalf; ++i) {
    float ev = 0.f, evc = 0.f, od = 0.f, odc = 0.f;
#pragma unroll
    for (int c = 0; c < kNC; ++c) {
      const double r = rval(i, c);
      if (r == 0.0) continue;
      if ((corder(c) & 1) == 0)
        dot2_add(ev, evc, a[c], r);
      else
        dot2_add(od, odc, a[c], r);
    }
    // v_i, v_opp(i) = (ev + evc) +- (od + odc), the corrections folded in before the last rounding
    const float t1 = ev + od, t2 = ev - od;
    v[i] = t1 + (two_sum_err(ev, od, t1) + (evc + odc));
    v[opp(i)] = t2 + (two_sum_err(ev, -od, t2) + (evc - odc));
  }
}

// rho > 0, theta = 1 + eps > 0 and |u|^2 < 4 (Hermite units), for every node held.
__device__ __forceinline__ bool physical(float rho, float eps, float usq) {
  return rho > 0.f && 1.f + eps > 0.f && usq < 4.f;
}
__device__ __forceinline__ bool physical(double rho, double eps, double usq) {
  return rho > 0.0 && 1.0 + eps > 0.0 && usq < 4.0;
}
__device__ __forceinline__ bool physical(f2 rho, f2 eps, f2 usq) {
  float r0, r1, e0, e1, u0, u1;
  unpack2(rho, r0, r1);
  unpack2(eps, e0, e1);
  unpack2(usq, u0, u1);
  return physical(r0, e0, u0) && physical(r1, e1, u1);
}

// Equilibrium coefficients a_0 (Maxwellian of rho, u, theta = 1 + eps, Hermite
// units) per component: rho g_p(u_x) g_q(u_y), g_0 = 1, g_1 = u, g_2 = u^2 + eps,
// g_3 = u^3 + 3 eps u, g_4 = u^4 + 6 eps u^2 + 3 eps^2.
template <typename T>
__device__ __forceinline__ void g_forms(T u, T eps, T (&g)[5]) {
  const T u2 = u * u;
  g[0] = cst<T>(1.0);
  g[1] = u;
  g[2] = u2 + eps;
  g[3] = u * (u2 + cst<T>(3.0) * eps);
  g[4] = fma_(u2, u2 + cst<T>(6.0) * eps, cst<T>(3.0) * eps * eps);
}

// The same forms split as g_n(u, eps) = g_n(0, eps_r) + dg_n with eps = eps_r + de,
// the increments dg_n written without subtracting nearly equal terms:
// dg_0 = 0, dg_1 = u, dg_2 = u^2 + de, dg_3 = g_3, dg_4 = u^2 (u^2 + 6 eps) + 3 de (eps + eps_r).
template <typename T>
__device__ __forceinline__ void g_increments(T u, T eps, T de, T er, T (&dg)[5]) {
  const T u2 = u * u;
  dg[0] = cst<T>(0.0);
  dg[1] = u;
  dg[2] = u2 + de;
  dg[3] = u * (u2 + cst<T>(3.0) * eps);
  dg[4] = fma_(u2, u2 + cst<T>(6.0) * eps, cst<T>(3.0) * de * (eps + er));
}

// [sum over the 3 (resp. 4) placements of u next to a rank-2 (resp. 3) tensor]
// at component (p, q): p u_x A_(p-1,q) + q u_y A_(p,q-1)
template <typename T, int NC>
__device__ __forceinline__ T shift1(const T (&A)[NC], int p, int q, T ux, T uy) {
  T s = cst<T>(0.0);
  if (p > 0) s = fma_(cst<T>(p) * ux, A[cidx(p - 1, q)], s);
  if (q > 0) s = fma_(cst<T>(q) * uy, A[cidx(p, q - 1)], s);
  return s;
}
// [sum over the 6 placements of u u next to a rank-2 tensor] at (p, q)
template <typename T, int NC>
__device__ __forceinline__ T shift2(const T (&A)[NC], int p, int q, T ux, T uy) {
  T s = cst<T>(0.0);
  if (p > 1) s = fma_(cst<T>(p * (p - 1) / 2) * ux * ux, A[cidx(p - 2, q)], s);
  if (p > 0 && q > 0) s = fma_(cst<T>(p * q) * ux * uy, A[cidx(p - 1, q - 1)], s);
  if (q > 1) s = fma_(cst<T>(q * (q - 1) / 2) * uy * uy, A[cidx(p, q - 2)], s);
  return s;
}
// [sum over the 6 placements of delta next to a rank-2 tensor] at (p, q)
template <typename T, int NC>
__device__ __forceinline__ T delta2(const T (&A)[NC], int p, int q) {
  T s = cst<T>(0.0);
  if (p > 1) s = s + cst<T>(p * (p - 1) / 2) * A[cidx(p - 2, q)];
  if (q > 1) s = s + cst<T>(q * (q - 1) / 2) * A[cidx(p, q - 2)];
  return s;
}

// The collision in Hermite space.  da: the NC (15 for N = 4, 10 for N = 3)
// Hermite coefficients of the offsets f - f_ref in, of the post-collision
// offsets out.  om[n]: rates of orders 2..4 (order 4 unused for N = 3).
// Returns false for an unphysical node.
template <typename T, int NC>
__device__ __forceinline__ bool collide_coeffs(T (&da)[NC], const T (&om)[5], const Model& m) {
  static_assert(NC == 10 || NC == 15, "Hermite truncation N = 3 or 4");
  const T er = cst<T>(m.eps_ref);
  const T drho = da[0];
  const T rho = cst<T>(1.0) + drho;
  const T irho = rcp_(rho);
  const T ux = da[cidx(1, 0)] * irho, uy = da[cidx(0, 1)] * irho;
  const T usq = ux * ux + uy * uy;
  // theta - theta_ref from tr a^(2) = rho (|u|^2 + 2 (theta - 1)), a = a_ref + da:
  // de = ((da_20 + da_02 - 2 eps_r drho) / rho - |u|^2) / 2
  T de = cst<T>(0.0);
  if (m.thermal)
    de = cst<T>(0.5) * ((da[cidx(2, 0)] + da[cidx(0, 2)] - cst<T>(2.0) * er * drho) * irho - usq);
  else
    de = cst<T>(0.0) - er;  // isothermal: theta = 1
  const T eps = er + de;
  T gx[5], gy[5], dgx[5], dgy[5], grf[5];
  g_forms<T>(ux, eps, gx);
  g_forms<T>(uy, eps, gy);
  g_increments<T>(ux, eps, de, er, dgx);
  g_increments<T>(uy, eps, de, er, dgy);
  g_forms<T>(cst<T>(0.0), er, grf);
  // non-equilibrium coefficients a_1 = a - a_0 = da - (a_0 - a_ref) for orders 2..4, with
  // a_0 - a_ref = drho g_p g_q + dg_p g_q + g_p(0, eps_r) dg_q (no cancellation)
  T a1[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    if (corder(c) < 2) {
      a1[c] = cst<T>(0.0);
      continue;
    }
    const int p = cp(c), q = cq(c);
    T d0 = drho * gx[p] * gy[q];
    if (p != 0) d0 = fma_(dgx[p], gy[q], d0);
    if (q != 0 && !((p & 1) != 0)) d0 = fma_(grf[p], dgy[q], d0);
    a1[c] = da[c] - d0;
  }
  T aO[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) aO[c] = cst<T>(0.0);
  if (m.raw) {
#pragma unroll
    for (int c = 3; c < NC; ++c) aO[c] = cst<T>(0.0) - om[corder(c)] * a1[c];
  } else {
    // relative frame (Eq. trans-s): b2 = a2, b3 = a3 - [3] u b2, b4 = a4 - [4] u a3 + [6] u u a2
    T b[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) b[c] = cst<T>(0.0);
#pragma unroll
    for (int c = 3; c < 6; ++c) b[c] = a1[c];
#pragma unroll
    for (int c = 6; c < 10; ++c) b[c] = a1[c] - shift1<T>(b, cp(c), cq(c), ux, uy);
#pragma unroll
    for (int c = 10; c < NC; ++c)
      b[c] = a1[c] - shift1<T>(a1, cp(c), cq(c), ux, uy) + shift2<T>(a1, cp(c), cq(c), ux, uy);
    // relax each central order (Eq. omega); order 4 carries the delta coupling
    // -K (omega_4 - omega_2) Sym(delta b2), K = 6 kfac
    T bO[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) bO[c] = cst<T>(0.0);
#pragma unroll
    for (int c = 3; c < NC; ++c) bO[c] = cst<T>(0.0) - om[corder(c)] * b[c];
    const T kc = cst<T>(m.kfac) * (om[4] - om[2]);
#pragma unroll
    for (int c = 10; c < NC; ++c) bO[c] = bO[c] - kc * delta2<T>(b, cp(c), cq(c));
    // back to the absolute frame: a2 = b2, a3 = b3 + [3] u b2, a4 = b4 + [4] u b3 + [6] u u b2
#pragma unroll
    for (int c = 3; c < 6; ++c) aO[c] = bO[c];
#pragma unroll
    for (int c = 6; c < 10; ++c) aO[c] = bO[c] + shift1<T>(bO, cp(c), cq(c), ux, uy);
#pragma unroll
    for (int c = 10; c < NC; ++c)
      aO[c] = bO[c] + shift1<T>(bO, cp(c), cq(c), ux, uy) + shift2<T>(bO, cp(c), cq(c), ux, uy);
  }
  // f* = f^ + Omega: its coefficients are a + a_Omega (f^ keeps a for n <= 4)
#pragma unroll
  for (int c = 0; c < NC; ++c) da[c] = da[c] + aO[c];
  return physical(rho, eps, usq);
}

// One node of the 37-velocity lattice.  v: offsets f_i - f_ref,i in,
// post-collision offsets out.  om[n]: rates of orders 2..4.
// EXACT (FP32 only): the correctly rounded transforms above.
template <typename T, bool EXACT = false>
__device__ __forceinline__ bool collide(T (&v)[kQ], const T (&om)[5], const Model& m, T* mom = nullptr) {
  static_assert(!EXACT || std::is_same<T, float>::value, "correctly rounded transforms are FP32");
  T da[kNC];
  if constexpr (EXACT)
    to_hermite_exact(v, da);
  else
    to_hermite<T>(v, da);
  if (mom) {  // the node's conserved moments: drho and j (Hermite units), unchanged by the collision
    mom[0] = da[0];
    mom[1] = da[cidx(1, 0)];
    mom[2] = da[cidx(0, 1)];
  }
  const bool ok = collide_coeffs<T, kNC>(da, om, m);
  if constexpr (EXACT)
    from_hermite_exact(da, v);
  else
    from_hermite<T>(da, v);
  return ok;
}

// Offsets of the equilibrium of (rho, u [Hermite units], theta): coefficients
// a_0 - a_ref reconstructed.
template <typename T>
__device__ __forceinline__ void equilibrium(T (&v)[kQ], T rho, T ux, T uy, T theta, double eps_ref) {
  T gx[5], gy[5];
  const T eps = theta - T(1);
  g_forms<T>(ux, eps, gx);
  g_forms<T>(uy, eps, gy);
  T da[kNC];
#pragma unroll
  for (int c = 0; c < kNC; ++c) da[c] = rho * gx[cp(c)] * gy[cq(c)] - aref<T>(c, (T)eps_ref);
  from_hermite<T>(da, v);
}

// Absolute reference population f_ref,i = f_eq,i(1, 0, theta_ref).
__device__ __forceinline__ double fref(int i, double eps_ref) {
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kNC; ++c) s += aref<double>(c, eps_ref) * rval(i, c);
  return s;
}

// ---- storage codecs: offsets (f - f_ref) for FP64/FP32, (f - f_ref)/w for FP16/BF16 ----
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

template <int S>
__device__ __forceinline__ typename Store<S>::calc decode(typename Store<S>::type s, int i) {
  if constexpr (S == LBM_F64 || S == LBM_F32) {
    return s;
  } else if constexpr (S == LBM_F16) {
    return __half2float(s) * (float)w_of(i);
  } else {
    return __bfloat162float(s) * (float)w_of(i);
  }
}
// Stochastically rounded encode (FP16 / BF16; the other types round as encode).
template <int S>
__device__ __forceinline__ typename Store<S>::type encode_sr(typename Store<S>::calc v, int i, uint32_t r) {
  if constexpr (S == LBM_F64 || S == LBM_F32) {
    return v;
  } else if constexpr (S == LBM_F16) {
    return __float2half_rz(dither(v * (float)(1.0 / w_of(i)), r, 13));
  } else {
    return __float2bfloat16_rz(dither(v * (float)(1.0 / w_of(i)), r, 16));
  }
}

template <int S>
__device__ __forceinline__ typename Store<S>::type encode(typename Store<S>::calc v, int i) {
  if constexpr (S == LBM_F64 || S == LBM_F32) {
    return v;
  } else if constexpr (S == LBM_F16) {
    return __float2half_rn(v * (float)(1.0 / w_of(i)));
  } else {
    return __float2bfloat16_rn(v * (float)(1.0 / w_of(i)));
  }
}

// ---- AA addressing (same convention as the tensor-product lattices) ----
// Even state: f_i(x) in slot (x, i).  Odd state: population opp(j) of node x in
// slot (x + e_j, j).  Requires nx, ny >= 3 (|e| <= 3 wraps once at most).
struct Grid2 {
  int nx, ny;
  int64_t N;
};

__device__ __forceinline__ uint32_t nbr(const Grid2& g, int x, int y, int j) {
  int xn = x + ex_of(j), yn = y + ey_of(j);
  xn = xn < 0 ? xn + g.nx : (xn >= g.nx ? xn - g.nx : xn);
  yn = yn < 0 ? yn + g.ny : (yn >= g.ny ? yn - g.ny : yn);
  return (uint32_t)xn + (uint32_t)g.nx * (uint32_t)yn;
}

template <int S>
__device__ __forceinline__ void gather(const typename Store<S>::type* __restrict__ f, const Grid2& g,
                                       int x, int y, int odd, typename Store<S>::calc (&v)[kQ]) {
  const uint32_t node = (uint32_t)x + (uint32_t)g.nx * (uint32_t)y;
#pragma unroll
  for (int j = 0; j < kQ; ++j) {
    if (!odd)
      v[j] = decode<S>(f[(size_t)j * g.N + node], j);
    else
      v[opp(j)] = decode<S>(f[(size_t)j * g.N + nbr(g, x, y, j)], j);
  }
}

template <int S>
__device__ __forceinline__ void scatter(typename Store<S>::type* __restrict__ f, const Grid2& g, int x,
                                        int y, int odd, const typename Store<S>::calc (&v)[kQ]) {
  const uint32_t node = (uint32_t)x + (uint32_t)g.nx * (uint32_t)y;
#pragma unroll
  for (int j = 0; j < kQ; ++j) {
    if (!odd)
      f[(size_t)j * g.N + node] = encode<S>(v[j], j);
    else
      f[(size_t)j * g.N + nbr(g, x, y, j)] = encode<S>(v[opp(j)], j);
  }
}

}  // namespace h37
}  // namespace lbm
