// Learned relaxation-rate closure for D3Q27 CM-MRT.
//
// Every central-moment rate above the second order is free in the paper's
// model (Sec. II.C after Eq. omega: each central moment relaxes at its own rate;
// only omega_2 and omega_3 set the transport coefficients).  Here a 20 -> 64 ->
// 64 -> 6 network (BF16 weights, FP32 accumulation, mma.sync tensor cores)
// chooses, per node, the rates of six classes of orders 3..6 from the node's
// non-equilibrium central moments:
//   classes 3:(2,1,0), 3:(1,1,1), 4:(2,2,0), 4:(2,1,1), 5:(2,2,1), 6:(2,2,2)
// (permutation classes of alpha), omega = 2 sigmoid(z).
//
// Training data come from the solver itself: fine populations are box-filtered
// onto a grid m times coarser (acoustic scaling); two filtered states one coarse
// step apart give, per coarse node, the features (19 non-equilibrium central
// moments of orders 2..4 divided by rho c_s^n, and tau_2 - 1/2, standardised)
// and the a-priori targets: the post-collision non-equilibrium moments k1* of
// the arriving populations pulled back along their velocity.  The loss per
// sample is sum_c cw_c sum_{alpha in c} ((1 - omega_c) k1 - k1*)^2, kept as
// A = sum k1^2, B = sum k1 k1*, C = sum k1*^2 per class.
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "lbm_internal.cuh"
#include "mlp.cuh"
#include "sweep_body.cuh"
#include "tc05.cuh"
#include "tp_common.cuh"

namespace lbm {
namespace {

using mlp::kH;
using mlp::kIn;
using mlp::kInPad;
using mlp::kOut;
using mlp::kOutPad;
using mlp::kParams;
constexpr int kParamsPad = 5904;  // kParams rounded up to 16, + 1 slot for the loss

// class of a D3Q27 moment index (orders 3..6), -1 otherwise
__host__ __device__ constexpr int class_of(int a) {
  return tp::order_of<3>(a) < 3 ? -1
         : tp::order_of<3>(a) == 3
             ? ((tp::dig(a, 0) == 1 && tp::dig(a, 1) == 1 && tp::dig(a, 2) == 1) ? 1 : 0)
         : tp::order_of<3>(a) == 4
             ? ((tp::dig(a, 0) == 1 || tp::dig(a, 1) == 1 || tp::dig(a, 2) == 1) ? 3 : 2)
         : tp::order_of<3>(a) == 5 ? 4
                                   : 5;
}
// 3^(n/2): 1 / c_s^n
__host__ __device__ constexpr double inv_cs_pow(int n) {
  return n == 2 ? 3.0 : n == 3 ? 5.196152422706632 : n == 4 ? 9.0 : n == 5 ? 15.588457268119896 : 27.0;
}

// ---- box filter -------------------------------------------------------------
template <int S>
__global__ void filter_kernel(const typename tp::Store<S>::type* __restrict__ f, tp::Grid g, int odd, int m,
                              int ncx, int ncy, int ncz, float* __restrict__ out) {
  using T = typename tp::Store<S>::calc;
  const int64_t Nc = (int64_t)ncx * ncy * ncz;
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= Nc) return;
  const int X = (int)(k % ncx), Y = (int)((k / ncx) % ncy), Z = (int)(k / ((int64_t)ncx * ncy));
  double acc[27];
#pragma unroll
  for (int i = 0; i < 27; ++i) acc[i] = 0.0;
  for (int c = 0; c < m; ++c)
    for (int b = 0; b < m; ++b)
      for (int a = 0; a < m; ++a) {
        T v[27];
        tp::gather<3, S>(f, g, m * X + a, m * Y + b, m * Z + c, odd, v);
#pragma unroll
        for (int i = 0; i < 27; ++i) acc[i] += (double)v[i];
      }
  const double inv = 1.0 / ((double)m * m * m);
#pragma unroll
  for (int i = 0; i < 27; ++i) out[(size_t)i * Nc + k] = (float)(acc[i] * inv);
}

// ---- a-priori dataset -------------------------------------------------------
// central moments of offsets v (27, natural layout) about the node velocity of
// the first state: K (in place), drho, Vel.
__device__ __forceinline__ void central_of(float (&v)[27], float& drho, tp::Vel<float, 3>& w, bool set_u) {
  tp::pops_to_raw<float, 3>(v);
  if (set_u) {
    drho = v[0];
    const float irho = 1.0f / (1.0f + drho);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      w.u[d] = v[tp::p3(d)] * irho;
      w.nu[d] = -w.u[d];
      w.usq[d] = w.u[d] * w.u[d];
      w.nusq[d] = -w.usq[d];
      w.kk2[d] = w.usq[d] + (1.0f / 3.0f);
    }
  }
  tp::raw_to_central<float, 3>(v, w.nu);
}

struct Norm {
  float mean[kIn], inv_std[kIn];
};

__global__ void dataset_kernel(const float* __restrict__ ft, const float* __restrict__ ft1, int nx, int ny, int nz,
                               float tau2, const float* __restrict__ norm, float* __restrict__ X,
                               float* __restrict__ abc) {
  const int64_t N = (int64_t)nx * ny * nz;
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  const int x = (int)(k % nx), y = (int)((k / nx) % ny), z = (int)(k / ((int64_t)nx * ny));
  float v[27], s[27];
#pragma unroll
  for (int i = 0; i < 27; ++i) v[i] = ft[(size_t)i * N + k];
  // pulled-back post-collision state: s_i(x) = f_{t+1, i}(x + e_i)
#pragma unroll
  for (int i = 0; i < 27; ++i) {
    int xn = x + tp::dig(i, 0) - 1, yn = y + tp::dig(i, 1) - 1, zn = z + tp::dig(i, 2) - 1;
    xn = xn < 0 ? nx - 1 : (xn >= nx ? 0 : xn);
    yn = yn < 0 ? ny - 1 : (yn >= ny ? 0 : yn);
    zn = zn < 0 ? nz - 1 : (zn >= nz ? 0 : zn);
    s[i] = ft1[(size_t)i * N + xn + (int64_t)nx * (yn + (int64_t)ny * zn)];
  }
  float drho, drho_s;
  tp::Vel<float, 3> w, ws;
  central_of(v, drho, w, true);
  central_of(s, drho_s, ws, true);  // the post-collision state in its own frame
  const float irho = 1.0f / (1.0f + drho);
  const float irho_s = 1.0f / (1.0f + drho_s);
  float feat[kIn];
  float A[kOut], B[kOut], C[kOut];
#pragma unroll
  for (int c = 0; c < kOut; ++c) A[c] = B[c] = C[c] = 0.0f;
  int fi = 0;
#pragma unroll
  for (int a = 0; a < 27; ++a) {
    const int n = tp::order_of<3>(a);
    if (n < 2) continue;
    const float k1 = (v[a] - tp::eq_deviation<float, 3>(a, drho, w)) * (float)inv_cs_pow(n) * irho;
    const float k1s = (s[a] - tp::eq_deviation<float, 3>(a, drho_s, ws)) * (float)inv_cs_pow(n) * irho_s;
    if (n <= 4) feat[fi++] = k1;
    const int c = class_of(a);
    if (c >= 0) {
      A[c] += k1 * k1;
      B[c] += k1 * k1s;
      C[c] += k1s * k1s;
    }
  }
  feat[19] = tau2 - 0.5f;
#pragma unroll
  for (int j = 0; j < kIn; ++j) X[k * kIn + j] = (feat[j] - norm[j]) * norm[kIn + j];
#pragma unroll
  for (int c = 0; c < kOut; ++c) {
    abc[k * 18 + 3 * c] = A[c];
    abc[k * 18 + 3 * c + 1] = B[c];
    abc[k * 18 + 3 * c + 2] = C[c];
  }
}

// f <- f^eq + s (f - f^eq) per node: every central moment of order >= 2 moves
// to kappa^eq + s (kappa - kappa^eq), i.e. a collision with omega = 1 - s.
__global__ void rescale_kernel(float* __restrict__ f, int64_t N, float scale) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  float v[27];
#pragma unroll
  for (int i = 0; i < 27; ++i) v[i] = f[(size_t)i * N + k];
  float drho;
  tp::Vel<float, 3> w;
  central_of(v, drho, w, true);
#pragma unroll
  for (int a = 0; a < 27; ++a) {
    if (tp::order_of<3>(a) < 2) continue;
    const float dev = tp::eq_deviation<float, 3>(a, drho, w);
    v[a] = fmaf(scale, v[a] - dev, dev);
  }
  tp::central_to_raw<float, 3>(v, w.u);
  tp::raw_to_pops<float, 3>(v);
#pragma unroll
  for (int i = 0; i < 27; ++i) f[(size_t)i * N + k] = v[i];
}

// ---- training ---------------------------------------------------------------
constexpr int kTile = 64;          // samples per block tile (4 warps x 16)
constexpr int kTrainThreads = 128;

struct TrainSmem {
  mlp::FwdW w;
  mlp::BwdW wb;
  __nv_bfloat16 xs[kTile][mlp::kLd1];
  __nv_bfloat16 h1[kTile][kH];
  __nv_bfloat16 h2[kTile][kH];
  __nv_bfloat16 dz1[kTile][kH];
  __nv_bfloat16 dz2[kTile][kH];
  __nv_bfloat16 dz3[kTile][kOutPad];
  float abc[kTile][18];
  float bias[4][kH + kH + kOutPad];
  float loss[4];
};

struct LossArgs {
  float cw[kOut];
  float lo, span;  // omega = lo + span sigmoid(z)
};

__device__ __forceinline__ uint64_t mix64(uint64_t z) {  // splitmix64 finaliser
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// One block: grid-stride over tiles of 64 batch slots; forward, loss, backward
// per warp (16 samples), weight gradients by tensor-core GEMMs over the tile;
// the block's gradient sums go to partials[blockIdx.x][0 .. kParams] (+ loss).
__global__ void __launch_bounds__(kTrainThreads)
    grad_kernel(const float* __restrict__ X, const float* __restrict__ abc, int64_t n, int64_t batch, int random,
                uint64_t seed, uint64_t iter, LossArgs la, const float* __restrict__ P, float* __restrict__ partials) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TrainSmem& sm = *reinterpret_cast<TrainSmem*>(smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  mlp::load_fwd(P, sm.w);
  mlp::load_bwd(P, sm.wb);
  float acc_w2[8][4], acc_w1[4][4], acc_w3[4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int k = 0; k < 4; ++k) acc_w2[i][k] = 0.0f;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int k = 0; k < 4; ++k) acc_w1[i][k] = 0.0f;
#pragma unroll
  for (int k = 0; k < 4; ++k) acc_w3[k] = 0.0f;
  float db1[16], db2[16], db3[2], loss = 0.0f;
#pragma unroll
  for (int i = 0; i < 16; ++i) db1[i] = db2[i] = 0.0f;
  db3[0] = db3[1] = 0.0f;
  const float inv_batch = 1.0f / (float)batch;
  const int64_t ntiles = (batch + kTile - 1) / kTile;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    __syncthreads();  // previous tile's shared data fully consumed
    for (int r = threadIdx.x; r < kTile; r += blockDim.x) {
      const int64_t slot = tile * kTile + r;
      const bool valid = slot < batch;
      int64_t idx = slot;
      if (random) idx = (int64_t)(mix64(seed ^ (iter << 32) ^ (uint64_t)slot) % (uint64_t)n);
      for (int j = 0; j < mlp::kLd1; ++j)
        sm.xs[r][j] = __float2bfloat16_rn(valid && j < kIn ? X[idx * kIn + j] : 0.0f);
      for (int j = 0; j < 18; ++j) sm.abc[r][j] = valid ? abc[idx * 18 + j] : 0.0f;
    }
    __syncthreads();
    const int r0 = warp * 16;
    uint32_t h1a[4][4], h2a[4][4];
    float z3[4];
    mlp::forward16(sm.w, &sm.xs[r0][0], mlp::kLd1, h1a, h2a, z3, &sm.h1[r0][0], &sm.h2[r0][0]);
    // loss and dL/dz3 for rows r0 + g, r0 + g + 8 and classes 2t, 2t + 1
    float dz3[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int row = r0 + g + (q >= 2 ? 8 : 0), c = 2 * t + (q & 1);
      dz3[q] = 0.0f;
      if (c < kOut) {
        const float sg = 1.0f / (1.0f + __expf(-z3[q]));
        const float gm = 1.0f - fmaf(la.span, sg, la.lo);
        const float A = sm.abc[row][3 * c], B = sm.abc[row][3 * c + 1], C = sm.abc[row][3 * c + 2];
        loss += la.cw[c] * (gm * gm * A - 2.0f * gm * B + C);
        const float dom = la.cw[c] * (-2.0f * gm * A + 2.0f * B) * inv_batch;
        dz3[q] = dom * la.span * sg * (1.0f - sg);
      }
    }
    db3[0] += dz3[0] + dz3[2];
    db3[1] += dz3[1] + dz3[3];
    *reinterpret_cast<uint32_t*>(&sm.dz3[r0 + g][2 * t]) = mlp::pack_bf16(dz3[0], dz3[1]);
    *reinterpret_cast<uint32_t*>(&sm.dz3[r0 + g + 8][2 * t]) = mlp::pack_bf16(dz3[2], dz3[3]);
    // dh2 = dz3 W3^T (k = classes, padded 8 -> 16), masked by h2 > 0
    uint32_t za[4] = {mlp::pack_bf16(dz3[0], dz3[1]), mlp::pack_bf16(dz3[2], dz3[3]), 0u, 0u};
    uint32_t d2a[4][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      float c[4] = {0.0f, 0.0f, 0.0f, 0.0f};
      mlp::mma(c, za, mlp::ld32(&sm.wb.w3s[8 * nt + g][2 * t]), 0u);
      const int col = 8 * nt + 2 * t;
      if (!(__bfloat162float(sm.h2[r0 + g][col]) > 0.0f)) c[0] = 0.0f;
      if (!(__bfloat162float(sm.h2[r0 + g][col + 1]) > 0.0f)) c[1] = 0.0f;
      if (!(__bfloat162float(sm.h2[r0 + g + 8][col]) > 0.0f)) c[2] = 0.0f;
      if (!(__bfloat162float(sm.h2[r0 + g + 8][col + 1]) > 0.0f)) c[3] = 0.0f;
      db2[2 * nt] += c[0] + c[2];
      db2[2 * nt + 1] += c[1] + c[3];
      const uint32_t lo = mlp::pack_bf16(c[0], c[1]), hi = mlp::pack_bf16(c[2], c[3]);
      d2a[nt >> 1][(nt & 1) ? 2 : 0] = lo;
      d2a[nt >> 1][(nt & 1) ? 3 : 1] = hi;
      *reinterpret_cast<uint32_t*>(&sm.dz2[r0 + g][col]) = lo;
      *reinterpret_cast<uint32_t*>(&sm.dz2[r0 + g + 8][col]) = hi;
    }
    // dh1 = dz2 W2^T, masked by h1 > 0
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      float c[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
      for (int kc = 0; kc < 4; ++kc)
        mlp::mma(c, d2a[kc], mlp::ld32(&sm.wb.w2s[8 * nt + g][16 * kc + 2 * t]),
                 mlp::ld32(&sm.wb.w2s[8 * nt + g][16 * kc + 2 * t + 8]));
      const int col = 8 * nt + 2 * t;
      if (!(__bfloat162float(sm.h1[r0 + g][col]) > 0.0f)) c[0] = 0.0f;
      if (!(__bfloat162float(sm.h1[r0 + g][col + 1]) > 0.0f)) c[1] = 0.0f;
      if (!(__bfloat162float(sm.h1[r0 + g + 8][col]) > 0.0f)) c[2] = 0.0f;
      if (!(__bfloat162float(sm.h1[r0 + g + 8][col + 1]) > 0.0f)) c[3] = 0.0f;
      db1[2 * nt] += c[0] + c[2];
      db1[2 * nt + 1] += c[1] + c[3];
      *reinterpret_cast<uint32_t*>(&sm.dz1[r0 + g][col]) = mlp::pack_bf16(c[0], c[1]);
      *reinterpret_cast<uint32_t*>(&sm.dz1[r0 + g + 8][col]) = mlp::pack_bf16(c[2], c[3]);
    }
    __syncthreads();
    // weight gradients over the tile's 64 samples: dW = act^T dz
    auto act_a = [&](const __nv_bfloat16* act, int ld, int mt, int kc, uint32_t (&a)[4]) {
      const int m0 = 16 * mt + g, k0 = 16 * kc + 2 * t;
      a[0] = mlp::pack2h(act[k0 * ld + m0], act[(k0 + 1) * ld + m0]);
      a[1] = mlp::pack2h(act[k0 * ld + m0 + 8], act[(k0 + 1) * ld + m0 + 8]);
      a[2] = mlp::pack2h(act[(k0 + 8) * ld + m0], act[(k0 + 9) * ld + m0]);
      a[3] = mlp::pack2h(act[(k0 + 8) * ld + m0 + 8], act[(k0 + 9) * ld + m0 + 8]);
    };
    auto dz_b = [&](const __nv_bfloat16* dz, int ld, int nt, int kc, uint32_t& b0, uint32_t& b1) {
      const int n0 = 8 * nt + g, k0 = 16 * kc + 2 * t;
      b0 = mlp::pack2h(dz[k0 * ld + n0], dz[(k0 + 1) * ld + n0]);
      b1 = mlp::pack2h(dz[(k0 + 8) * ld + n0], dz[(k0 + 9) * ld + n0]);
    };
#pragma unroll
    for (int kc = 0; kc < 4; ++kc) {
      uint32_t a[4];
      act_a(&sm.h1[0][0], kH, warp, kc, a);  // dW2: rows 16 warp .. of W2
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        uint32_t b0, b1;
        dz_b(&sm.dz2[0][0], kH, nt, kc, b0, b1);
        mlp::mma(acc_w2[nt], a, b0, b1);
      }
      act_a(&sm.h2[0][0], kH, warp, kc, a);  // dW3: rows 16 warp ..
      {
        uint32_t b0, b1;
        dz_b(&sm.dz3[0][0], kOutPad, 0, kc, b0, b1);
        mlp::mma(acc_w3, a, b0, b1);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {  // dW1: tiles 4 warp .. 4 warp + 3 of (2 x 8)
        const int tt = 4 * warp + q, mt = tt >> 3, nt = tt & 7;
        uint32_t a1[4], b0, b1;
        act_a(&sm.xs[0][0], mlp::kLd1, mt, kc, a1);
        dz_b(&sm.dz1[0][0], kH, nt, kc, b0, b1);
        mlp::mma(acc_w1[q], a1, b0, b1);
      }
    }
  }
  // ---- write this block's gradient sums ----
  float* out = partials + (size_t)blockIdx.x * kParamsPad;
#pragma unroll
  for (int nt = 0; nt < 8; ++nt)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = 16 * warp + g + (q >= 2 ? 8 : 0), o = 8 * nt + 2 * t + (q & 1);
      out[mlp::kOffW2 + i * kH + o] = acc_w2[nt][q];
    }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = 16 * warp + g + (q >= 2 ? 8 : 0), c = 2 * t + (q & 1);
    if (c < kOut) out[mlp::kOffW3 + i * kOut + c] = acc_w3[q];
  }
#pragma unroll
  for (int qq = 0; qq < 4; ++qq) {
    const int tt = 4 * warp + qq, mt = tt >> 3, nt = tt & 7;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = 16 * mt + g + (q >= 2 ? 8 : 0), o = 8 * nt + 2 * t + (q & 1);
      if (i < kIn) out[mlp::kOffW1 + i * kH + o] = acc_w1[qq][q];
    }
  }
  // bias sums: reduce over the 8 lanes sharing t, then over warps in a fixed order
#pragma unroll
  for (int i = 0; i < 16; ++i)
#pragma unroll
    for (int o = 4; o < 32; o <<= 1) {
      db1[i] += __shfl_xor_sync(0xffffffffu, db1[i], o);
      db2[i] += __shfl_xor_sync(0xffffffffu, db2[i], o);
    }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int o = 4; o < 32; o <<= 1) db3[i] += __shfl_xor_sync(0xffffffffu, db3[i], o);
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) loss += __shfl_xor_sync(0xffffffffu, loss, o);
  __syncthreads();
  if (g == 0) {
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      sm.bias[warp][8 * nt + 2 * t] = db1[2 * nt];
      sm.bias[warp][8 * nt + 2 * t + 1] = db1[2 * nt + 1];
      sm.bias[warp][kH + 8 * nt + 2 * t] = db2[2 * nt];
      sm.bias[warp][kH + 8 * nt + 2 * t + 1] = db2[2 * nt + 1];
    }
    sm.bias[warp][2 * kH + 2 * t] = db3[0];
    sm.bias[warp][2 * kH + 2 * t + 1] = db3[1];
  }
  if (lane == 0) sm.loss[warp] = loss;
  __syncthreads();
  for (int i = threadIdx.x; i < 2 * kH + kOut; i += blockDim.x) {
    const float v = sm.bias[0][i] + sm.bias[1][i] + sm.bias[2][i] + sm.bias[3][i];
    const int off = i < kH ? mlp::kOffB1 + i : i < 2 * kH ? mlp::kOffB2 + (i - kH) : mlp::kOffB3 + (i - 2 * kH);
    out[off] = v;
  }
  if (threadIdx.x == 0) out[kParams] = sm.loss[0] + sm.loss[1] + sm.loss[2] + sm.loss[3];
}

// grad[k] = sum over blocks (fixed order); grad[kParams] = loss sum
__global__ void grad_reduce_kernel(const float* __restrict__ partials, int nblocks, int64_t batch,
                                   float* __restrict__ grad, float* __restrict__ loss_out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k > kParams) return;
  float s = 0.0f;
  for (int b = 0; b < nblocks; ++b) s += partials[(size_t)b * kParamsPad + k];
  grad[k] = s;
  if (k == kParams && loss_out) *loss_out = s / (float)batch;
}

__global__ void adam_kernel(float* __restrict__ P, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ grad, float lr, float b1t, float b2t) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= kParams) return;
  const float gk = grad[k];
  const float mk = 0.9f * m[k] + 0.1f * gk;
  const float vk = 0.999f * v[k] + 0.001f * gk * gk;
  m[k] = mk;
  v[k] = vk;
  P[k] -= lr * (mk / b1t) / (sqrtf(vk / b2t) + 1e-8f);
}

int train_blocks(int64_t batch) {
  const int64_t tiles = (batch + kTile - 1) / kTile;
  return (int)(tiles < 304 ? tiles : 304);
}

size_t train_smem() { return sizeof(TrainSmem); }

}  // namespace

size_t closure_partials_bytes(int64_t batch) { return (size_t)train_blocks(batch) * kParamsPad * sizeof(float); }

cudaError_t closure_grad(const float* X, const float* abc, int64_t n, int64_t batch, int random, uint64_t seed,
                         uint64_t iter, const float* cw, double lo, double hi, const float* P, float* partials,
                         float* grad, float* loss, cudaStream_t stream) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)train_smem());
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  LossArgs la;
  for (int c = 0; c < kOut; ++c) la.cw[c] = cw[c];
  la.lo = (float)lo;
  la.span = (float)(hi - lo);
  const int nb = train_blocks(batch);
  grad_kernel<<<nb, kTrainThreads, train_smem(), stream>>>(X, abc, n, batch, random, seed, iter, la, P, partials);
  grad_reduce_kernel<<<(kParams + 1 + 255) / 256, 256, 0, stream>>>(partials, nb, batch, grad, loss);
  return cudaGetLastError();
}

cudaError_t closure_adam(float* P, float* m, float* v, const float* grad, double lr, int64_t step,
                         cudaStream_t stream) {
  const float b1t = (float)(1.0 - std::pow(0.9, (double)step));
  const float b2t = (float)(1.0 - std::pow(0.999, (double)step));
  adam_kernel<<<(kParams + 255) / 256, 256, 0, stream>>>(P, m, v, grad, (float)lr, b1t, b2t);
  return cudaGetLastError();
}

cudaError_t closure_filter(Sim* s, int m, float* out) {
  tp::Grid g{(int)s->nx, (int)s->ny, (int)s->nz, s->N};
  const int ncx = (int)(s->nx / m), ncy = (int)(s->ny / m), ncz = (int)(s->nz / m);
  const int64_t Nc = (int64_t)ncx * ncy * ncz;
  const unsigned blocks = (unsigned)((Nc + 127) / 128);
  const int odd = (int)(s->step & 1);
  switch (s->storage) {
    case LBM_F64:
      filter_kernel<LBM_F64><<<blocks, 128, 0, s->stream>>>(static_cast<const double*>(s->pop), g, odd, m, ncx, ncy,
                                                            ncz, out);
      break;
    case LBM_F32:
      filter_kernel<LBM_F32><<<blocks, 128, 0, s->stream>>>(static_cast<const float*>(s->pop), g, odd, m, ncx, ncy,
                                                            ncz, out);
      break;
    case LBM_F16:
      filter_kernel<LBM_F16><<<blocks, 128, 0, s->stream>>>(static_cast<const __half*>(s->pop), g, odd, m, ncx, ncy,
                                                            ncz, out);
      break;
    default:
      filter_kernel<LBM_BF16><<<blocks, 128, 0, s->stream>>>(static_cast<const __nv_bfloat16*>(s->pop), g, odd, m,
                                                             ncx, ncy, ncz, out);
  }
  return cudaGetLastError();
}

cudaError_t closure_rescale(int64_t N, float* f, double scale, cudaStream_t stream) {
  rescale_kernel<<<(unsigned)((N + 127) / 128), 128, 0, stream>>>(f, N, (float)scale);
  return cudaGetLastError();
}

cudaError_t closure_dataset(const int64_t dims[3], const float* ft, const float* ft1, double tau2, const float* norm,
                            float* X, float* abc, cudaStream_t stream) {
  const int64_t N = dims[0] * dims[1] * dims[2];
  dataset_kernel<<<(unsigned)((N + 127) / 128), 128, 0, stream>>>(ft, ft1, (int)dims[0], (int)dims[1], (int)dims[2],
                                                                  (float)tau2, norm, X, abc);
  return cudaGetLastError();
}

// ---- sweep with the network fused into the collision ------------------------
namespace {

constexpr int kLearnThreads = 128;

#ifndef LBM_LEARN_MINB
#define LBM_LEARN_MINB 4  // 128 registers (a few words spill to L1): 16 warps per SM
#endif
constexpr int kRateLd = kOutPad + 1;  // odd row stride: each lane reads its own row conflict-free

struct LearnSmem {
  mlp::FwdW w;
  __nv_bfloat16 xs[kLearnThreads / 32][32][mlp::kLd1];
  float rates[kLearnThreads / 32][32][kRateLd];
  float stash[27][kLearnThreads];  // central moments parked while the network runs
};

// Forward weight image built once per lbm_set_closure (one block).
__global__ void build_image_kernel(const float* __restrict__ P, mlp::FwdW* __restrict__ img) {
  mlp::load_fwd(P, *img);
}

// One node per thread (D3Q27, FP32 offsets), AA pattern as tp_sweep.cu; blocks
// stride over 128-wide x tiles of the grid so the weight image is copied once
// per block.  All 32 lanes of a warp take part in the MLP (lanes past nx carry
// a rest-state node and store nothing).
template <bool ODD>
__global__ void __launch_bounds__(kLearnThreads, LBM_LEARN_MINB)
    learned_sweep_kernel(float* __restrict__ f, tp::Grid g, Rates r, const mlp::FwdW* __restrict__ img,
                         const float* __restrict__ norm, int* __restrict__ status) {
  __shared__ __align__(16) LearnSmem sm;
  mlp::copy_fwd(img, sm.w);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int xtiles = (g.nx + kLearnThreads - 1) / kLearnThreads;
  const int64_t ntile = (int64_t)xtiles * g.ny * g.nz;
  const float tau2m = 1.0f / (float)r.w[2] - 0.5f;
  const float lo = norm[2 * kIn], span = norm[2 * kIn + 1] - norm[2 * kIn];
  for (int64_t tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
    const int xt = (int)(tile % xtiles);
    const int64_t yz = tile / xtiles;
    const int y = (int)(yz % g.ny), z = (int)(yz / g.ny);
    const int x = xt * kLearnThreads + threadIdx.x;
    const bool active = x < g.nx;
    const int xc = active ? x : 0;
    float v[27];
    if (active) {
      tp::gather<3, LBM_F32>(f, g, xc, y, z, ODD ? 1 : 0, v);
    } else {
#pragma unroll
      for (int i = 0; i < 27; ++i) v[i] = 0.0f;
    }
    // moments, velocity, central moments (deviation form)
    tp::pops_to_raw<float, 3>(v);
    const float drho = v[0];
    const float rho = 1.0f + drho;
    const float irho = 1.0f / rho;
    tp::Vel<float, 3> w;
    float usq = 0.0f;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      w.u[d] = v[tp::p3(d)] * irho;
      w.nu[d] = -w.u[d];
      w.usq[d] = w.u[d] * w.u[d];
      w.nusq[d] = -w.usq[d];
      w.kk2[d] = w.usq[d] + (1.0f / 3.0f);
      usq += w.usq[d];
    }
    tp::raw_to_central<float, 3>(v, w.nu);
    // features: non-equilibrium central moments of orders 2..4 / (rho c_s^n), tau_2 - 1/2
    // (stored as BF16 pairs: 32-bit stores into the lane's own padded row)
    uint32_t* xrow = reinterpret_cast<uint32_t*>(&sm.xs[warp][lane][0]);
    float prev = 0.0f;
    int fi = 0;
#pragma unroll
    for (int a = 0; a < 27; ++a) {
      const int n = tp::order_of<3>(a);
      if (n < 2 || n > 4) continue;
      const float k1 = (v[a] - tp::eq_deviation<float, 3>(a, drho, w)) * (float)inv_cs_pow(n) * irho;
      const float x = (k1 - norm[fi]) * norm[kIn + fi];
      if (fi & 1)
        xrow[fi >> 1] = mlp::pack_bf16(prev, x);
      else
        prev = x;
      ++fi;
    }
    xrow[9] = mlp::pack_bf16(prev, (tau2m - norm[19]) * norm[kIn + 19]);
#pragma unroll
    for (int j = kIn / 2; j < kInPad / 2; ++j) xrow[j] = 0u;
#pragma unroll
    for (int a = 0; a < 27; ++a) sm.stash[a][threadIdx.x] = v[a];
    __syncwarp();
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      uint32_t h1a[4][4], h2a[4][4];
      float z3[4];
      mlp::forward16(sm.w, &sm.xs[warp][16 * half][0], mlp::kLd1, h1a, h2a, z3, nullptr, nullptr);
      const int gg = lane >> 2, t = lane & 3;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int row = 16 * half + gg + (q >= 2 ? 8 : 0), c = 2 * t + (q & 1);
        sm.rates[warp][row][c] = fmaf(span, 1.0f / (1.0f + __expf(-z3[q])), lo);
      }
    }
    __syncwarp();
    float cr[kOut];
#pragma unroll
    for (int c = 0; c < kOut; ++c) cr[c] = sm.rates[warp][lane][c];
#pragma unroll
    for (int a = 0; a < 27; ++a) v[a] = sm.stash[a][threadIdx.x];
    // relax: order 2 at omega_2, orders 3..6 at the class rates
    const float om2 = (float)r.w[2];
#pragma unroll
    for (int a = 0; a < 27; ++a) {
      const int n = tp::order_of<3>(a);
      if (n <= 1) continue;
      const float om = n == 2 ? om2 : cr[class_of(a)];
      v[a] = fmaf(om, tp::eq_deviation<float, 3>(a, drho, w) - v[a], v[a]);
    }
    tp::central_to_raw<float, 3>(v, w.u);
    tp::raw_to_pops<float, 3>(v);
    if (active) {
      if (!(rho > 0.0f && usq < 1.0f)) atomicOr(status, 1);
      // even sweep: population i to slot (x, opp(i)); odd sweep: to slot (x + e_i, i)
      const uint32_t node = (uint32_t)xc + (uint32_t)g.nx * ((uint32_t)y + (uint32_t)g.ny * (uint32_t)z);
#pragma unroll
      for (int j = 0; j < 27; ++j) {
        if (!ODD)
          f[(size_t)j * g.N + node] = v[tp::opp<3>(j)];
        else
          f[(size_t)j * g.N + tp::neighbour<3>(g, xc, y, z, j)] = v[j];
      }
    }
    __syncwarp();
  }
}

// ---- the same sweep with the network on tcgen05 -----------------------------
// A 128-node tile is one M = 128 MMA chain: features A1[128 x 32], hidden
// activations A2 / A3[128 x 80] (shared, K-major core-matrix layout), weights
// B1[64 x 32], B2[64 x 80], B3[16 x 80].  Biases ride in three extra K columns
// (BF16 high, middle and low parts) against constant-one inputs, so the FP32
// accumulators hold W x + b with the bias to FP32 precision.
// Accumulators: tensor-memory columns 0..63 (layers 1 and 2), 64..79 (layer 3).
namespace tcimg {
constexpr int kK1 = 32, kK2 = 80, kN3 = 16;
constexpr int kB1 = 0, kB2 = kB1 + 64 * kK1 * 2, kB3 = kB2 + 64 * kK2 * 2, kBytes = kB3 + kN3 * kK2 * 2;  // 16896
constexpr int kA1Bytes = 128 * kK1 * 2, kA2Bytes = 128 * kK2 * 2;
constexpr uint32_t kCols = 128;
constexpr int kWaitPolls = 1 << 20;
}  // namespace tcimg

// b = hi + mid + lo to FP32 precision (each part the BF16 rounding of what is left)
__device__ __forceinline__ void split_bf16(float b, __nv_bfloat16 (&part)[3]) {
  float rest = b;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    part[i] = __float2bfloat16_rn(rest);
    rest -= __bfloat162float(part[i]);
  }
}

// 1 / c_s^n of the order of feature k (the features are the order-2..4 central
// moments in index order, then tau_2 - 1/2)
__host__ __device__ constexpr double feature_scale(int k) {
  int fi = 0;
  for (int a = 0; a < 27; ++a) {
    const int n = tp::order_of<3>(a);
    if (n < 2 || n > 4) continue;
    if (fi == k) return inv_cs_pow(n);
    ++fi;
  }
  return 1.0;
}

// The standardisation of the moment features is folded into layer 1: with
// x_k = (k1_k s_k - mean_k) istd_k (s_k = 1 / c_s^n), W1 x + b1 =
// W1' k1 + b1' with W1'_kn = W1_kn s_k istd_k and b1'_n = b1_n - sum_k W1_kn
// mean_k istd_k, so the sweep feeds the raw moments k1 (tau_2 - 1/2 keeps its
// standardisation: the rates may change after the image is built).  The
// standardisation (40 values) follows the 5904 parameter slots in the closure
// workspace.
__global__ void build_tc_image_kernel(const float* __restrict__ P, unsigned char* __restrict__ img) {
  using namespace tcimg;
  const float* norm = P + kParamsPad;
  __nv_bfloat16* b1 = reinterpret_cast<__nv_bfloat16*>(img + kB1);
  __nv_bfloat16* b2 = reinterpret_cast<__nv_bfloat16*>(img + kB2);
  __nv_bfloat16* b3 = reinterpret_cast<__nv_bfloat16*>(img + kB3);
  for (int i = threadIdx.x; i < 64 * kK1; i += blockDim.x) {
    const int n = i / kK1, k = i % kK1;
    __nv_bfloat16 v = __float2bfloat16_rn(0.0f), part[3];
    float bias = P[mlp::kOffB1 + n];
    for (int kk = 0; kk < kIn - 1; ++kk) bias -= P[mlp::kOffW1 + kk * kH + n] * norm[kk] * norm[kIn + kk];
    split_bf16(bias, part);
    if (k < kIn - 1)
      v = __float2bfloat16_rn(P[mlp::kOffW1 + k * kH + n] * (float)feature_scale(k) * norm[kIn + k]);
    if (k == kIn - 1) v = __float2bfloat16_rn(P[mlp::kOffW1 + k * kH + n]);
    if (k >= kIn && k < kIn + 3) v = part[k - kIn];
    b1[tc05::core_offset(n, k, kK1) / 2] = v;
  }
  for (int i = threadIdx.x; i < 64 * kK2; i += blockDim.x) {
    const int n = i / kK2, k = i % kK2;
    __nv_bfloat16 v = __float2bfloat16_rn(0.0f), part[3];
    split_bf16(P[mlp::kOffB2 + n], part);
    if (k < kH) v = __float2bfloat16_rn(P[mlp::kOffW2 + k * kH + n]);
    if (k >= kH && k < kH + 3) v = part[k - kH];
    b2[tc05::core_offset(n, k, kK2) / 2] = v;
  }
  for (int i = threadIdx.x; i < kN3 * kK2; i += blockDim.x) {
    const int n = i / kK2, k = i % kK2;
    __nv_bfloat16 v = __float2bfloat16_rn(0.0f);
    if (n < kOut) {
      __nv_bfloat16 part[3];
      split_bf16(P[mlp::kOffB3 + n], part);
      if (k < kH) v = __float2bfloat16_rn(P[mlp::kOffW3 + k * kOut + n]);
      if (k >= kH && k < kH + 3) v = part[k - kH];
    }
    b3[tc05::core_offset(n, k, kK2) / 2] = v;
  }
}

struct TcSmem {
  unsigned char w[tcimg::kBytes];
  unsigned char a1[tcimg::kA1Bytes];
  unsigned char a2[tcimg::kA2Bytes];
  uint64_t mbar;
  uint32_t tbase;
};

// Write 8 consecutive K entries (16 bytes) of row r of a K-major tile.
__device__ __forceinline__ void put8(unsigned char* tile, int K, int r, int kgroup, uint4 v) {
  *reinterpret_cast<uint4*>(tile + tc05::core_offset(r, 8 * kgroup, K)) = v;
}

// One thread issues the MMAs of one layer (K / 16 slices) and commits them.
__device__ __forceinline__ void issue_layer(uint32_t d_tmem, const unsigned char* a, const unsigned char* b, int K,
                                            uint32_t idesc, uint64_t* mbar) {
  const uint32_t a0 = tc05::smem_u32(a), b0 = tc05::smem_u32(b), sbo = (uint32_t)(K / 8) * 128;
  for (int s = 0; s < K / 16; ++s)
    tc05::mma(d_tmem, tc05::make_desc(a0 + 256 * s, 128, sbo), tc05::make_desc(b0 + 256 * s, 128, sbo), idesc,
              s > 0 ? 1u : 0u);
  tc05::commit(mbar);
}

// Read 64 accumulator columns of this thread's row, apply ReLU, and write them
// as BF16 into row r (K groups 0..7) of the 80-wide activation tile.
__device__ __forceinline__ void relu_to_tile(uint32_t taddr, unsigned char* a2, int r) {
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    float x[16];
    tc05::ld16(taddr + 16 * c, x);
    uint4 lo, hi;
    lo.x = tc05::relu_bf16x2(x[0], x[1]);
    lo.y = tc05::relu_bf16x2(x[2], x[3]);
    lo.z = tc05::relu_bf16x2(x[4], x[5]);
    lo.w = tc05::relu_bf16x2(x[6], x[7]);
    hi.x = tc05::relu_bf16x2(x[8], x[9]);
    hi.y = tc05::relu_bf16x2(x[10], x[11]);
    hi.z = tc05::relu_bf16x2(x[12], x[13]);
    hi.w = tc05::relu_bf16x2(x[14], x[15]);
    put8(a2, tcimg::kK2, r, 2 * c, lo);
    put8(a2, tcimg::kK2, r, 2 * c + 1, hi);
  }
}

template <bool ODD>
__global__ void __launch_bounds__(kLearnThreads, 4)
    learned_tc_kernel(float* __restrict__ f, tp::Grid g, Rates r, const unsigned char* __restrict__ img,
                      const float* __restrict__ norm, int* __restrict__ status) {
  using namespace tcimg;
  extern __shared__ __align__(16) unsigned char tc_smem_raw[];
  // operand tiles start on 128-byte boundaries (descriptors need 16)
  TcSmem& sm = *reinterpret_cast<TcSmem*>(tc_smem_raw + ((128u - (tc05::smem_u32(tc_smem_raw) & 127u)) & 127u));
  const int tid = threadIdx.x, warp = tid >> 5;
  {
    const uint4* src = reinterpret_cast<const uint4*>(img);
    uint4* dst = reinterpret_cast<uint4*>(sm.w);
    for (int i = tid; i < kBytes / 16; i += blockDim.x) dst[i] = src[i];
  }
  // constant K columns of this thread's rows: A1 k 24..31 zero; A2 k 64..66 one, 67..79 zero
  const uint32_t one2 = mlp::pack_bf16(1.0f, 1.0f), one0 = mlp::pack_bf16(1.0f, 0.0f);
  put8(sm.a1, kK1, tid, 3, make_uint4(0u, 0u, 0u, 0u));
  put8(sm.a2, kK2, tid, 8, make_uint4(one2, one0, 0u, 0u));
  put8(sm.a2, kK2, tid, 9, make_uint4(0u, 0u, 0u, 0u));
  if (warp == 0) {
    tc05::alloc(&sm.tbase, kCols);
    tc05::relinquish();
  }
  if (tid == 0) {
    tc05::mbar_init(&sm.mbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc05::fence_before();
  __syncthreads();
  tc05::fence_after();
  const uint32_t tmem = sm.tbase;
  const uint32_t trow = tmem + ((uint32_t)(32 * warp) << 16);  // this warp's lane quarter
  const uint32_t id64 = tc05::idesc_bf16(128, 64), id16 = tc05::idesc_bf16(128, kN3);
  const int xtiles = (g.nx + kLearnThreads - 1) / kLearnThreads;
  const int64_t ntile = (int64_t)xtiles * g.ny * g.nz;
  const float tau2m = 1.0f / (float)r.w[2] - 0.5f;
  const float x_tau = (tau2m - norm[kIn - 1]) * norm[2 * kIn - 1];  // the one standardised feature
  const float lo = norm[2 * kIn], span = norm[2 * kIn + 1] - norm[2 * kIn];
  const float om2 = (float)r.w[2];
  uint32_t phase = 0;
  int bad = 0;
  for (int64_t tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
    const int xt = (int)(tile % xtiles);
    const int64_t yz = tile / xtiles;
    const int y = (int)(yz % g.ny), z = (int)(yz / g.ny);
    const int x = xt * kLearnThreads + tid;
    const bool active = x < g.nx;
    const int xc = active ? x : 0;
    float v[27];
    if (active) {
      // the slots of this node in the parity's AA layout: per-axis wrapped
      // offsets once, two adds per population (the sweep's own addressing)
      const tp::NodeAddr<3, ODD> A(g, xc, y, z);
      tp::node_load<3, LBM_F32, ODD>(f, g, A, v);
    } else {
#pragma unroll
      for (int i = 0; i < 27; ++i) v[i] = 0.0f;
    }
    tp::pops_to_raw<float, 3>(v);
    const float drho = v[0];
    const float rho = 1.0f + drho;
    const float irho = 1.0f / rho;
    tp::Vel<float, 3> w;
    float usq = 0.0f;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      w.u[d] = v[tp::p3(d)] * irho;
      w.nu[d] = -w.u[d];
      w.usq[d] = w.u[d] * w.u[d];
      w.nusq[d] = -w.usq[d];
      w.kk2[d] = w.usq[d] + (1.0f / 3.0f);
      usq += w.usq[d];
    }
    tp::raw_to_central<float, 3>(v, w.nu);
    // features -> A1 row tid: k 0..19 features, 20..22 one (bias), 23..31 zero
    uint32_t fp[12];
    {
      float prev = 0.0f;
      int fi = 0;
#pragma unroll
      for (int a = 0; a < 27; ++a) {
        const int n = tp::order_of<3>(a);
        if (n < 2 || n > 4) continue;
        // the raw non-equilibrium moment: scale and standardisation sit in W1 and b1
        const float xf = (v[a] - tp::eq_deviation<float, 3>(a, drho, w)) * irho;
        if (fi & 1)
          fp[fi >> 1] = mlp::pack_bf16(prev, xf);
        else
          prev = xf;
        ++fi;
      }
      fp[9] = mlp::pack_bf16(prev, x_tau);
      fp[10] = one2;
      fp[11] = one0;
    }
    put8(sm.a1, kK1, tid, 0, make_uint4(fp[0], fp[1], fp[2], fp[3]));
    put8(sm.a1, kK1, tid, 1, make_uint4(fp[4], fp[5], fp[6], fp[7]));
    put8(sm.a1, kK1, tid, 2, make_uint4(fp[8], fp[9], fp[10], fp[11]));
    tc05::fence_proxy_async();
    tc05::fence_before();
    if (__syncthreads_or(bad)) break;
    tc05::fence_after();
    // layer 1
    if (tid == 0) issue_layer(tmem, sm.a1, sm.w + kB1, kK1, id64, &sm.mbar);
    bad |= !tc05::mbar_wait(&sm.mbar, phase, kWaitPolls);
    phase ^= 1u;
    tc05::fence_after();
    if (!bad) relu_to_tile(trow, sm.a2, tid);
    tc05::fence_proxy_async();
    tc05::fence_before();
    if (__syncthreads_or(bad)) break;
    tc05::fence_after();
    // layer 2
    if (tid == 0) issue_layer(tmem, sm.a2, sm.w + kB2, kK2, id64, &sm.mbar);
    bad |= !tc05::mbar_wait(&sm.mbar, phase, kWaitPolls);
    phase ^= 1u;
    tc05::fence_after();
    if (!bad) relu_to_tile(trow, sm.a2, tid);
    tc05::fence_proxy_async();
    tc05::fence_before();
    if (__syncthreads_or(bad)) break;
    tc05::fence_after();
    // layer 3 -> columns 64..79
    if (tid == 0) issue_layer(tmem + 64, sm.a2, sm.w + kB3, kK2, id16, &sm.mbar);
    bad |= !tc05::mbar_wait(&sm.mbar, phase, kWaitPolls);
    phase ^= 1u;
    tc05::fence_after();
    float zo[16];
    if (!bad) tc05::ld16(trow + 64, zo);
    tc05::fence_before();
    if (__syncthreads_or(bad)) break;
    float cr[kOut];
#pragma unroll
    for (int c = 0; c < kOut; ++c) cr[c] = fmaf(span, 1.0f / (1.0f + __expf(-zo[c])), lo);
    // relax: order 2 at omega_2, orders 3..6 at the class rates
#pragma unroll
    for (int a = 0; a < 27; ++a) {
      const int n = tp::order_of<3>(a);
      if (n <= 1) continue;
      const float om = n == 2 ? om2 : cr[class_of(a)];
      v[a] = fmaf(om, tp::eq_deviation<float, 3>(a, drho, w) - v[a], v[a]);
    }
    tp::central_to_raw<float, 3>(v, w.u);
    tp::raw_to_pops<float, 3>(v);
    if (active) {
      if (!(rho > 0.0f && usq < 1.0f)) atomicOr(status, 1);
      // even sweep: population i to slot (x, opp(i)); odd sweep: to slot (x + e_i, i)
      const tp::NodeAddr<3, ODD> A(g, xc, y, z);
      tp::node_store<3, LBM_F32, ODD>(f, g, A, v);
    }
  }
  if (bad) {
    // a wait gave up: report it, give in-flight MMAs a bounded chance to finish
    if (tid == 0) atomicOr(status, 2);
    tc05::mbar_wait(&sm.mbar, phase, kWaitPolls);
  }
  tc05::fence_before();
  __syncthreads();
  tc05::fence_after();
  if (warp == 0) tc05::dealloc(tmem, kCols);
}

}  // namespace

cudaError_t closure_build_image(const float* P, void* img, cudaStream_t stream) {
  build_image_kernel<<<1, 256, 0, stream>>>(P, static_cast<mlp::FwdW*>(img));
  build_tc_image_kernel<<<1, 256, 0, stream>>>(P, static_cast<unsigned char*>(img) + kTcImageOffset);
  return cudaGetLastError();
}

size_t closure_image_bytes() { return kTcImageOffset + tcimg::kBytes; }

// The network of the fused sweep runs on tcgen05; LBM_LEARNED_MMA=sync selects
// the warp-level mma.sync kernel instead (read at every launch).
bool closure_uses_tcgen05() {
  const char* e = std::getenv("LBM_LEARNED_MMA");
  return !(e && std::strcmp(e, "sync") == 0);
}

static cudaError_t closure_sweep_tc(Sim* s, int odd, const void* img, const float* norm, int blocks) {
  tp::Grid g{(int)s->nx, (int)s->ny, (int)s->nz, s->N};
  static bool attr = false;
  const int smem = (int)sizeof(TcSmem) + 1024;  // + alignment slack of the dynamic base
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(learned_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(learned_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  float* f = static_cast<float*>(s->pop);
  const unsigned char* w = static_cast<const unsigned char*>(img) + kTcImageOffset;
  if (odd)
    learned_tc_kernel<true><<<blocks, kLearnThreads, smem, s->stream>>>(f, g, s->rates, w, norm, status_word(s));
  else
    learned_tc_kernel<false><<<blocks, kLearnThreads, smem, s->stream>>>(f, g, s->rates, w, norm, status_word(s));
  return cudaGetLastError();
}

cudaError_t closure_sweep(Sim* s, int odd, const void* img, const float* norm) {
  tp::Grid g{(int)s->nx, (int)s->ny, (int)s->nz, s->N};
  const int64_t xtiles = (s->nx + kLearnThreads - 1) / kLearnThreads;
  const int64_t ntile = xtiles * s->ny * s->nz;
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t cap = (int64_t)sms * 8;
  const unsigned blocks = (unsigned)(ntile < cap ? ntile : cap);
  if (closure_uses_tcgen05()) {
    const int64_t cap_tc = (int64_t)sms * 4;  // resident blocks: 4 x 128 tensor-memory columns per SM
    return closure_sweep_tc(s, odd, img, norm, (int)(ntile < cap_tc ? ntile : cap_tc));
  }
  float* f = static_cast<float*>(s->pop);
  const mlp::FwdW* w = static_cast<const mlp::FwdW*>(img);
  if (odd)
    learned_sweep_kernel<true><<<blocks, kLearnThreads, 0, s->stream>>>(f, g, s->rates, w, norm, status_word(s));
  else
    learned_sweep_kernel<false><<<blocks, kLearnThreads, 0, s->stream>>>(f, g, s->rates, w, norm, status_word(s));
  return cudaGetLastError();
}

}  // namespace lbm
