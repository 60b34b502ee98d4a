// Internal definitions shared by the library's translation units: the handle,
// the workspace layout, error reporting and the storage codecs.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <memory>

#include "lbm.h"

namespace lbm {

constexpr int kMaxOrders = 7;  // central-moment orders 0..6 on D3Q27

// Workspace layout (byte offsets into the caller's work buffer).
constexpr size_t kWsStatus = 0;            // int32 status word (+ padding)
constexpr size_t kWsResult = 256;          // 32 doubles of reduction results
constexpr size_t kWsPartials = 512;        // kRedBlocks x 8 doubles of block partials
constexpr int kRedBlocks = 1216;           // 8 x 152 SMs
constexpr int kRedThreads = 256;
constexpr int kMaxHistory = 4096;         // records of lbm_mode_history
constexpr size_t kWsHistory = kWsPartials + (size_t)kRedBlocks * 8 * sizeof(double);
constexpr size_t kWsFit = kWsHistory + (size_t)kMaxHistory * 2 * sizeof(double);  // 4 + 2n doubles
constexpr size_t kWsClosure = kWsFit + (((size_t)(4 + 2 * kMaxHistory) * sizeof(double) + 255) & ~(size_t)255);
// network parameters (padded to 5904) + standardisation (40) and rate range (2) in 64
// slots + the BF16 forward weight image (<= 4096 floats, 16-byte aligned)
constexpr int kClosureImageFloats = 8448;  // mma.sync image (16032 B) + tcgen05 image at byte 16384 (16896 B)
constexpr size_t kTcImageOffset = 16384;
constexpr int kClosureFloats = 5904 + 64 + kClosureImageFloats;
constexpr size_t kWsStaging = kWsClosure + (((size_t)kClosureFloats * sizeof(float) + 255) & ~(size_t)255);
constexpr size_t kStagingMax = (size_t)32 << 20;  // host<->device staging, bytes

struct Rates {
  double w[kMaxOrders];  // omega_n = 1 / tau_n for n = 0..2D (0 for n <= 1)
};

// A caller-supplied two-dimensional Hermite lattice (LBM_HERMITE): Q velocities
// xi_i = c e_i with |e| <= 3, weights, opposite-velocity map, truncation order N.
constexpr int kHQMax = 37;
struct HLattice {
  int q = 0, order = 0;
  int ex[kHQMax], ey[kHQMax], opp[kHQMax];
  double w[kHQMax];
  double c = 0.0;
};

// Projection tables of a Hermite lattice, built on the host once per
// simulation and passed to its kernels by value (component k = cidx(p, q) of
// order p + q <= N): H[k][i] = He_p(xi_ix) He_q(xi_iy),
// R[i][k] = w_i H[k][i] / (p! q!), fref[i] = f_eq,i(1, 0, theta_ref).
struct HTables {
  int q, nc;
  int ex[kHQMax], ey[kHQMax], opp[kHQMax];
  double H[15][kHQMax];
  double R[kHQMax][15];
  double fref[kHQMax];
  double c;
};

struct Sim {
  int lattice;
  int D, Q;
  int storage;
  unsigned flags;    // LBM_THERMAL / LBM_K72 / LBM_RAW_MRT (37-velocity lattice)
  double theta_ref;  // offset base temperature (37-velocity lattice)
  int64_t nx, ny, nz, N;
  Rates rates;
  void* pop;
  size_t pop_bytes;
  unsigned char* work;
  size_t work_bytes;
  size_t staging_bytes;
  cudaStream_t stream;
  int64_t step;  // steps since init; parity selects the AA layout
  // planes z_lo .. z_lo + z_cnt - 1 are swept and reduced (D3Q27 slabs of a
  // decomposed grid); z_cnt == 0 means the whole grid
  int64_t z_lo, z_cnt;
  int closure;   // 1: orders 3..6 relax at rates from the learned network (D3Q27, FP32)
  HLattice hl;                          // LBM_HERMITE only
  std::shared_ptr<const HTables> ht;    // LBM_HERMITE only
};

int set_error(int code, const char* fmt, ...);
int cuda_check(cudaError_t e, const char* what);

inline int64_t active_z0(const Sim* s) { return s->z_cnt > 0 ? s->z_lo : 0; }
inline int64_t active_nz(const Sim* s) { return s->z_cnt > 0 ? s->z_cnt : s->nz; }

inline int* status_word(Sim* s) { return reinterpret_cast<int*>(s->work + kWsStatus); }
inline double* result_buf(Sim* s) { return reinterpret_cast<double*>(s->work + kWsResult); }
inline double* partials_buf(Sim* s) { return reinterpret_cast<double*>(s->work + kWsPartials); }
// zero at creation (the status clear covers it); the totals sum resets it after use
inline unsigned* ticket_buf(Sim* s) { return reinterpret_cast<unsigned*>(s->work + kWsResult + 192); }
inline unsigned char* staging_buf(Sim* s) { return s->work + kWsStaging; }
inline double* history_buf(Sim* s) { return reinterpret_cast<double*>(s->work + kWsHistory); }
inline double* fit_buf(Sim* s) { return reinterpret_cast<double*>(s->work + kWsFit); }
inline float* closure_params(Sim* s) { return reinterpret_cast<float*>(s->work + kWsClosure); }
inline float* closure_norm(Sim* s) { return reinterpret_cast<float*>(s->work + kWsClosure) + 5904; }
inline float* closure_image(Sim* s) { return reinterpret_cast<float*>(s->work + kWsClosure) + 5904 + 64; }

size_t storage_elem_bytes(int storage);

// --- launches for the tensor-product lattices ---
// one node per thread, every storage type (tp_sweep.cu)
cudaError_t tp_launch_sweep(Sim* s, int odd);
// two nodes per thread in packed FP32x2, FP32/FP16/BF16 storage, nx even (tp_pair.cu)
bool tp_pair_supported(const Sim* s);
cudaError_t tp_launch_pair_sweep(Sim* s, int odd);
// The pair sweep that also writes FP32 partials (8 floats per warp, the first
// 5 used) of the totals of the state it consumed; tp_pair_warps of them.
int64_t tp_pair_warps(const Sim* s);
cudaError_t tp_launch_pair_sweep_totals(Sim* s, int odd, float* partials);
// Deterministic FP64 sum of n partials (stride 8 floats) into out[0..5): block
// sums in scratch, then the last block to finish (a ticket in the workspace)
// adds them in a fixed order and resets the ticket.
cudaError_t launch_sum_partials(const float* partials, int64_t n, double* scratch, unsigned* ticket, double* out,
                                cudaStream_t stream);
// fields: rho (N), u (D x N) as f64 or f32 device arrays covering nodes [n0, n0 + cnt)
cudaError_t tp_launch_init(Sim* s, const void* rho, const void* u, int dtype, int64_t n0,
                           int64_t cnt, int64_t ld);
cudaError_t tp_launch_moments(Sim* s, void* rho, void* u, int dtype, int64_t n0, int64_t cnt,
                              int64_t ld);
cudaError_t tp_launch_get_pops(Sim* s, double* f, int64_t n0, int64_t cnt, int64_t ld);
cudaError_t tp_launch_set_pops(Sim* s, const double* f, int64_t n0, int64_t cnt, int64_t ld);
// the grid totals into explicit scratch: nblocks x 8 partials, result[0..4]
cudaError_t tp_launch_reduce_into(Sim* s, double* partials, int nblocks, double* result);
// the single-wavenumber amplitude written to out2[0..1] (device)
cudaError_t tp_launch_mode_into(Sim* s, int field, const int64_t mode[3], double* out2);

// --- launches for caller-supplied Hermite lattices (hgen.cu), as the 37-velocity ones ---
void hgen_build_tables(const HLattice& L, double theta_ref, HTables* t);
cudaError_t hgen_launch_sweep(Sim* s, int odd);
cudaError_t hgen_launch_init(Sim* s, const void* rho, const void* u, const void* theta, int dtype, int64_t n0,
                             int64_t cnt, int64_t ld);
cudaError_t hgen_launch_moments(Sim* s, void* rho, void* u, void* theta, int dtype, int64_t n0, int64_t cnt,
                                int64_t ld);
cudaError_t hgen_launch_get_pops(Sim* s, double* f, int64_t n0, int64_t cnt, int64_t ld);
cudaError_t hgen_launch_set_pops(Sim* s, const double* f, int64_t n0, int64_t cnt, int64_t ld);
cudaError_t hgen_launch_reduce_into(Sim* s, double* partials, int nblocks, double* result);
cudaError_t hgen_launch_mode_into(Sim* s, int field, const int64_t mode[3], double* out2);

// --- launches for the 37-velocity lattice (h37.cu); fields as above plus theta
// (nullable), velocities in lattice units ---
cudaError_t h37_launch_sweep(Sim* s, int odd);
// The 37-velocity pair sweep (16/32-bit storage, even nx) with per-warp FP32
// partials of the consumed state's totals, as tp_launch_pair_sweep_totals.
bool h37_pair_supported(const Sim* s);
int64_t h37_pair_warps(const Sim* s);
cudaError_t h37_launch_pair_sweep_totals(Sim* s, int odd, float* partials);
cudaError_t h37_launch_init(Sim* s, const void* rho, const void* u, const void* theta, int dtype, int64_t n0,
                            int64_t cnt, int64_t ld);
cudaError_t h37_launch_moments(Sim* s, void* rho, void* u, void* theta, int dtype, int64_t n0, int64_t cnt,
                               int64_t ld);
cudaError_t h37_launch_get_pops(Sim* s, double* f, int64_t n0, int64_t cnt, int64_t ld);
cudaError_t h37_launch_set_pops(Sim* s, const double* f, int64_t n0, int64_t cnt, int64_t ld);
cudaError_t h37_launch_reduce_into(Sim* s, double* partials, int nblocks, double* result);
cudaError_t h37_launch_mode_into(Sim* s, int field, const int64_t mode[3], double* out2);

// --- lattice dispatch (lbm_abi.cu) ---
cudaError_t launch_sweep(Sim* s);  // one step at the current parity
cudaError_t launch_reduce_into(Sim* s, double* partials, int nblocks, double* result);

// --- learned closure (closure.cu) ---
cudaError_t closure_filter(Sim* s, int m, float* out);
cudaError_t closure_dataset(const int64_t dims[3], const float* ft, const float* ft1, double tau2, const float* norm,
                            float* X, float* abc, cudaStream_t stream);
size_t closure_partials_bytes(int64_t batch);
cudaError_t closure_grad(const float* X, const float* abc, int64_t n, int64_t batch, int random, uint64_t seed,
                         uint64_t iter, const float* cw, double lo, double hi, const float* P, float* partials,
                         float* grad, float* loss, cudaStream_t stream);
cudaError_t closure_rescale(int64_t N, float* f, double scale, cudaStream_t stream);
cudaError_t closure_adam(float* P, float* m, float* v, const float* grad, double lr, int64_t step,
                         cudaStream_t stream);
cudaError_t closure_sweep(Sim* s, int odd, const void* img, const float* norm);
cudaError_t closure_build_image(const float* P, void* img, cudaStream_t stream);
size_t closure_image_bytes();

// --- lattice-independent kernels (fit.cu) ---
// FP64 least-squares fit of ln|A_r| and of the unwrapped phase of A_r against
// t_r = r * stride for the n complex records hist[2r], hist[2r+1] (re_offset is
// added to every real part first); writes fit[0] = decay rate, fit[1] = angular
// frequency, fit[2] = ln|A| intercept, fit[3] = phase intercept (device); uses
// fit[4 .. 4 + 2n) as scratch.
// n elements of value v (f64 or f32 by dtype) written to device memory p
cudaError_t launch_fill(void* p, int dtype, int64_t n, double v, cudaStream_t stream);
cudaError_t launch_decay_fit(const double* hist, int n, double stride, double re_offset, double* fit,
                             cudaStream_t stream);

}  // namespace lbm
