/*
 * lbm.h -- C ABI of the GB300 central-moment MRT lattice Boltzmann library.
 *
 * The library advances a periodic lattice Boltzmann simulation with the
 * central-moment multiple-relaxation-time (CM-MRT) collision of
 * X. Shan, "A central-moment multiple-relaxation-time collision model"
 * (arXiv:1808.04406):
 *   - Sec. II.C, Eq. (omega): every central moment of order n of the
 *     collision term is -omega_n times that moment of the non-equilibrium
 *     part f^(1) = f - f^(0), omega_n = 1/tau_n;
 *   - Sec. II.C, final update: f_i(x + xi_i, t + 1) = f_i^ + Omega_i
 *     (collide, then stream along the discrete velocity).
 * One lbm_step is one fused stream+collide sweep over every node, done in
 * place with the AA access pattern: each step reads and writes every
 * population exactly once.
 *
 * Conventions shared by every call:
 *   - Return value: LBM_OK (0) or a negative LBM_E* code; lbm_last_error()
 *     then holds a message for the calling thread.  No call aborts or traps.
 *   - Memory: the library allocates no device memory.  The caller allocates
 *     the population buffer and the workspace (sizes from lbm_query_bytes)
 *     on the current CUDA device and keeps them alive until lbm_destroy.
 *     Buffers passed to other calls are never retained after they return
 *     (lbm_step_totals_async, below, writes its output later).
 *   - Streams: work is enqueued on the stream set by lbm_set_stream (default:
 *     the legacy default stream).  lbm_step returns without waiting.  Calls
 *     that return data to host memory synchronise that stream, except
 *     lbm_step_totals_async.
 *   - Fields use the layout rho[node], u[d * N + node] (d = 0..D-1),
 *     node = x + nx * (y + ny * z), N = nx * ny * nz.
 *   - Populations exchanged with lbm_get/set_populations are FP64 absolute
 *     values f[i * N + node] at the current time (after streaming, before
 *     collision) whatever the storage type and AA parity.  Velocity index on
 *     D2Q9 / D3Q27: i = sum_d (e_id + 1) * 3^d, e_id in {-1, 0, 1}.
 *   - One handle is used by one host thread at a time.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_sim* lbm_handle;

/* Lattices.  D2Q9 and D3Q27 are the tensor products of the three-point
 * Gauss-Hermite rule (Sec. II.A, Eq. quad) in lattice units, c_s^2 = 1/3;
 * moment orders run 0..2D (the paper runs D2Q9 with BGK only, Sec. III.B).
 * D2Q37 is the 37-velocity rule of algebraic degree 9 (shells (0,0), (1,0),
 * (1,1), (2,0), (2,1), (2,2), (3,0), (3,1); xi_i = c e_i, c = 1.19697977...),
 * the lattice of the paper's numerical tests (Sec. III): Hermite projection
 * and equilibrium truncation N = M = 4, relaxation orders 2..4, closed-form
 * collision of Eq. mrt; it needs nx, ny >= 3. */
#define LBM_D2Q9 1
#define LBM_D3Q27 2
#define LBM_D2Q37 3
#define LBM_HERMITE 4 /* a caller-supplied 2D Hermite lattice (lbm_create_hermite) */

/* Model flags for lbm_create_ex (37-velocity lattice; LBM_THERMAL and
 * LBM_FAST_TRANSFORMS also for lbm_create_hermite).
 *   LBM_THERMAL: temperature from the moments, rho (u^2 + 2 eps) = sum f xi^2,
 *     eps = D theta / 2 (Sec. II.A); without it theta is frozen at 1 (the
 *     paper's isothermal runs, Sec. III.B).
 *   LBM_K72: the 4th-order coupling constant as printed in Eq. mrt (72) instead
 *     of 6, the value Eq. omega gives with the n!-normalised polynomials.
 *   LBM_RAW_MRT: relax each Hermite coefficient in the absolute frame (the
 *     earlier high-order MRT of Sec. II.B) instead of the central moments.
 *   LBM_STOCHASTIC_ROUND: FP16 / BF16 storage only (no effect otherwise): every
 *     sweep rounds the stored offsets stochastically (random bits below the
 *     stored precision, from a per-node stream seeded by a hash of step and
 *     node, then truncation), so a change smaller than half a unit in the last place
 *     survives in expectation instead of being rounded away; results stay
 *     deterministic for a given run.
 *   LBM_FAST_TRANSFORMS: FP32 storage only, also for caller-supplied lattices
 *     (lbm_create_hermite).  By default FP32 runs on the Hermite lattices
 *     compute the 37 <-> 15 Hermite transforms (Eqs. an, fi) correctly rounded:
 *     FP32 constants rounded once leave the two transforms slightly off being
 *     inverses and plain FP32 sums round at every term, and both errors recur
 *     every step, so plain FP32 transforms drift by ~1e-5 relative on the
 *     velocity per 1000 steps; compensated (error-free) products and sums keep
 *     it at ~4e-7, at about four times the arithmetic (one node per thread).
 *     This flag selects the plain transforms and the two-node sweep instead. */
#define LBM_THERMAL 1u
#define LBM_K72 2u
#define LBM_RAW_MRT 4u
#define LBM_STOCHASTIC_ROUND 8u
#define LBM_FAST_TRANSFORMS 16u

/* Population storage.  Every type stores offsets from a rest equilibrium
 * f_ref,i (rho = 1, u = 0; theta = theta_ref on D2Q37, so f_ref,i = w_i when
 * theta_ref = 1): s_i = f_i - f_ref,i for FP64 / FP32 and
 * s_i = (f_i - f_ref,i) / w_i for FP16 / BF16 (round to nearest even). */
#define LBM_F64 0
#define LBM_F32 1
#define LBM_F16 2
#define LBM_BF16 3

/* Field element types for lbm_init_fields / lbm_moments. */
#define LBM_DTYPE_F64 0
#define LBM_DTYPE_F32 1

/* Status codes. */
#define LBM_OK 0
#define LBM_EINVAL (-1)    /* bad argument (lattice, dims, tau <= 1/2, null pointer, size) */
#define LBM_ECUDA (-2)     /* a CUDA runtime call failed */
#define LBM_EDIVERGED (-3) /* a node left the range the collision is defined on (lbm_status) */
#define LBM_ESIZE (-4)     /* a caller buffer is smaller than lbm_query_bytes asks */
#define LBM_ETIMEOUT (-5)  /* a bounded device-side wait (tensor-core completion) gave up; the
                              sweep that saw it skipped its remaining tiles */
#define LBM_EOOM (-6)      /* a host allocation of the library's own bookkeeping failed */

/* Bytes of the population buffer and of the workspace a simulation needs.
 * dims[2] must be 1 for a 2D lattice.  Limits: nx * ny * nz < 2^31,
 * ny <= 65535, nz <= 65535.  Host-only; no CUDA call. */
int lbm_query_bytes(int lattice, const int64_t dims[3], int storage, size_t* pop_bytes,
                    size_t* work_bytes);

/* Create a simulation on caller-owned device memory.
 *   tau_per_order[k] is the relaxation time of central-moment order k + 2
 *   (tau_2 sets the viscosity nu = c_s^2 (tau_2 - 1/2), Eq. sigma); orders past
 *   n_tau use tau = 1.  Every tau must exceed 1/2.
 *   pop / work: device buffers of at least the sizes lbm_query_bytes returns,
 *   256-byte aligned (any cudaMalloc or torch allocation is).
 * The populations are left undefined until lbm_init_fields or
 * lbm_set_populations; the workspace's status word is cleared. */
int lbm_create(int lattice, const int64_t dims[3], const double* tau_per_order, int n_tau,
               int storage, void* pop, size_t pop_bytes, void* work, size_t work_bytes,
               lbm_handle* out);

/* lbm_create with model flags (LBM_THERMAL | LBM_K72 | LBM_RAW_MRT, 37-velocity
 * lattice only; 0 elsewhere) and the offset base temperature theta_ref > 0
 * (1 on D2Q9 / D3Q27).  On D2Q37 tau_per_order = [tau_2, tau_3, tau_4]:
 * nu = theta (tau_2 - 1/2) and kappa = theta (tau_3 - 1/2) in the paper's units
 * (Eq. sigma), i.e. nu / c^2 and kappa / c^2 in lattice units. */
int lbm_create_ex(int lattice, const int64_t dims[3], const double* tau_per_order, int n_tau,
                  int storage, unsigned flags, double theta_ref, void* pop, size_t pop_bytes,
                  void* work, size_t work_bytes, lbm_handle* out);

/* Destroy the handle (host memory only; the caller frees its buffers). */
void lbm_destroy(lbm_handle h);

/* Stream for all later work of this handle (a cudaStream_t; NULL = default). */
int lbm_set_stream(lbm_handle h, void* stream);

/* Replace the relaxation times tau_n = 1 / omega_n of Eq. (omega), Sec. II.C
 * (same meaning and the same checks as in lbm_create: LBM_EINVAL for a tau
 * that is not above 1/2 or not finite).  Later steps use them. */
int lbm_set_tau(lbm_handle h, const double* tau_per_order, int n_tau);

/* Set every node to the equilibrium of the given fields (rho, u[D], theta) and
 * reset the step count to 0.  rho, u and theta are host (on_device = 0) or
 * device (on_device = 1) arrays of element type dtype; u in lattice units
 * (lattice spacings per step).  theta (the paper's dimensionless temperature)
 * is used on D2Q37 only and may be NULL (theta = 1).  Equilibria: central
 * moments rho * prod_d m_{alpha_d}, m = (1, 0, c_s^2) on D2Q9 / D3Q27; the
 * Maxwellian's Hermite coefficients up to order 4 on D2Q37 (Eq. fi). */
int lbm_init_fields(lbm_handle h, const void* rho, const void* u, const void* theta, int dtype,
                    int on_device);

/* Advance n >= 0 time steps: each is the collide-then-stream update of
 * Sec. II.C (Eq. omega, final update) in one sweep.  Asynchronous on the
 * handle's stream; n = 0 does nothing, n < 0 is LBM_EINVAL.  A node that turns
 * unphysical sets the status word (lbm_status) instead of stopping the run. */
int lbm_step(lbm_handle h, int64_t n);

/* Density, velocity (lattice units) and, if theta is not NULL, temperature at
 * the current time (Sec. II.A moment definitions: rho = sum_i f_i,
 * rho u = sum_i f_i e_i, rho (u^2 + 2 eps) = sum f xi^2 with eps = D theta / 2;
 * theta is written as 1 on isothermal runs and on D2Q9 / D3Q27).
 * Synchronises the stream.  Returns LBM_EDIVERGED if any sweep since the last
 * lbm_init_fields flagged a node. */
int lbm_moments(lbm_handle h, void* rho, void* u, void* theta, int dtype, int on_device);

/* The discrete distribution f_i (Sec. II.A) as FP64 absolute populations in
 * the natural layout above, to (get) or from (set) host (on_device = 0) or
 * device (on_device = 1) memory of Q * N doubles.  Set keeps the step count and
 * encodes into the storage type (rounding to 16-bit offsets where stored so).
 * Both synchronise the stream. */
int lbm_get_populations(lbm_handle h, double* f, int on_device);
int lbm_set_populations(lbm_handle h, const double* f, int on_device);

/* FP64 totals over the grid of the moments of Sec. II.A (mass and momentum
 * are conserved by the collision, Sec. II.C), written to host out[5]:
 *   out[0] = sum (rho - 1), out[1..3] = sum rho u_d (zero past D),
 *   out[4] = sum rho |u|^2 / 2.
 * Deterministic (fixed summation order).  Uses the workspace as scratch.
 * Synchronises the stream. */
int lbm_reduce(lbm_handle h, double out[5]);

/* One step (as lbm_step(h, 1)) that also returns the FP64 totals of the state
 * it advanced from (the quantities and order of lbm_reduce, as lbm_reduce
 * would give them just before the step, up to FP32 rounding: per node with
 * 16/32-bit storage, and in the sum over a warp's 64 nodes when the sweep
 * accumulates them).  Totals of a step's input, read back every step, are the
 * per-step result of a run (Sec. II.A moment definitions; conservation of mass
 * and momentum, Sec. II.C).  On the tensor-product lattices and the built-in
 * 37-velocity lattice with 16/32-bit storage and even nx the sweep accumulates
 * them itself (no extra pass over the populations); otherwise a reduction runs
 * before the sweep.  Synchronises the stream. */
int lbm_step_totals(lbm_handle h, double out[5]);

/* lbm_step_totals without waiting: the step and a copy of its totals to host
 * out[0..5) are enqueued on the handle's stream and the call returns.  The
 * exception to "buffers are never retained": out must stay valid until the
 * stream has passed this point, and holds the totals only from then on (after
 * any synchronising call such as lbm_status, or the caller's own stream
 * synchronisation).  With page-locked, 8-byte aligned out (cudaHostAlloc, a
 * pinned tensor) the GPU writes the totals there itself at the end of the
 * step, with no copy after it, so a run that logs its totals every step keeps
 * the GPU busy; other out gets an asynchronous copy on the stream (pageable
 * memory makes that copy wait for the step).  Errors of the enqueue are
 * returned; divergence shows in lbm_status. */
int lbm_step_totals_async(lbm_handle h, double* out);

/* lbm_reduce for callers that cannot allocate device memory.  The paper has no
 * counterpart; this is a deployment aid.  Some callers cannot call cudaMalloc:
 * a plugin inside a host application whose memory manager owns the whole
 * device, or a time-critical loop that cannot afford cudaMalloc's implicit
 * device-wide synchronisation.  They may hold a population buffer (pop, at
 * least lbm_query_bytes' pop_bytes, 256-byte aligned as lbm_create requires,
 * laid out as a simulation of the same lattice, dims and storage leaves it
 * after `step` steps) but no workspace.  The result is bitwise that of
 * lbm_reduce on the same state (same kernels, grid and summation order).
 * This call needs no handle and allocates nothing: its scratch is a fixed
 * 77,888-byte array in the library's own device memory (1216 block partials
 * of 8 doubles plus the result), which every GPU that loads the library holds
 * until the process exits.  The reduction strides over the grid, so that
 * scratch does not grow with it; grids beyond the library's limits (see
 * lbm_query_bytes), a misaligned or NULL pop, a negative step and too-small
 * pop_bytes are rejected (LBM_EINVAL / LBM_ESIZE) before any CUDA call.  Work runs on `stream` (a cudaStream_t; NULL = default), which
 * is synchronised before the host out[5] (same meaning as lbm_reduce) is
 * written.  The first call on a device looks up the array's device address
 * with that device current and keeps it; make that first call before any
 * stream capture.  The kept address assumes the device's context lives as
 * long as the process: it is not valid after cudaDeviceReset.
 * Every call shares the one array and leaves its last contents there: calls
 * that overlap on the GPU (other host threads, other streams) race and must
 * be serialised by the caller. */
int lbm_reduce_noalloc(int lattice, const int64_t dims[3], int storage, const void* pop,
                       size_t pop_bytes, int64_t step, void* stream, double out[5]);

/* Sweep a slab of planes only (D3Q27): lbm_step, lbm_step_totals(_async) and
 * lbm_reduce then work on the nodes of planes z_lo .. z_lo + z_count - 1 and
 * no others; every other call still covers the whole grid.  This is the local
 * part of a domain decomposition along z (Sec. II.A: streaming moves
 * populations by one node, so a slab needs one ghost plane on each side):
 * a rank holds its planes plus one ghost plane below and above (a grid of
 * nz_local + 2 planes, z_lo = 1, z_count = nz_local).  In the AA pattern only
 * the odd sweep reaches across planes: each boundary node reads and writes the
 * slots of the nine populations with e_z pointing out of the slab in the ghost
 * plane, so the caller copies the neighbour's boundary plane of those nine
 * populations into the ghost plane before an odd sweep and returns the ghost
 * plane to the neighbour after it (paper_1808_04406_gb300/slab.py).  Without a
 * wrap in z inside the range, the ghost planes must lie outside it.
 * z_lo = 0, z_count = nz restores the whole grid.  LBM_EINVAL for another
 * lattice, a range outside the grid, or a handle with the learned closure. */
int lbm_set_active_planes(lbm_handle h, int64_t z_lo, int64_t z_count);

/* Name of the sweep kernel that lbm_step launches for this handle with the
 * current settings (environment switches included), for example
 * "tp_pair_kernel" (two nodes per thread), "tp_pair_zrun_kernel" (the same
 * walking several planes per thread: D3Q27 with FP16 / BF16 offsets),
 * "tp_sweep_kernel" (one node per thread), "h37_pair_kernel", "learned_tc_kernel".  Measurement and tests only;
 * the string is static.  NULL for a NULL handle (no error code). */
const char* lbm_sweep_kernel(lbm_handle h);

/* Failure-detection self-test.  The paper has no counterpart; it exercises the
 * give-up path of the library's bounded device waits without a fault.  The
 * tensor-core sweeps wait on an mbarrier for their MMAs with a poll limit; a
 * wait that runs out sets the timeout bit of the handle's status word, and
 * lbm_status then returns LBM_ETIMEOUT.  This call enqueues, on the handle's
 * stream, one warp that runs that same bounded wait on an mbarrier nothing
 * ever arrives at (1 <= polls <= 2^20; nothing asynchronous is in flight and
 * no tensor memory is held), so the wait runs out, the kernel returns and the
 * bit is set.  The context stays usable: the next lbm_init_fields clears the
 * status.  LBM_EINVAL for a NULL handle or polls out of range. */
int lbm_selftest_wait_timeout(lbm_handle h, int polls);

/* Arithmetic-throughput probe: the measured denominator of the ALU rooflines
 * of the sweeps that arithmetic, not memory, binds (the 37-velocity lattice in
 * FP32 / packed FP32x2, D2Q9 in FP64).  The paper has no counterpart; this is
 * measurement only.  Enqueues one kernel on `stream` (a cudaStream_t; NULL =
 * default) of `blocks` x `threads` threads (threads a multiple of 32, at most
 * 1024), each running 8 independent chains of `iters` fused multiply-adds of
 * the kind given (LBM_PROBE_F32: scalar FP32 fma.rn.f32; LBM_PROBE_F32X2:
 * packed fma.rn.f32x2, two FP32 FMAs per instruction; LBM_PROBE_F64: fma.rn.f64)
 * on registers only, and returns at once; the caller times it (CUDA events on
 * the stream) and divides *flops (written on the host: 2 per FMA, all threads)
 * by the time.  sink: caller-owned device memory of at least 4 bytes, written
 * only under a condition no chain meets (it keeps the work from being removed).
 * LBM_EINVAL for an unknown kind, a bad shape or NULL pointers. */
#define LBM_PROBE_F32 0
#define LBM_PROBE_F32X2 1
#define LBM_PROBE_F64 2
int lbm_alu_probe(int kind, int iters, int blocks, int threads, void* sink, void* stream, double* flops);

/* Single-wavenumber Fourier amplitude of a field, Sec. III.A:
 *   A = sum_x q(x) exp(-2 pi i sum_d m_d x_d / L_d), FP64, written to host
 *   out[2] = {Re A, Im A}.  field: 0 = rho, 1 + d = u_d (lattice units); on
 *   D2Q37 also 3 = theta and 4 = p = rho theta.  Synchronises. */
int lbm_mode_amplitude(lbm_handle h, int field, const int64_t mode[3], double out[2]);

/* Wave-decay measurement of Sec. III.A: record the single-wavenumber amplitude
 * A_r of `field` (as lbm_mode_amplitude) at the current time and after every
 * further `stride` steps, n_records in all (2 <= n_records <= 4096; the
 * simulation advances (n_records - 1) * stride steps), then fit the modal form
 * A(t) = A(0) exp(omega t) (Eq. modes) in FP64 on the device by least squares
 * of ln|A_r| and of the unwrapped phase of A_r against t_r = r * stride:
 *   fit[0] = decay rate -Re(omega) per step (|A| ~ exp(-fit[0] t)),
 *   fit[1] = angular frequency Im(omega) in rad per step,
 *   fit[2] = fitted ln|A(0)|, fit[3] = fitted phase at t = 0.
 * For the viscous mode (field u_perp) Eq. dr gives fit[0] = nu k^2.
 * amplitudes (nullable, host) receives {Re A_r, Im A_r} pairs.  Uses the
 * workspace; synchronises; returns LBM_EDIVERGED (fit still written) if a node
 * diverged. */
int lbm_mode_history(lbm_handle h, int field, const int64_t mode[3], int n_records, int64_t stride,
                     double* amplitudes, double fit[4]);

/* Steps taken since the last lbm_init_fields. */
int64_t lbm_step_count(lbm_handle h);

/* Divergence flag: reads the device status word (synchronises); LBM_OK or
 * LBM_EDIVERGED.  A sweep flags a node where the moments of Sec. II.A leave
 * the range the collision is defined on: rho <= 0 or |u|^2 >= 1 in lattice
 * units on D2Q9 / D3Q27; rho <= 0, theta <= 0 or |u|^2 >= 4 in Hermite units on
 * D2Q37; or any NaN.  LBM_ETIMEOUT reports a bounded device wait that gave up
 * (the learned sweep's wait for tensor-core completion). */
int lbm_status(lbm_handle h);

/* ---- Batches of independent runs ----------------------------------------
 * Many independent periodic D2Q9 CM-MRT runs of different sizes advance
 * together, one kernel launch per step for the whole batch (a grid-stride walk
 * over a tile list; the launch boundary is the step barrier).  Each run keeps
 * its own AA-layout slice of one caller-owned population buffer.  A run whose
 * nodes go unphysical is flagged and skipped from then on; the others are not
 * affected.  The paper has no counterpart (its runs are single grids); the
 * per-run step is the same CM-MRT sweep as lbm_step. */
typedef struct lbm_batch* lbm_batch_handle;

/* Sizes for n_runs runs; dims[3 r + 0..2] = (nx_r, ny_r, 1).  Host-only. */
int lbm_batch_query_bytes(int lattice, int n_runs, const int64_t* dims, int storage,
                          size_t* pop_bytes, size_t* work_bytes);

/* Create a batch (lattice LBM_D2Q9).  tau_per_order[r * n_tau + k] is run r's
 * relaxation time of order k + 2 (orders past n_tau: tau = 1).  The tile shape
 * starts at 128 threads x 1 row; see lbm_batch_autotune. */
int lbm_batch_create(int lattice, int n_runs, const int64_t* dims, const double* tau_per_order,
                     int n_tau, int storage, void* pop, size_t pop_bytes, void* work,
                     size_t work_bytes, lbm_batch_handle* out);
void lbm_batch_destroy(lbm_batch_handle b);
int lbm_batch_set_stream(lbm_batch_handle b, void* stream);

/* Initialise run `run` to the equilibrium of its fields (rho[N_r], u[2][N_r],
 * lattice units), as lbm_init_fields; only before the batch's first step. */
int lbm_batch_init_run(lbm_batch_handle b, int run, const void* rho, const void* u, int dtype,
                       int on_device);

/* Initialise every run at once: rho[r], u[r] are run r's fields as for
 * lbm_batch_init_run (n_runs pointers in each array, one dtype for all).  When
 * all of them are device memory (on_device = 1) or page-locked host memory,
 * one kernel reads them all where they are and the call synchronises once;
 * otherwise each run goes through lbm_batch_init_run.  The populations equal
 * those of lbm_batch_init_run bit for bit.  LBM_EINVAL for NULL arrays or
 * pointers, an unknown dtype, or a batch that has taken a step. */
int lbm_batch_init_runs(lbm_batch_handle b, const void* const* rho, const void* const* u, int dtype,
                        int on_device);

/* Advance every run n steps, each the update of Sec. II.C as in lbm_step
 * (asynchronous; n < 0 is LBM_EINVAL).  With lbm_batch_use_graph(b, 1)
 * pairs of steps are replayed from a captured two-step CUDA graph; that needs a
 * non-default stream (LBM_EINVAL otherwise). */
int lbm_batch_step(lbm_batch_handle b, int64_t n);
int lbm_batch_use_graph(lbm_batch_handle b, int enable);

/* Tile shape: threads per block (64, 128, 256) and rows per tile (1, 2, 4, 8,
 * 16).  With 16/32-bit storage a thread holds two nodes in packed FP32x2:
 * x-neighbours when nx is even, (x, y) and (x, y + 1) when nx is odd (a tile
 * then covers 2 x rows rows); FP64 runs take one node per thread.  Results do
 * not depend on the shape. */
int lbm_batch_set_tiles(lbm_batch_handle b, int threads, int rows);

/* Launch mode.  staged = k >= 1 (default 1): runs with 16/32-bit storage whose
 * rows fit a band (nx <= 4096 and nx <= band capacity) advance through shared
 * memory, in bands of whole rows moved by bulk asynchronous copies, one launch
 * per step for all of them, with launch shape k (updating threads, stages x
 * bytes per population and stage, CTAs per SM; 1: 256, 2 x 6 KB, 2;
 * 2: 256, 3 x 4 KB, 2; 3: 512, 2 x 12 KB, 1; 4: 512, 3 x 8 KB, 1); the other
 * runs go through the tile sweep.  staged = 0: every run goes through the tile
 * sweep.  Tile sweep: split = 0: one launch per step covers every tile;
 * split = 1: one launch per kind of run (x-neighbour pairs, column pairs,
 * single nodes), each kernel specialised to its kind; depth = 1 or 2: how many
 * rows' loads a thread keeps in flight while it collides a row (node pairs
 * only).  Results do not depend on the mode. */
int lbm_batch_set_launch(lbm_batch_handle b, int split, int depth, int staged);

/* The current tile shape and launch mode (any output pointer may be NULL). */
int lbm_batch_get_launch(lbm_batch_handle b, int* threads, int* rows, int* split, int* depth, int* staged);

/* Time every tile shape in every launch mode for steps_per_trial steps and keep
 * the fastest (the tile shape written to *threads, *rows).  Runs on the rest state and leaves every run at rest:
 * call it before lbm_batch_init_run.  With the environment variable
 * LBM_AUTOTUNE_CACHE naming a file, results are looked up there first and
 * appended after a search. */
int lbm_batch_autotune(lbm_batch_handle b, int steps_per_trial, int* threads, int* rows);

/* Per-run status (host flags[n_runs]: LBM_OK or LBM_EDIVERGED); synchronises. */
int lbm_batch_status(lbm_batch_handle b, int* flags);

/* Per-run FP64 totals (host out[5 * n_runs], the quantities of lbm_reduce;
 * one launch for all runs, each run's nodes added in a fixed order, so the
 * totals are deterministic but may differ from a single-grid lbm_reduce of the
 * same run in the last bits); synchronises. */
int lbm_batch_reduce(lbm_batch_handle b, double* out);

/* Fields and FP64 populations of one run, as lbm_moments / lbm_get_populations. */
int lbm_batch_moments(lbm_batch_handle b, int run, void* rho, void* u, int dtype, int on_device);
int lbm_batch_get_populations(lbm_batch_handle b, int run, double* f, int on_device);
int64_t lbm_batch_step_count(lbm_batch_handle b);

/* ---- Learned relaxation-rate closure (D3Q27) ------------------------------
 * Sec. II.C, after Eq. omega: every central moment relaxes at its own rate
 * and only omega_2 (shear and bulk viscosity) is fixed by the transport
 * coefficients; the rates of orders 3..6 are free.  The closure picks them
 * per node with a 20 -> 64 -> 64 -> 6 network (ReLU, ReLU,
 * omega = omega_lo + (omega_hi - omega_lo) sigmoid(z); 0 and 2 span every rate
 * Eq. omega allows), one rate per permutation class of alpha:
 *   3:(2,1,0)  3:(1,1,1)  4:(2,2,0)  4:(2,1,1)  5:(2,2,1)  6:(2,2,2).
 * Inputs: the 19 non-equilibrium central moments of orders 2..4 of the node,
 * each divided by rho c_s^n, and tau_2 - 1/2, standardised as
 * (x - mean[j]) * inv_std[j].  The network runs in BF16 on tensor cores with
 * FP32 accumulation.
 *
 * Parameter vector (FP32, 5894 values, device memory):
 *   W1[20][64], b1[64], W2[64][64], b2[64], W3[64][6], b3[6]
 * with W[k][n] the weight from input k to output n.
 * Standardisation vector (FP32, 40 values, device memory): mean[20], inv_std[20]. */
#define LBM_MLP_PARAMS 5894

/* Relax orders 3..6 of every later lbm_step at the network's rates; order 2
 * keeps omega_2 from the relaxation times.  D3Q27 with FP32 storage only
 * (LBM_EINVAL otherwise; also for a range outside 0 <= omega_lo < omega_hi <= 2).
 * params / norm are copied (synchronously) into the simulation's workspace;
 * the caller keeps ownership.  params == NULL switches the closure off again. */
int lbm_set_closure(lbm_handle h, const float* params, const float* norm, double omega_lo, double omega_hi);

/* Box filter onto a grid m times coarser (D3Q27, any storage): out[27 * Nc]
 * (device, FP32, population-major, x fastest, Nc = (nx/m)(ny/m)(nz/m)) holds
 * the mean over each m^3 block of the population offsets f_i - w_i of the
 * current state.  m must divide every dimension.  Asynchronous on the
 * simulation's stream. */
int lbm_closure_filter(lbm_handle h, int m, float* out);

/* In place, per node of a periodic FP32 offset field f[27 * N] (device,
 * N = dims[0] dims[1] dims[2]): f <- f^eq(rho, u) + scale (f - f^eq(rho, u)),
 * i.e. a collision with omega = 1 - scale at every order >= 2.  A fine state
 * box-filtered m-fold holds tau_f / (m tau_c) of the coarse model's first-order
 * non-equilibrium (Chapman-Enskog: f^(1) = -tau dt D f^(0)); scale = m tau_c / tau_f
 * makes it a coarse-model state.  Asynchronous. */
int lbm_closure_rescale(const int64_t dims[3], float* f, double scale, void* stream);

/* Training samples from two coarse states one coarse step apart (device,
 * FP32 offsets [27 * N] as written by lbm_closure_filter, N = dims[0] dims[1]
 * dims[2], periodic).  Per node k:
 *   X[20 k + j]   standardised features (norm as above);
 *   abc[18 k + 3 c + {0, 1, 2}] = A_c, B_c, C_c = sums over the moments of class c
 *   of k1^2, k1 k1*, k1*^2, where k1 is the node's scaled non-equilibrium
 *   central moment and k1* that of the ideal post-collision state, the
 *   populations of f_t1 pulled back along their velocity,
 *   f*_i(x) = f_t1,i(x + e_i), taken about that state's own velocity.
 * tau2 is the second-order relaxation time of the coarse model.  stream is a
 * cudaStream_t (NULL: legacy default stream).  Asynchronous. */
int lbm_closure_dataset(const int64_t dims[3], const float* f_t, const float* f_t1, double tau2,
                        const float* norm, float* X, float* abc, void* stream);

/* Device workspace needed by the two calls below for a batch of `batch`
 * samples (0 for batch < 1).  The workspace must be 256-byte aligned. */
size_t lbm_mlp_work_bytes(int64_t batch);

/* Loss L = (1/n) sum_k sum_c cw[c] ((1 - omega_c)^2 A_c - 2 (1 - omega_c) B_c + C_c)
 * over all n samples and its gradient with respect to the parameters, with the
 * rates in [omega_lo, omega_hi] as above.  X, abc, params, grad (5894 floats,
 * may be NULL) and work are device pointers; cw (6 class weights) and loss (may
 * be NULL) are host pointers.  The sums run in a fixed order (deterministic).
 * Synchronises the stream. */
int lbm_mlp_loss_grad(const float* X, const float* abc, int64_t n, const float* cw, double omega_lo,
                      double omega_hi, const float* params, float* grad, double* loss, void* work,
                      size_t work_bytes, void* stream);

/* `iters` Adam steps (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr) on
 * mini-batches of `batch` samples drawn with replacement from the n samples by
 * a counter-based hash of (seed, t0 + iteration, slot).  params, adam_m and
 * adam_v (5894 floats each, device) are updated in place; t0 is the number of
 * Adam steps already taken (bias correction).  loss_hist (device, iters
 * floats, may be NULL) receives each mini-batch loss.  cw is a host pointer.
 * Asynchronous. */
int lbm_mlp_train(const float* X, const float* abc, int64_t n, const float* cw, double omega_lo, double omega_hi,
                  float* params, float* adam_m, float* adam_v, int64_t iters, int64_t batch, double lr,
                  uint64_t seed, int64_t t0, float* loss_hist, void* work, size_t work_bytes, void* stream);

/* ---- Caller-supplied Hermite lattices (Sec. III.A, Fig. 2) -----------------
 * The CM-MRT of Sec. II.C on any square-symmetric two-dimensional velocity set
 * xi_i = c e_i (integer e with |e_x|, |e_y| <= 3) with weights w_i, Hermite
 * expansion and equilibrium truncated at order N (Eqs. fi, reg, omega; the
 * 4th-order coupling K = 6 when N = 4).  Supported shapes: 17 velocities with
 * N = 3 (the minimal degree-7 rules) and 37 velocities with N = 3 or 4 (the
 * minimal degree-9 rules).  The rule must integrate the unit Gaussian exactly
 * to degree 2N (checked; LBM_EINVAL otherwise), every velocity needs its
 * opposite.  Storage FP64 or FP32 offsets from f_eq(1, 0, theta_ref); flags
 * LBM_THERMAL or 0.  The handle then takes every single-simulation call of
 * this header (fields with theta, populations in the caller's velocity order,
 * totals, mode amplitudes and fits with fields 0..4 as on LBM_D2Q37) except
 * the learned closure and lbm_reduce_noalloc.  tau_per_order: orders 2..N. */
int lbm_hermite_query_bytes(int q, const int64_t dims[3], int storage, size_t* pop_bytes,
                            size_t* work_bytes);
int lbm_create_hermite(int q, const int* e /* [2 q]: e_x, e_y per velocity */, const double* w, double c,
                       int order, const int64_t dims[3], const double* tau_per_order, int n_tau,
                       int storage, unsigned flags, double theta_ref, void* pop, size_t pop_bytes,
                       void* work, size_t work_bytes, lbm_handle* out);

/* Message of the last failed call on this thread ("" if none). */
const char* lbm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
