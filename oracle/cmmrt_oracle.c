/*
 * FP64 CPU oracle for the central-moment multiple-relaxation-time (CM-MRT)
 * lattice Boltzmann step on the tensor-product lattices D2Q9 and D3Q27.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA path is checked against.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header, table
 * or constant generator with the CUDA library; the library never links it.
 *
 * What it computes (X. Shan, "A central-moment multiple-relaxation-time
 * collision model", arXiv:1808.04406):
 *   - Sec. II.A, Eq. (an) and the moment definitions: rho = sum f_i,
 *     rho u = sum f_i xi_i.
 *   - Sec. II.C, Eq. (omega): every central moment of order n of the
 *     collision term equals -omega_n times the same central moment of the
 *     non-equilibrium part f^(1) = f - f^(0).  Orders 0 and 1 of Omega vanish
 *     (mass and momentum conservation).
 *   - Sec. II.C, last equation: f_i(x + xi_i, t + 1) = f_i^ + Omega_i.  The
 *     tensor-product basis is complete, so f^ = f here.
 *
 * Reading used where the paper is silent (the paper runs D2Q9 only with BGK):
 *   the moment basis on D1Q3^D is the set of central monomials
 *   prod_d (e_id - u_d)^{alpha_d} with alpha_d in {0,1,2}; the order of a
 *   moment is |alpha| = sum_d alpha_d; the equilibrium central moments are
 *   rho * prod_d m_{alpha_d} with m_0 = 1, m_1 = 0, m_2 = c_s^2 = 1/3
 *   (the isothermal Maxwellian restricted to the lattice's basis).
 *
 * The step is computed by definition, node by node:
 *   1. rho, u from f;
 *   2. the central-moment matrix C(u)_{a,i} = prod_d (e_id - u_d)^{alpha_d(a)};
 *   3. kappa = C f, kappa_eq = rho prod m;
 *   4. kappa*_a = kappa_a - omega_{|a|} (kappa_a - kappa_eq_a) for |a| >= 2,
 *      kappa*_a = kappa_a for |a| <= 1;
 *   5. f* solves C(u) f* = kappa* (Gaussian elimination with partial
 *      pivoting on the full Q x Q system, variant ORC_DEFINITIONAL) or
 *      f* = C(u)^{-1} kappa* with C^{-1} built as the Kronecker product of the
 *      three 3x3 inverses, (A (x) B)^{-1} = A^{-1} (x) B^{-1} (variant
 *      ORC_KRONECKER, the same map in O(Q^2) per node);
 *   6. stream: f_i(x + e_i) <- f*_i(x) with periodic wrap (two arrays).
 * An independent LBGK step (Sec. II.A, Eq. lbgk) with the product-form
 * equilibrium is variant ORC_LBGK; with all omega_n equal the CM-MRT step
 * must reproduce it (Sec. II.C, remark after Eq. regnmrt).
 *
 * Layout: f[i * N + node], node = x + nx * (y + ny * z), velocity index
 * i = sum_d (e_id + 1) * 3^d.  Compiled with -ffp-contract=off.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_DEFINITIONAL 0
#define ORC_KRONECKER 1
#define ORC_LBGK 2

#define ORC_QMAX 27

static const double CS2 = 1.0 / 3.0;

static int pow3(int d) {
    int p = 1;
    for (int k = 0; k < d; ++k) p *= 3;
    return p;
}

/* Base-3 digits of the indices 0..26, filled once at load time:
 * velocity component e_id = digit_d(i) - 1, moment exponent alpha_d(a) = digit_d(a). */
static int digit_tab[ORC_QMAX][3];

__attribute__((constructor)) static void fill_digit_tab(void) {
    for (int i = 0; i < ORC_QMAX; ++i)
        for (int d = 0; d < 3; ++d) digit_tab[i][d] = (i / pow3(d)) % 3;
}

static int tp_e(int i, int d) { return digit_tab[i][d] - 1; }

static int tp_alpha(int a, int d) { return digit_tab[a][d]; }

static double ipow(double x, int k) {
    double r = 1.0;
    for (int j = 0; j < k; ++j) r *= x;
    return r;
}

/* 1D Gauss-Hermite three-point weights in lattice units: 2/3 at rest, 1/6 moving */
static double w1(int e) { return e == 0 ? 2.0 / 3.0 : 1.0 / 6.0; }

int orc_tp_weight(int D, double* w) {
    int Q = pow3(D);
    for (int i = 0; i < Q; ++i) {
        double p = 1.0;
        for (int d = 0; d < D; ++d) p *= w1(tp_e(i, d));
        w[i] = p;
    }
    return Q;
}

int orc_tp_velocities(int D, int* e /* Q x D */) {
    int Q = pow3(D);
    for (int i = 0; i < Q; ++i)
        for (int d = 0; d < D; ++d) e[i * D + d] = tp_e(i, d);
    return Q;
}

/* Solve A x = b in place (A is n x n row-major, destroyed; b becomes x).
 * Gaussian elimination with partial pivoting.  Returns 0, or -1 if singular. */
static int gauss_solve(int n, double* A, double* b) {
    for (int k = 0; k < n; ++k) {
        int p = k;
        double best = fabs(A[k * n + k]);
        for (int r = k + 1; r < n; ++r) {
            double v = fabs(A[r * n + k]);
            if (v > best) { best = v; p = r; }
        }
        if (best == 0.0) return -1;
        if (p != k) {
            for (int c = 0; c < n; ++c) {
                double t = A[k * n + c]; A[k * n + c] = A[p * n + c]; A[p * n + c] = t;
            }
            double t = b[k]; b[k] = b[p]; b[p] = t;
        }
        for (int r = k + 1; r < n; ++r) {
            double m = A[r * n + k] / A[k * n + k];
            if (m == 0.0) continue;
            for (int c = k; c < n; ++c) A[r * n + c] -= m * A[k * n + c];
            b[r] -= m * b[k];
        }
    }
    for (int k = n - 1; k >= 0; --k) {
        double s = b[k];
        for (int c = k + 1; c < n; ++c) s -= A[k * n + c] * b[c];
        b[k] = s / A[k * n + k];
    }
    return 0;
}

/* macroscopic density and velocity of one node (Sec. II.A moment definitions) */
static void tp_rho_u(int D, const double* f, double* rho, double* u) {
    int Q = pow3(D);
    double r = 0.0, j[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < Q; ++i) {
        r += f[i];
        for (int d = 0; d < D; ++d) j[d] += f[i] * (double)tp_e(i, d);
    }
    *rho = r;
    for (int d = 0; d < D; ++d) u[d] = j[d] / r;
}

/* C(u)_{a,i} = prod_d (e_id - u_d)^{alpha_d(a)} */
static void tp_central_matrix(int D, const double* u, double* C) {
    int Q = pow3(D);
    for (int a = 0; a < Q; ++a)
        for (int i = 0; i < Q; ++i) {
            double p = 1.0;
            for (int d = 0; d < D; ++d) p *= ipow((double)tp_e(i, d) - u[d], tp_alpha(a, d));
            C[a * Q + i] = p;
        }
}

/* equilibrium central moment rho * prod_d m_{alpha_d}, m = (1, 0, c_s^2) */
static double tp_keq(int D, int a, double rho) {
    double p = rho;
    for (int d = 0; d < D; ++d) {
        int al = tp_alpha(a, d);
        p *= (al == 0) ? 1.0 : (al == 1 ? 0.0 : CS2);
    }
    return p;
}

static int tp_order(int D, int a) {
    int n = 0;
    for (int d = 0; d < D; ++d) n += tp_alpha(a, d);
    return n;
}

/* Product-form LBGK equilibrium: f_eq_i = rho prod_d g(e_id, u_d),
 * g(0,u) = 1 - c_s^2 - u^2, g(+-1,u) = (c_s^2 + u^2 +- u) / 2.
 * Written independently of the central-moment machinery. */
static double g1(int e, double u) {
    if (e == 0) return 1.0 - CS2 - u * u;
    return 0.5 * (CS2 + u * u + (double)e * u);
}

/* One node of the collision.  omega[n], n = 0..2D, is the rate of order n. */
int orc_tp_collide_node(int D, const double* omega, int variant, const double* f, double* out) {
    int Q = pow3(D);
    double rho, u[3] = {0.0, 0.0, 0.0};
    tp_rho_u(D, f, &rho, u);
    if (variant == ORC_LBGK) {
        double om = omega[2];
        for (int i = 0; i < Q; ++i) {
            double feq = rho;
            for (int d = 0; d < D; ++d) feq *= g1(tp_e(i, d), u[d]);
            out[i] = f[i] + om * (feq - f[i]);
        }
        return 0;
    }
    double C[ORC_QMAX * ORC_QMAX];
    double kap[ORC_QMAX], kstar[ORC_QMAX];
    tp_central_matrix(D, u, C);
    for (int a = 0; a < Q; ++a) {
        double s = 0.0;
        for (int i = 0; i < Q; ++i) s += C[a * Q + i] * f[i];
        kap[a] = s;
    }
    for (int a = 0; a < Q; ++a) {
        int n = tp_order(D, a);
        if (n <= 1)
            kstar[a] = kap[a];
        else
            kstar[a] = kap[a] - omega[n] * (kap[a] - tp_keq(D, a, rho));
    }
    if (variant == ORC_DEFINITIONAL) {
        memcpy(out, kstar, sizeof(double) * (size_t)Q);
        return gauss_solve(Q, C, out);
    }
    /* ORC_KRONECKER: C^{-1}_{i,a} = prod_d C1_d^{-1}[i_d][alpha_d] */
    double inv[3][9];
    for (int d = 0; d < D; ++d) {
        for (int col = 0; col < 3; ++col) {
            double A[9], b[3] = {0.0, 0.0, 0.0};
            for (int al = 0; al < 3; ++al)
                for (int k = 0; k < 3; ++k) A[al * 3 + k] = ipow((double)(k - 1) - u[d], al);
            b[col] = 1.0;
            if (gauss_solve(3, A, b)) return -1;
            for (int k = 0; k < 3; ++k) inv[d][k * 3 + col] = b[k];
        }
    }
    for (int i = 0; i < Q; ++i) {
        double s = 0.0;
        for (int a = 0; a < Q; ++a) {
            double p = 1.0;
            for (int d = 0; d < D; ++d) p *= inv[d][(tp_e(i, d) + 1) * 3 + tp_alpha(a, d)];
            s += p * kstar[a];
        }
        out[i] = s;
    }
    return 0;
}

/* Collision with one rate per central moment: omega_a[a] for every moment a
 * (orders 0 and 1 are never relaxed); same definitional solve as above. */
int orc_tp_collide_node_rates(int D, const double* omega_a, const double* f, double* out) {
    int Q = pow3(D);
    double rho, u[3] = {0.0, 0.0, 0.0};
    tp_rho_u(D, f, &rho, u);
    double C[ORC_QMAX * ORC_QMAX];
    tp_central_matrix(D, u, C);
    for (int a = 0; a < Q; ++a) {
        double s = 0.0;
        for (int i = 0; i < Q; ++i) s += C[a * Q + i] * f[i];
        out[a] = tp_order(D, a) <= 1 ? s : s - omega_a[a] * (s - tp_keq(D, a, rho));
    }
    return gauss_solve(Q, C, out);
}

/* Equilibrium populations from (rho, u) by definition: f_eq = C(u)^{-1} kappa_eq. */
int orc_tp_equilibrium_node(int D, double rho, const double* u, double* f) {
    int Q = pow3(D);
    double C[ORC_QMAX * ORC_QMAX];
    double uu[3] = {0.0, 0.0, 0.0};
    for (int d = 0; d < D; ++d) uu[d] = u[d];
    tp_central_matrix(D, uu, C);
    for (int a = 0; a < Q; ++a) f[a] = tp_keq(D, a, rho);
    return gauss_solve(Q, C, f);
}

/* Product-form equilibrium (the LBGK one), for the equal-rate pin. */
int orc_tp_product_equilibrium_node(int D, double rho, const double* u, double* f) {
    int Q = pow3(D);
    for (int i = 0; i < Q; ++i) {
        double p = rho;
        for (int d = 0; d < D; ++d) p *= g1(tp_e(i, d), u[d]);
        f[i] = p;
    }
    return 0;
}

/* Central moments kappa_a = sum_i f_i prod_d (e_id - u_d)^alpha_d of one node about u. */
int orc_tp_central_moments_node(int D, const double* u, const double* f, double* kap) {
    int Q = pow3(D);
    double C[ORC_QMAX * ORC_QMAX];
    double uu[3] = {0.0, 0.0, 0.0};
    for (int d = 0; d < D; ++d) uu[d] = u[d];
    tp_central_matrix(D, uu, C);
    for (int a = 0; a < Q; ++a) {
        double s = 0.0;
        for (int i = 0; i < Q; ++i) s += C[a * Q + i] * f[i];
        kap[a] = s;
    }
    return 0;
}

/* Field equilibrium: f[i*N + n] from rho[n], u[d*N + n]. */
int orc_tp_init(int D, int64_t N, const double* rho, const double* u, double* f) {
    int Q = pow3(D);
    int err = 0;
#pragma omp parallel for schedule(static) reduction(| : err)
    for (int64_t n = 0; n < N; ++n) {
        double uu[3] = {0.0, 0.0, 0.0}, fl[ORC_QMAX];
        for (int d = 0; d < D; ++d) uu[d] = u[(int64_t)d * N + n];
        err |= orc_tp_equilibrium_node(D, rho[n], uu, fl) ? 1 : 0;
        for (int i = 0; i < Q; ++i) f[(int64_t)i * N + n] = fl[i];
    }
    return err ? -1 : 0;
}

int orc_tp_moments(int D, int64_t N, const double* f, double* rho, double* u) {
    int Q = pow3(D);
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < N; ++n) {
        double fl[ORC_QMAX], r, uu[3];
        for (int i = 0; i < Q; ++i) fl[i] = f[(int64_t)i * N + n];
        tp_rho_u(D, fl, &r, uu);
        rho[n] = r;
        for (int d = 0; d < D; ++d) u[(int64_t)d * N + n] = uu[d];
    }
    return 0;
}

/* Collide every node (f -> post), then stream post back into f with periodic wrap. */
int orc_tp_step(int D, const int64_t* dims, const double* omega, int variant, double* f,
                double* post, int64_t nsteps) {
    int Q = pow3(D);
    int64_t nx = dims[0], ny = dims[1], nz = D == 3 ? dims[2] : 1;
    int64_t N = nx * ny * nz;
    for (int64_t s = 0; s < nsteps; ++s) {
        int err = 0;
#pragma omp parallel for schedule(static) reduction(| : err)
        for (int64_t n = 0; n < N; ++n) {
            double fl[ORC_QMAX], fo[ORC_QMAX];
            for (int i = 0; i < Q; ++i) fl[i] = f[(int64_t)i * N + n];
            err |= orc_tp_collide_node(D, omega, variant, fl, fo) ? 1 : 0;
            for (int i = 0; i < Q; ++i) post[(int64_t)i * N + n] = fo[i];
        }
        if (err) return -1;
#pragma omp parallel for schedule(static)
        for (int64_t n = 0; n < N; ++n) {
            int64_t x = n % nx, y = (n / nx) % ny, z = n / (nx * ny);
            for (int i = 0; i < Q; ++i) {
                int64_t xd = (x + tp_e(i, 0) + nx) % nx;
                int64_t yd = (y + tp_e(i, 1) + ny) % ny;
                int64_t zd = D == 3 ? (z + tp_e(i, 2) + nz) % nz : 0;
                f[(int64_t)i * N + xd + nx * (yd + ny * zd)] = post[(int64_t)i * N + n];
            }
        }
    }
    return 0;
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
