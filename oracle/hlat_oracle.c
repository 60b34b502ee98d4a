/*
 * FP64 CPU oracle for the thermal / isothermal CM-MRT step on any
 * square-symmetric two-dimensional Hermite lattice (up to 37 velocities,
 * Hermite projection and equilibrium truncation N = M = 3 or 4), written from
 * X. Shan, arXiv:1808.04406.
 *
 * TEST INFRASTRUCTURE ONLY: the checker of the CUDA path; shares nothing with
 * it.  The lattice (velocities, weights, scale c with xi_i = c e_i), the
 * truncation order and the Gauss-Hermite points used to integrate the
 * Maxwellian are handed in by hl_setup into a caller-owned context, so several
 * lattices can be used side by side.
 *
 * Definitions used (as in the 37-velocity oracle):
 *   - tensor Hermite polynomials by the recursion of the Appendix, full
 *     (unsymmetrised) 2^n-component tensors, n <= N;
 *   - a^(n) = sum_i f_i H^(n)(xi_i) (Eq. an); f_i = w_i sum_n (1/n!) a^(n) : H^(n)(xi_i)
 *     (Eq. fi);
 *   - rho, u, and theta from rho (u^2 + 2 eps) = sum f xi^2, eps = D theta / 2
 *     (Sec. II.A); isothermal runs freeze theta = 1;
 *   - f^(0): the Maxwellian projected onto n <= N, its coefficients by
 *     Gauss-Hermite quadrature of the Maxwellian itself;
 *   - f^(1) = f - f^(0); f^ (1) = sum_{n<=N} M^(n) f^(1) (Eqs. m, reg);
 *   - the collision of Sec. II.C: Omega has no components above order N, its
 *     central moments of order n equal -omega_n times those of f^ (1) for all
 *     |alpha| <= N (Eq. omega), zero for orders 0 and 1; solved node by node
 *     as a linear system over the (N + 1)(N + 2) / 2 symmetric components;
 *   - update f_i(x + e_i, t + 1) = f^_i + Omega_i with f^ = f^(0) + f^ (1).
 * Layout f[i * Nn + node], node = x + nx * y.  Compiled with -ffp-contract=off.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <string.h>

#define HL_QMAX 37
#define HL_NTMAX 31 /* full tensor components of orders 0..4 */
#define HL_NAMAX 15 /* symmetric components x^p y^q, p + q <= 4 */

typedef struct {
    int q, nmax, nt, na, ngh;
    int E[HL_QMAX][2];
    double W[HL_QMAX];
    double XI[HL_QMAX][2];
    double HT[HL_QMAX][HL_NTMAX];
    double GHX[16], GHW[16];
    int ALPHA[HL_NAMAX][2];
} hl_ctx;

size_t hl_ctx_bytes(void) { return sizeof(hl_ctx); }

static int off(int n) { return (1 << n) - 1; }

static double fact(int n) {
    double r = 1.0;
    for (int k = 2; k <= n; ++k) r *= k;
    return r;
}

/* Hermite tensors of orders 0..nmax at xi (full components, offset off(n)) */
static void hermite_full(const double xi[2], int nmax, double* H) {
    H[0] = 1.0;
    for (int n = 0; n < nmax; ++n)
        for (int t = 0; t < (1 << n); ++t)
            for (int j = 0; j < 2; ++j) {
                double v = xi[j] * H[off(n) + t];
                for (int k = 0; k < n; ++k)
                    if (((t >> k) & 1) == j) {
                        int tr = (t & ((1 << k) - 1)) | ((t >> (k + 1)) << k);
                        v -= H[off(n - 1) + tr];
                    }
                H[off(n + 1) + (t | (j << n))] = v;
            }
}

int hl_setup(void* vctx, int q, const int* e, const double* w, double c, int nmax, int ngh, const double* ghx,
             const double* ghw) {
    hl_ctx* C = (hl_ctx*)vctx;
    if (q < 1 || q > HL_QMAX || nmax < 2 || nmax > 4 || ngh < 1 || ngh > 16) return -1;
    C->q = q;
    C->nmax = nmax;
    C->nt = off(nmax + 1);
    C->na = (nmax + 1) * (nmax + 2) / 2;
    for (int i = 0; i < q; ++i) {
        C->E[i][0] = e[2 * i];
        C->E[i][1] = e[2 * i + 1];
        C->W[i] = w[i];
        C->XI[i][0] = c * e[2 * i];
        C->XI[i][1] = c * e[2 * i + 1];
        hermite_full(C->XI[i], nmax, C->HT[i]);
    }
    C->ngh = ngh;
    for (int k = 0; k < ngh; ++k) {
        C->GHX[k] = ghx[k];
        C->GHW[k] = ghw[k];
    }
    int a = 0;
    for (int n = 0; n <= nmax; ++n)
        for (int p = n; p >= 0; --p) {
            C->ALPHA[a][0] = p;
            C->ALPHA[a][1] = n - p;
            ++a;
        }
    return 0;
}

static int gauss_solve(int n, double* A, double* b) {
    for (int k = 0; k < n; ++k) {
        int p = k;
        double best = fabs(A[k * n + k]);
        for (int r = k + 1; r < n; ++r)
            if (fabs(A[r * n + k]) > best) {
                best = fabs(A[r * n + k]);
                p = r;
            }
        if (best == 0.0) return -1;
        if (p != k) {
            for (int cc = 0; cc < n; ++cc) {
                double t = A[k * n + cc];
                A[k * n + cc] = A[p * n + cc];
                A[p * n + cc] = t;
            }
            double t = b[k];
            b[k] = b[p];
            b[p] = t;
        }
        for (int r = k + 1; r < n; ++r) {
            double m = A[r * n + k] / A[k * n + k];
            for (int cc = k; cc < n; ++cc) A[r * n + cc] -= m * A[k * n + cc];
            b[r] -= m * b[k];
        }
    }
    for (int k = n - 1; k >= 0; --k) {
        double s = b[k];
        for (int cc = k + 1; cc < n; ++cc) s -= A[k * n + cc] * b[cc];
        b[k] = s / A[k * n + k];
    }
    return 0;
}

static void coefficients(const hl_ctx* C, const double* f, double* a) {
    for (int k = 0; k < C->nt; ++k) {
        double s = 0.0;
        for (int i = 0; i < C->q; ++i) s += f[i] * C->HT[i][k];
        a[k] = s;
    }
}

/* f_i = w_i sum_{n = n0..N} (1/n!) a^(n) : H^(n)(xi_i) */
static void reconstruct(const hl_ctx* C, const double* a, int n0, double* f) {
    for (int i = 0; i < C->q; ++i) {
        double s = 0.0;
        for (int n = n0; n <= C->nmax; ++n) {
            double t = 0.0;
            for (int k = 0; k < (1 << n); ++k) t += a[off(n) + k] * C->HT[i][off(n) + k];
            s += t / fact(n);
        }
        f[i] = C->W[i] * s;
    }
}

static void macro(const hl_ctx* C, const double* f, int thermal, double* rho, double u[2], double* theta) {
    double r = 0.0, j0 = 0.0, j1 = 0.0;
    for (int i = 0; i < C->q; ++i) {
        r += f[i];
        j0 += f[i] * C->XI[i][0];
        j1 += f[i] * C->XI[i][1];
    }
    u[0] = j0 / r;
    u[1] = j1 / r;
    *rho = r;
    if (thermal) {
        double e = 0.0;
        for (int i = 0; i < C->q; ++i) {
            double c0 = C->XI[i][0] - u[0], c1 = C->XI[i][1] - u[1];
            e += f[i] * (c0 * c0 + c1 * c1);
        }
        *theta = e / (2.0 * r);
    } else {
        *theta = 1.0;
    }
}

static void maxwellian_coefficients(const hl_ctx* C, double rho, const double u[2], double theta, double* a) {
    double H[HL_NTMAX];
    double st = sqrt(theta);
    for (int k = 0; k < C->nt; ++k) a[k] = 0.0;
    for (int p = 0; p < C->ngh; ++p)
        for (int q = 0; q < C->ngh; ++q) {
            double x[2] = {u[0] + st * C->GHX[p], u[1] + st * C->GHX[q]};
            hermite_full(x, C->nmax, H);
            double wt = rho * C->GHW[p] * C->GHW[q];
            for (int k = 0; k < C->nt; ++k) a[k] += wt * H[k];
        }
}

int hl_equilibrium_node(const void* vctx, double rho, const double* u, double theta, double* f) {
    const hl_ctx* C = (const hl_ctx*)vctx;
    double a[HL_NTMAX];
    maxwellian_coefficients(C, rho, u, theta, a);
    reconstruct(C, a, 0, f);
    return 0;
}

static double central(const hl_ctx* C, const double* g, const double u[2], int p, int q) {
    double s = 0.0;
    for (int i = 0; i < C->q; ++i) {
        double cx = C->XI[i][0] - u[0], cy = C->XI[i][1] - u[1];
        double m = 1.0;
        for (int k = 0; k < p; ++k) m *= cx;
        for (int k = 0; k < q; ++k) m *= cy;
        s += g[i] * m;
    }
    return s;
}

/* One node.  omega[n] for n = 0..N (0 and 1 unused). */
int hl_collide_node(const void* vctx, const double* omega, int thermal, const double* f, double* out) {
    const hl_ctx* C = (const hl_ctx*)vctx;
    const int Q = C->q, NA = C->na;
    double rho, u[2], theta;
    macro(C, f, thermal, &rho, u, &theta);
    double a0[HL_NTMAX], f0[HL_QMAX], f1[HL_QMAX], a1[HL_NTMAX], f1h[HL_QMAX], Om[HL_QMAX];
    maxwellian_coefficients(C, rho, u, theta, a0);
    reconstruct(C, a0, 0, f0);
    for (int i = 0; i < Q; ++i) f1[i] = f[i] - f0[i];
    coefficients(C, f1, a1);
    reconstruct(C, a1, 0, f1h);
    /* basis of Omega: one function per symmetric component (p x's, q y's) */
    double basis[HL_NAMAX][HL_QMAX];
    for (int k = 0; k < NA; ++k) {
        int p = C->ALPHA[k][0], q = C->ALPHA[k][1], n = p + q;
        int t = ((1 << n) - 1) & ~((1 << p) - 1); /* p x-indices then q y-indices */
        for (int i = 0; i < Q; ++i) basis[k][i] = C->W[i] * C->HT[i][off(n) + t] / (fact(p) * fact(q));
    }
    double A[HL_NAMAX * HL_NAMAX], rhs[HL_NAMAX];
    for (int r = 0; r < NA; ++r) {
        int p = C->ALPHA[r][0], q = C->ALPHA[r][1], n = p + q;
        for (int k = 0; k < NA; ++k) A[r * NA + k] = central(C, basis[k], u, p, q);
        rhs[r] = n <= 1 ? 0.0 : -omega[n] * central(C, f1h, u, p, q);
    }
    if (gauss_solve(NA, A, rhs)) return -1;
    for (int i = 0; i < Q; ++i) {
        double s = 0.0;
        for (int k = 0; k < NA; ++k) s += rhs[k] * basis[k][i];
        Om[i] = s;
    }
    for (int i = 0; i < Q; ++i) out[i] = f0[i] + f1h[i] + Om[i];
    return 0;
}

int hl_init(const void* vctx, int64_t N, const double* rho, const double* u, const double* theta, double* f) {
    const hl_ctx* C = (const hl_ctx*)vctx;
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < N; ++n) {
        double uu[2] = {u[n], u[N + n]}, fl[HL_QMAX];
        hl_equilibrium_node(C, rho[n], uu, theta ? theta[n] : 1.0, fl);
        for (int i = 0; i < C->q; ++i) f[(int64_t)i * N + n] = fl[i];
    }
    return 0;
}

int hl_moments(const void* vctx, int64_t N, const double* f, int thermal, double* rho, double* u, double* theta) {
    const hl_ctx* C = (const hl_ctx*)vctx;
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < N; ++n) {
        double fl[HL_QMAX], r, uu[2], th;
        for (int i = 0; i < C->q; ++i) fl[i] = f[(int64_t)i * N + n];
        macro(C, fl, thermal, &r, uu, &th);
        rho[n] = r;
        u[n] = uu[0];
        u[N + n] = uu[1];
        if (theta) theta[n] = th;
    }
    return 0;
}

int hl_step(const void* vctx, const int64_t* dims, const double* omega, int thermal, double* f, double* post,
            int64_t nsteps) {
    const hl_ctx* C = (const hl_ctx*)vctx;
    int64_t nx = dims[0], ny = dims[1], N = nx * ny;
    for (int64_t s = 0; s < nsteps; ++s) {
        int err = 0;
#pragma omp parallel for schedule(static) reduction(| : err)
        for (int64_t n = 0; n < N; ++n) {
            double fl[HL_QMAX], fo[HL_QMAX];
            for (int i = 0; i < C->q; ++i) fl[i] = f[(int64_t)i * N + n];
            err |= hl_collide_node(C, omega, thermal, fl, fo) ? 1 : 0;
            for (int i = 0; i < C->q; ++i) post[(int64_t)i * N + n] = fo[i];
        }
        if (err) return -1;
#pragma omp parallel for schedule(static)
        for (int64_t n = 0; n < N; ++n) {
            int64_t x = n % nx, y = n / nx;
            for (int i = 0; i < C->q; ++i) {
                int64_t xd = ((x + C->E[i][0]) % nx + nx) % nx;
                int64_t yd = ((y + C->E[i][1]) % ny + ny) % ny;
                f[(int64_t)i * N + xd + nx * yd] = post[(int64_t)i * N + n];
            }
        }
    }
    return 0;
}
