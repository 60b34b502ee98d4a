/*
 * FP64 CPU oracle for the thermal / isothermal CM-MRT step on the 37-velocity
 * degree-9 lattice E^9_{2,37} (Hermite projection order N = 4, equilibrium
 * truncation M = 4), written from X. Shan, arXiv:1808.04406.
 *
 * TEST INFRASTRUCTURE ONLY: the checker of the CUDA path; shares nothing with
 * it.  The lattice (velocities, weights, scale c with xi_i = c e_i) and the
 * Gauss-Hermite points used to integrate the Maxwellian are handed in by
 * h37_setup from the Python side of the oracle.
 *
 * Definitions used:
 *   - tensor Hermite polynomials by the recursion of the Appendix,
 *     H^(n+1)_{t j} = xi_j H^(n)_t - sum_k delta(t_k, j) H^(n-1)_{t \ k},
 *     stored as full (unsymmetrised) 2^n-component tensors;
 *   - Hermite coefficients a^(n) = sum_i f_i H^(n)(xi_i) (Eq. an) and the
 *     reconstruction f_i = w_i sum_n (1/n!) a^(n) : H^(n)(xi_i) (Eq. fi);
 *   - rho, u, and theta from rho (u^2 + 2 eps) = sum f xi^2, eps = D theta / 2
 *     (Sec. II.A moments); isothermal runs freeze theta = 1;
 *   - f^(0): the Maxwellian (Eq. maxwellian) projected onto n <= 4, its
 *     coefficients a_0^(n) = int f^(0) H^(n) obtained by Gauss-Hermite
 *     quadrature of the Maxwellian itself (exact: polynomial integrands);
 *   - f^(1) = f - f^(0); f^ (1) = sum_{n<=4} M^(n) f^(1) (Eqs. m, reg);
 *   - the collision of Sec. II.C: Omega has no components above order 4, its
 *     central moments of order n equal -omega_n times those of f^(1) for all
 *     |alpha| <= 4 (Eq. omega), zero for orders 0 and 1;
 *     H37_DEFINITIONAL solves that 15 x 15 linear system node by node;
 *     H37_CLOSED evaluates the closed form of Eq. mrt with the 4th-order
 *     coupling constant K (K = 6 follows from Eq. omega with the n! norm;
 *     the printed equations carry 72);
 *     H37_RBGK is the regularised BGK of Eq. lbgk-reg (omega_2 for all);
 *     H37_RAWMRT relaxes each absolute-frame coefficient at its own rate
 *     (the earlier high-order MRT, Sec. II.B);
 *   - update f_i(x + e_i, t + 1) = f^_i + Omega_i with f^ = f^(0) + f^ (1).
 * Layout f[i * N + node], node = x + nx * y.  Compiled with -ffp-contract=off.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#define H37_Q 37
#define H37_NT 31 /* full tensor components of orders 0..4: 1+2+4+8+16 */
#define H37_NA 15 /* central monomials x^p y^q with p + q <= 4 */

#define H37_DEFINITIONAL 0
#define H37_CLOSED 1
#define H37_RBGK 2
#define H37_RAWMRT 3

static int E[H37_Q][2];
static double W[H37_Q];
static double XI[H37_Q][2];
static double HT[H37_Q][H37_NT];
static int NGH;
static double GHX[16], GHW[16];
static int ALPHA[H37_NA][2];

static int off(int n) { return (1 << n) - 1; }

static double fact(int n) {
    double r = 1.0;
    for (int k = 2; k <= n; ++k) r *= k;
    return r;
}

static void hermite_full(const double xi[2], double* H) {
    H[0] = 1.0;
    for (int n = 0; n < 4; ++n) {
        for (int t = 0; t < (1 << n); ++t) {
            for (int j = 0; j < 2; ++j) {
                double v = xi[j] * H[off(n) + t];
                for (int k = 0; k < n; ++k) {
                    if (((t >> k) & 1) == j) {
                        int tr = (t & ((1 << k) - 1)) | ((t >> (k + 1)) << k);
                        v -= H[off(n - 1) + tr];
                    }
                }
                H[off(n + 1) + (t | (j << n))] = v;
            }
        }
    }
}

int h37_setup(const int* e, const double* w, double c, int ngh, const double* ghx, const double* ghw) {
    if (ngh > 16) return -1;
    for (int i = 0; i < H37_Q; ++i) {
        E[i][0] = e[2 * i];
        E[i][1] = e[2 * i + 1];
        W[i] = w[i];
        XI[i][0] = c * E[i][0];
        XI[i][1] = c * E[i][1];
        hermite_full(XI[i], HT[i]);
    }
    NGH = ngh;
    for (int k = 0; k < ngh; ++k) {
        GHX[k] = ghx[k];
        GHW[k] = ghw[k];
    }
    int a = 0;
    for (int n = 0; n <= 4; ++n)
        for (int p = n; p >= 0; --p) {
            ALPHA[a][0] = p;
            ALPHA[a][1] = n - p;
            ++a;
        }
    return 0;
}

/* Hermite polynomial components at one point (for tests). */
int h37_hermite(const double* xi, double* H) {
    hermite_full(xi, H);
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

/* a^(n) = sum_i f_i H^(n)(xi_i), full tensors n = 0..4 */
static void coefficients(const double* f, double* a) {
    for (int c = 0; c < H37_NT; ++c) {
        double s = 0.0;
        for (int i = 0; i < H37_Q; ++i) s += f[i] * HT[i][c];
        a[c] = s;
    }
}

/* f_i = w_i sum_{n = n0..4} (1/n!) a^(n) : H^(n)(xi_i) */
static void reconstruct(const double* a, int n0, double* f) {
    for (int i = 0; i < H37_Q; ++i) {
        double s = 0.0;
        for (int n = n0; n <= 4; ++n) {
            double t = 0.0;
            for (int k = 0; k < (1 << n); ++k) t += a[off(n) + k] * HT[i][off(n) + k];
            s += t / fact(n);
        }
        f[i] = W[i] * s;
    }
}

static void macro(const double* f, int thermal, double* rho, double u[2], double* theta) {
    double r = 0.0, j0 = 0.0, j1 = 0.0;
    for (int i = 0; i < H37_Q; ++i) {
        r += f[i];
        j0 += f[i] * XI[i][0];
        j1 += f[i] * XI[i][1];
    }
    u[0] = j0 / r;
    u[1] = j1 / r;
    *rho = r;
    if (thermal) {
        double e = 0.0;
        for (int i = 0; i < H37_Q; ++i) {
            double c0 = XI[i][0] - u[0], c1 = XI[i][1] - u[1];
            e += f[i] * (c0 * c0 + c1 * c1);
        }
        *theta = e / (2.0 * r);
    } else {
        *theta = 1.0;
    }
}

/* Maxwellian coefficients: a_0^(n) = rho * E[H^(n)(X)], X ~ N(u, theta I),
 * by the tensor Gauss-Hermite rule in z = (X - u)/sqrt(theta). */
static void maxwellian_coefficients(double rho, const double u[2], double theta, double* a) {
    double H[H37_NT];
    double st = sqrt(theta);
    for (int c = 0; c < H37_NT; ++c) a[c] = 0.0;
    for (int p = 0; p < NGH; ++p)
        for (int q = 0; q < NGH; ++q) {
            double x[2] = {u[0] + st * GHX[p], u[1] + st * GHX[q]};
            hermite_full(x, H);
            double wt = rho * GHW[p] * GHW[q];
            for (int c = 0; c < H37_NT; ++c) a[c] += wt * H[c];
        }
}

int h37_maxwellian_coefficients(double rho, const double* u, double theta, double* a) {
    maxwellian_coefficients(rho, u, theta, a);
    return 0;
}

int h37_equilibrium_node(double rho, const double* u, double theta, double* f) {
    double a[H37_NT];
    maxwellian_coefficients(rho, u, theta, a);
    reconstruct(a, 0, f);
    return 0;
}

/* central monomial (xi - u)^alpha summed against g */
static double central(const double* g, const double u[2], int p, int q) {
    double s = 0.0;
    for (int i = 0; i < H37_Q; ++i) {
        double cx = XI[i][0] - u[0], cy = XI[i][1] - u[1];
        double m = 1.0;
        for (int k = 0; k < p; ++k) m *= cx;
        for (int k = 0; k < q; ++k) m *= cy;
        s += g[i] * m;
    }
    return s;
}

/* ---- full-tensor algebra for the closed form ---- */
/* symmetrise a rank-n tensor in place (average over the n! index permutations) */
static void symmetrise(double* T, int n) {
    int perm[4] = {0, 1, 2, 3};
    double out[16];
    int np = (int)fact(n);
    for (int t = 0; t < (1 << n); ++t) out[t] = 0.0;
    /* iterate permutations with Heap's algorithm */
    int c[4] = {0, 0, 0, 0};
    for (int cnt = 0; cnt < np;) {
        for (int t = 0; t < (1 << n); ++t) {
            int tp = 0;
            for (int k = 0; k < n; ++k) tp |= ((t >> perm[k]) & 1) << k;
            out[t] += T[tp];
        }
        ++cnt;
        if (cnt == np) break;
        int i = 1;
        while (c[i] >= i) {
            c[i] = 0;
            ++i;
        }
        if (i % 2 == 0) {
            int x = perm[0]; perm[0] = perm[i]; perm[i] = x;
        } else {
            int x = perm[c[i]]; perm[c[i]] = perm[i]; perm[i] = x;
        }
        ++c[i];
    }
    for (int t = 0; t < (1 << n); ++t) T[t] = out[t] / np;
}

/* (A (x) B) with A of rank na, B of rank nb: index bits of A first */
static void outer(const double* A, int na, const double* B, int nb, double* out) {
    for (int s = 0; s < (1 << na); ++s)
        for (int t = 0; t < (1 << nb); ++t) out[s | (t << na)] = A[s] * B[t];
}

/* Omega's coefficients by Eq. mrt with 4th-order coupling constant K */
static void closed_form(const double* a1, const double u[2], const double* om, double K, double* aO) {
    double uu[4], t3[8], t4a[16], t4b[16], t4c[16], d2[4] = {1.0, 0.0, 0.0, 1.0};
    const double* a2 = a1 + off(2);
    const double* a3 = a1 + off(3);
    const double* a4 = a1 + off(4);
    double w2 = om[2], w3 = om[3], w4 = om[4];
    for (int c = 0; c < H37_NT; ++c) aO[c] = 0.0;
    for (int t = 0; t < 4; ++t) aO[off(2) + t] = -w2 * a2[t];
    outer(u, 1, a2, 2, t3);
    symmetrise(t3, 3);
    for (int t = 0; t < 8; ++t) aO[off(3) + t] = -w3 * a3[t] + 3.0 * (w3 - w2) * t3[t];
    outer(u, 1, a3, 3, t4a);
    symmetrise(t4a, 4);
    outer(u, 1, u, 1, uu);
    outer(uu, 2, a2, 2, t4b);
    symmetrise(t4b, 4);
    outer(d2, 2, a2, 2, t4c);
    symmetrise(t4c, 4);
    for (int t = 0; t < 16; ++t)
        aO[off(4) + t] = -w4 * a4[t] + 4.0 * (w4 - w3) * t4a[t] - 6.0 * (w4 + w2 - 2.0 * w3) * t4b[t] -
                         K * (w4 - w2) * t4c[t];
}

/* One node.  omega[n] for n = 0..4 (0 and 1 unused). */
int h37_collide_node(const double* omega, int thermal, int variant, double K, const double* f,
                     double* out) {
    double rho, u[2], theta;
    macro(f, thermal, &rho, u, &theta);
    double a0[H37_NT], f0[H37_Q], f1[H37_Q], a1[H37_NT], f1h[H37_Q], Om[H37_Q];
    maxwellian_coefficients(rho, u, theta, a0);
    reconstruct(a0, 0, f0);
    for (int i = 0; i < H37_Q; ++i) f1[i] = f[i] - f0[i];
    coefficients(f1, a1);
    reconstruct(a1, 0, f1h);
    if (variant == H37_RBGK) {
        for (int i = 0; i < H37_Q; ++i) out[i] = f0[i] + (1.0 - omega[2]) * f1h[i];
        return 0;
    }
    if (variant == H37_RAWMRT) {
        double aO[H37_NT];
        for (int c = 0; c < H37_NT; ++c) aO[c] = 0.0;
        for (int n = 2; n <= 4; ++n)
            for (int t = 0; t < (1 << n); ++t) aO[off(n) + t] = -omega[n] * a1[off(n) + t];
        reconstruct(aO, 2, Om);
    } else if (variant == H37_CLOSED) {
        double aO[H37_NT];
        closed_form(a1, u, omega, K, aO);
        reconstruct(aO, 2, Om);
    } else {
        /* basis of Omega: one function per symmetric component (n; p x's, q y's) */
        double basis[H37_NA][H37_Q];
        for (int c = 0; c < H37_NA; ++c) {
            int p = ALPHA[c][0], q = ALPHA[c][1], n = p + q;
            int t = ((1 << n) - 1) & ~((1 << p) - 1); /* p x-indices then q y-indices */
            for (int i = 0; i < H37_Q; ++i) basis[c][i] = W[i] * HT[i][off(n) + t] / (fact(p) * fact(q));
        }
        double A[H37_NA * H37_NA], rhs[H37_NA];
        for (int r = 0; r < H37_NA; ++r) {
            int p = ALPHA[r][0], q = ALPHA[r][1], n = p + q;
            for (int c = 0; c < H37_NA; ++c) A[r * H37_NA + c] = central(basis[c], u, p, q);
            rhs[r] = n <= 1 ? 0.0 : -omega[n] * central(f1h, u, p, q);
        }
        if (gauss_solve(H37_NA, A, rhs)) return -1;
        for (int i = 0; i < H37_Q; ++i) {
            double s = 0.0;
            for (int c = 0; c < H37_NA; ++c) s += rhs[c] * basis[c][i];
            Om[i] = s;
        }
    }
    for (int i = 0; i < H37_Q; ++i) out[i] = f0[i] + f1h[i] + Om[i];
    return 0;
}

int h37_init(int64_t N, const double* rho, const double* u, const double* theta, double* f) {
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < N; ++n) {
        double uu[2] = {u[n], u[N + n]}, fl[H37_Q];
        h37_equilibrium_node(rho[n], uu, theta ? theta[n] : 1.0, fl);
        for (int i = 0; i < H37_Q; ++i) f[(int64_t)i * N + n] = fl[i];
    }
    return 0;
}

int h37_moments(int64_t N, const double* f, int thermal, double* rho, double* u, double* theta) {
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < N; ++n) {
        double fl[H37_Q], r, uu[2], th;
        for (int i = 0; i < H37_Q; ++i) fl[i] = f[(int64_t)i * N + n];
        macro(fl, thermal, &r, uu, &th);
        rho[n] = r;
        u[n] = uu[0];
        u[N + n] = uu[1];
        if (theta) theta[n] = th;
    }
    return 0;
}

int h37_step(const int64_t* dims, const double* omega, int thermal, int variant, double K, double* f,
             double* post, int64_t nsteps) {
    int64_t nx = dims[0], ny = dims[1], N = nx * ny;
    for (int64_t s = 0; s < nsteps; ++s) {
        int err = 0;
#pragma omp parallel for schedule(static) reduction(| : err)
        for (int64_t n = 0; n < N; ++n) {
            double fl[H37_Q], fo[H37_Q];
            for (int i = 0; i < H37_Q; ++i) fl[i] = f[(int64_t)i * N + n];
            err |= h37_collide_node(omega, thermal, variant, K, fl, fo) ? 1 : 0;
            for (int i = 0; i < H37_Q; ++i) post[(int64_t)i * N + n] = fo[i];
        }
        if (err) return -1;
#pragma omp parallel for schedule(static)
        for (int64_t n = 0; n < N; ++n) {
            int64_t x = n % nx, y = n / nx;
            for (int i = 0; i < H37_Q; ++i) {
                int64_t xd = ((x + E[i][0]) % nx + nx) % nx;
                int64_t yd = ((y + E[i][1]) % ny + ny) % ny;
                f[(int64_t)i * N + xd + nx * yd] = post[(int64_t)i * N + n];
            }
        }
    }
    return 0;
}
