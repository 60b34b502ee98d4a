"""The 37-velocity, degree-9 two-dimensional quadrature (E^9_{2,37}) for the oracle.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. II.A, Eq. quad: abscissas xi_i = c e_i on the integer lattice and weights
w_i integrate every polynomial of degree <= 9 exactly against the unit-variance
Gaussian weight function.  The paper takes its rules from another publication
(not available here), so the oracle derives one: the eight velocity shells
(0,0), (1,0), (1,1), (2,0), (2,1), (2,2), (3,0), (3,1) (1+4+4+4+8+4+4+8 = 37
velocities) with one weight per shell.  By the shells' symmetry every odd
moment vanishes; the nine even moment conditions of degree 0..8
(x^0, x^2, x^4, x^2y^2, x^6, x^4y^2, x^8, x^6y^2, x^4y^4) fix the eight weights
and the scale c.  For a trial c the conditions are linear in the weights; c is
the root of the determinant of the augmented 9 x 9 system, found by bracketing,
and the weights are the least-squares solution of the nine conditions.  All of
it runs in 50-digit arithmetic (mpmath), so the FP64 results are correctly
rounded.
"""
import mpmath
import numpy as np

mpmath.mp.dps = 50

SHELLS = [(0, 0), (1, 0), (1, 1), (2, 0), (2, 1), (2, 2), (3, 0), (3, 1)]
CONDITIONS = [(0, 0), (2, 0), (4, 0), (2, 2), (6, 0), (4, 2), (8, 0), (6, 2), (4, 4)]


def shell_members(shell):
    a, b = shell
    out = set()
    for p, q in ((a, b), (b, a)):
        for sx in (1, -1):
            for sy in (1, -1):
                out.add((sx * p, sy * q))
    return sorted(out)


def gaussian_moment(a):
    """E[X^a] for a unit-variance Gaussian: (a-1)!! for even a, 0 for odd a."""
    if a % 2:
        return 0.0
    r = 1.0
    for k in range(a - 1, 0, -2):
        r *= k
    return r


def _system(c):
    members = [shell_members(s) for s in SHELLS]
    A = mpmath.matrix(len(CONDITIONS), len(SHELLS))
    b = mpmath.matrix(len(CONDITIONS), 1)
    for r, (p, q) in enumerate(CONDITIONS):
        for j, mem in enumerate(members):
            A[r, j] = mpmath.fsum((c * ex) ** p * (c * ey) ** q for ex, ey in mem)
        b[r] = mpmath.mpf(gaussian_moment(p)) * gaussian_moment(q)
    return A, b


def _det(c):
    A, b = _system(c)
    M = mpmath.matrix(len(CONDITIONS), len(SHELLS) + 1)
    for r in range(len(CONDITIONS)):
        for j in range(len(SHELLS)):
            M[r, j] = A[r, j]
        M[r, len(SHELLS)] = b[r]
    return mpmath.det(M)


def _bisect(f, lo, hi, iters=200):
    flo = f(lo)
    for _ in range(iters):
        mid = (lo + hi) / 2
        fm = f(mid)
        if (fm < 0) == (flo < 0):
            lo, flo = mid, fm
        else:
            hi = mid
    return (lo + hi) / 2


def solve_d2q37():
    """Return (e[37, 2] int, w[37], c) with the rest velocity first and shells in
    the order above, each shell's members sorted."""
    cs = [mpmath.mpf(3) / 10 + mpmath.mpf(k) / 500 for k in range(601)]  # 0.3 .. 1.5
    vals = [_det(c) for c in cs]
    roots = []
    for i in range(len(cs) - 1):
        if (vals[i] < 0) != (vals[i + 1] < 0):
            c = _bisect(_det, cs[i], cs[i + 1])
            A, b = _system(c)
            wsh, _ = mpmath.qr_solve(A, b)
            if all(wsh[j] > 0 for j in range(len(SHELLS))):
                roots.append((c, wsh))
    if len(roots) != 1:
        raise RuntimeError("expected one positive-weight solution, found %d" % len(roots))
    c, wsh = roots[0]
    e, w = [], []
    for j, s in enumerate(SHELLS):
        for m in shell_members(s):
            e.append(m)
            w.append(float(wsh[j]))
    return np.array(e, dtype=np.int32), np.array(w), float(c)
