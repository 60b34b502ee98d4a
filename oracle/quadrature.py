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


def conditions(degree):
    """Even moment conditions x^p y^q (p >= q, p + q <= degree - 1) that make a
    square-symmetric rule exact to `degree` (odd moments vanish by symmetry)."""
    out = []
    for tot in range(0, degree, 2):
        for p in range(tot, -1, -2):
            if p >= tot - p:
                out.append((p, tot - p))
    return out


def _general_system(c, shells, conds):
    members = [shell_members(s) for s in shells]
    A = mpmath.matrix(len(conds), len(shells))
    b = mpmath.matrix(len(conds), 1)
    for r, (p, q) in enumerate(conds):
        for j, mem in enumerate(members):
            A[r, j] = mpmath.fsum((c * ex) ** p * (c * ey) ** q for ex, ey in mem)
        b[r] = mpmath.mpf(gaussian_moment(p)) * gaussian_moment(q)
    return A, b


def _general_det_float(c, shells, conds):
    M = np.zeros((len(conds), len(shells) + 1))
    for r, (p, q) in enumerate(conds):
        for j, s in enumerate(shells):
            M[r, j] = sum((c * ex) ** p * (c * ey) ** q for ex, ey in shell_members(s))
        M[r, -1] = gaussian_moment(p) * gaussian_moment(q)
    return np.linalg.det(M)


def _general_det(c, shells, conds):
    A, b = _general_system(c, shells, conds)
    M = mpmath.matrix(len(conds), len(shells) + 1)
    for r in range(len(conds)):
        for j in range(len(shells)):
            M[r, j] = A[r, j]
        M[r, len(shells)] = b[r]
    return mpmath.det(M)


def rules(degree, max_speed=3):
    """Every square-symmetric rule of the given degree with one weight per shell,
    velocities |e_x|, |e_y| <= max_speed, the fewest velocities (degree 7: the rest
    velocity and four 4-velocity shells, 17 velocities; degree 9: the rest velocity,
    five 4-velocity and two 8-velocity shells, 37) and all weights positive.
    For each shell set the scale c is a root of the augmented determinant (found
    by a float64 scan of c in [0.3, 3] and 50-digit bisection), the weights the
    least-squares solution of the conditions.  Returns a list of (e, w, c) sorted by
    c, then by the shell list."""
    conds = conditions(degree)
    four = [(a, 0) for a in range(1, max_speed + 1)] + [(a, a) for a in range(1, max_speed + 1)]
    eight = [(a, b) for a in range(2, max_speed + 1) for b in range(1, a)]
    n_shells = len(conds) - 1  # with the scale: as many unknowns as conditions
    import itertools
    found = []
    for n8 in range(0, len(eight) + 1):
        n4 = n_shells - 1 - n8
        if n4 < 0:
            continue
        if 1 + 4 * n4 + 8 * n8 != (17 if degree == 7 else 37 if degree == 9 else -1):
            continue
        for f4 in itertools.combinations(four, n4):
            for f8 in itertools.combinations(eight, n8):
                shells = [(0, 0)] + list(f4) + list(f8)
                cs = np.linspace(0.3, 3.0, 541)
                d = [_general_det_float(c, shells, conds) for c in cs]
                for k in range(len(cs) - 1):
                    if (d[k] < 0) == (d[k + 1] < 0):
                        continue
                    c = _bisect(lambda x: _general_det(x, shells, conds), mpmath.mpf(cs[k]), mpmath.mpf(cs[k + 1]))
                    A, b = _general_system(c, shells, conds)
                    # [A | b] is singular at the root, so solve the consistent system
                    # A w = b by its normal equations (50 digits) and check the residual
                    try:
                        wsh = mpmath.lu_solve(A.T * A, A.T * b)
                    except ZeroDivisionError:  # the shell columns are dependent at this c: no rule
                        continue
                    res = mpmath.norm(A * wsh - b) / mpmath.norm(b)
                    if all(wsh[j] > 0 for j in range(len(shells))) and res < mpmath.mpf(10) ** -30:
                        e, w = [], []
                        for j, sh in enumerate(shells):
                            for m in shell_members(sh):
                                e.append(m)
                                w.append(float(wsh[j]))
                        found.append((float(c), shells, np.array(e, dtype=np.int32), np.array(w)))
    found.sort(key=lambda t: (t[0], t[1]))
    return [(e, w, c) for c, _, e, w in found]


def exact_degree(e, w, c, max_degree=12):
    """Largest degree d such that every monomial x^p y^q with p + q <= d is
    integrated exactly (to 1e-12 relative) against the unit Gaussian."""
    xi = c * np.asarray(e, dtype=np.float64)
    for d in range(max_degree + 1):
        for p in range(d + 1):
            q = d - p
            got = np.sum(w * xi[:, 0] ** p * xi[:, 1] ** q)
            want = gaussian_moment(p) * gaussian_moment(q)
            if abs(got - want) > 1e-12 * max(1.0, abs(want)):
                return d - 1
    return max_degree


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
