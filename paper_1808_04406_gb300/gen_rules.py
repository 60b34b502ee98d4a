"""Minimal square-symmetric quadrature rules on the integer lattice (Sec. III.A).

The paper compares four degree-7 rules with 17 velocities and four degree-9
rules with 37 (its E^7_{2,17} and E^9_{2,37}, Fig. 2) without printing them.
This module finds them: a rule is the rest velocity plus a set of velocity
shells (the orbits of (a, 0), (a, a) and (a, b) under the square's symmetries)
with one weight per shell and a scale c (xi = c e) such that every monomial of
degree <= d has its unit-Gaussian moment.  Odd moments vanish by symmetry; the
even ones x^p y^q (p >= q, p + q <= d - 1) give as many conditions as there are
unknowns (the weights and c) when degree 7 has four 4-velocity shells and
degree 9 five 4-velocity and two 8-velocity shells.  Inside |e_x|, |e_y| <= 3
there are exactly four positive rules of each kind; they are labelled A..D by
increasing c, then by shell list.

Method.  Row r of the moment matrix scales as c^{n_r} (n_r its degree), so the
determinant of [A(c) | b] equals prod_r c^{n_r} times a polynomial in
y = 1/c^2 whose coefficients are b_r times the cofactors of the shell matrix S
(the power sums of each shell, integers: the cofactors are exact).  Its
positive real roots, found at 50 digits, give c; the weights come from a square
subsystem (one condition left out and checked afterwards).
"""
import functools
import itertools

import mpmath
import numpy as np


def _gauss_moment(a):
    if a % 2:
        return 0
    r = 1
    for k in range(a - 1, 0, -2):
        r *= k
    return r


def _members(a, b):
    out = set()
    for p, q in ((a, b), (b, a)):
        for sx in (1, -1):
            for sy in (1, -1):
                out.add((sx * p, sy * q))
    return sorted(out)


def _conditions(degree):
    return [(p, t - p) for t in range(0, degree, 2) for p in range(t, -1, -1) if p % 2 == 0 and p >= t - p]


def _power_sums(shell, conds):
    return [sum(ex ** p * ey ** q for ex, ey in _members(*shell)) for p, q in conds]


def _int_det(M):
    """Exact determinant of an integer matrix (fraction-free Bareiss elimination)."""
    A = [list(row) for row in M]
    n = len(A)
    if n == 0:
        return 1
    sign, prev = 1, 1
    for k in range(n - 1):
        if A[k][k] == 0:
            sw = next((r for r in range(k + 1, n) if A[r][k] != 0), None)
            if sw is None:
                return 0
            A[k], A[sw] = A[sw], A[k]
            sign = -sign
        for i in range(k + 1, n):
            for j in range(k + 1, n):
                A[i][j] = (A[i][j] * A[k][k] - A[i][k] * A[k][j]) // prev
        prev = A[k][k]
    return sign * A[n - 1][n - 1]


def _solve_shells(shells, conds):
    """Positive-weight rules for one shell set: list of (c, weights per shell)."""
    m = len(conds)
    deg = [p + q for p, q in conds]
    rhs = [_gauss_moment(p) * _gauss_moment(q) for p, q in conds]
    S = [[_power_sums(sh, conds)[r] for sh in shells] for r in range(m)]  # conditions x shells, integers
    coef = [0] * (max(deg) // 2 + 1)  # exact integer coefficients of the polynomial in y = 1 / c^2
    for r in range(m):
        minor = [S[k] for k in range(m) if k != r]
        coef[deg[r] // 2] += (-1) ** (r + m - 1) * rhs[r] * _int_det(minor)
    while coef and coef[-1] == 0:
        coef.pop()
    if len(coef) < 2:
        return []
    out = []
    with mpmath.workdps(50):
        roots = mpmath.polyroots([mpmath.mpf(x) for x in coef[::-1]], maxsteps=200, extraprec=200)
        for y in roots:
            if abs(mpmath.im(y)) > mpmath.mpf(10) ** -30 or mpmath.re(y) <= 0:
                continue
            c = 1 / mpmath.sqrt(mpmath.re(y))
            A = [[mpmath.mpf(S[r][j]) * c ** deg[r] for j in range(len(shells))] for r in range(m)]
            w = None
            for drop in range(m - 1, -1, -1):  # a square subsystem, the dropped row checked after
                keep = [k for k in range(m) if k != drop]
                try:
                    ws = mpmath.lu_solve(mpmath.matrix([A[k] for k in keep]), mpmath.matrix([rhs[k] for k in keep]))
                except ZeroDivisionError:
                    continue
                if abs(mpmath.fsum(A[drop][j] * ws[j] for j in range(len(shells))) - rhs[drop]) < mpmath.mpf(10) ** -35:
                    w = ws
                    break
            if w is not None and all(w[j] > 0 for j in range(len(shells))):
                out.append((c, [w[j] for j in range(len(shells))]))
    return out


@functools.lru_cache(maxsize=None)
def rules(degree, max_speed=3):
    """The minimal rules of degree 7 or 9 as a tuple of (label, e[Q, 2] int32,
    w[Q] float64, c float64), velocities in shell order, rest velocity first."""
    if degree not in (7, 9):
        raise ValueError("degree 7 or 9")
    conds = _conditions(degree)
    four = [(a, 0) for a in range(1, max_speed + 1)] + [(a, a) for a in range(1, max_speed + 1)]
    eight = [(a, b) for a in range(2, max_speed + 1) for b in range(1, a)]
    n4, n8 = (4, 0) if degree == 7 else (5, 2)
    found = []
    for f4 in itertools.combinations(four, n4):
        for f8 in itertools.combinations(eight, n8):
            shells = [(0, 0)] + list(f4) + list(f8)
            for c, w in _solve_shells(shells, conds):
                found.append((float(c), sorted(shells), shells, w))
    found.sort(key=lambda t: (t[0], t[1]))
    out = []
    for k, (c, _, shells, w) in enumerate(found):
        e, ww = [], []
        for sh, wj in zip(shells, w):
            for v in _members(*sh):
                e.append(v)
                ww.append(float(wj))
        out.append(("ABCDEFGH"[k], np.array(e, dtype=np.int32), np.array(ww), c))
    return tuple(out)


def rule(name):
    """A rule by name: "E7-A" .. "E7-D", "E9-A" .. "E9-D" -> (e, w, c, order N)."""
    kind, label = name.split("-")
    degree = {"E7": 7, "E9": 9}[kind]
    for lab, e, w, c in rules(degree):
        if lab == label:
            return e, w, c, (3 if degree == 7 else 4)
    raise KeyError(name)


if __name__ == "__main__":
    for d in (7, 9):
        for lab, e, w, c in rules(d):
            print("E%d-%s  Q=%d  c=%.17g" % (d, lab, len(w), c))
