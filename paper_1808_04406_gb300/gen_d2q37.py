"""Generate ``csrc/d2q37_lattice.cuh``: the 37-velocity degree-9 lattice.

The lattice of Sec. II.A (Eq. quad) with abscissas xi_i = c e_i on the integer
lattice: the shells (0,0), (1,0), (1,1), (2,0), (2,1), (2,2), (3,0), (3,1),
one weight per shell, must integrate every monomial of degree <= 9 against the
unit-variance Gaussian.  Odd moments vanish by symmetry; the even conditions
x^0, x^2, x^4, x^2 y^2, x^6, x^4 y^2, x^8, x^6 y^2, x^4 y^4 remain.  For a trial
scale c all but x^8 are linear in the eight shell weights; c is then the zero of
the x^8 residual, bracketed on a grid and refined by bisection; the root with
all weights positive is kept.  The solve runs in 50-digit arithmetic (mpmath),
so the emitted FP64 constants are correctly rounded.

Velocity order of the header: opposite velocities sit at i and 36 - i and the
rest velocity at 18, so the AA pattern's opposite index is 36 - i.

Run ``python -m paper_1808_04406_gb300.gen_d2q37`` to rewrite the header; the
test suite checks that the committed header is what this script produces.
"""
import os

import mpmath
import numpy as np

mpmath.mp.dps = 50

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(HERE, "csrc", "d2q37_lattice.cuh")

SHELLS = [(0, 0), (1, 0), (1, 1), (2, 0), (2, 1), (2, 2), (3, 0), (3, 1)]
EVEN_CONDITIONS = [(0, 0), (2, 0), (4, 0), (2, 2), (6, 0), (4, 2), (8, 0), (6, 2), (4, 4)]


def _moment(n):
    """E[X^n] for X ~ N(0, 1)."""
    if n % 2:
        return mpmath.mpf(0)
    r = mpmath.mpf(1)
    for k in range(n - 1, 0, -2):
        r *= k
    return r


def _orbit(a, b):
    pts = {(sx * p, sy * q) for p, q in ((a, b), (b, a)) for sx in (1, -1) for sy in (1, -1)}
    return sorted(pts)


def _weights_and_residual(c):
    """Weights from the eight conditions other than x^8 (a well-conditioned 8 x 8
    system: the mixed conditions are not independent of each other on these
    shells, so one of the pure x^n conditions has to be the one left out) and
    the residual of x^8."""
    keep = [pq for pq in EVEN_CONDITIONS if pq != (8, 0)]
    row = lambda p, q: [mpmath.fsum((c * x) ** p * (c * y) ** q for x, y in _orbit(*s)) for s in SHELLS]
    A = mpmath.matrix([row(p, q) for p, q in keep])
    b = mpmath.matrix([_moment(p) * _moment(q) for p, q in keep])
    w = mpmath.lu_solve(A, b)
    r8 = row(8, 0)
    return w, mpmath.fsum(r8[j] * w[j] for j in range(len(SHELLS))) - _moment(8)


def solve():
    """Return (velocities e[37, 2], weights w[37], scale c) in the header's order."""
    grid = [mpmath.mpf(1) / 2 + mpmath.mpf(k) / 1000 for k in range(1101)]  # 0.5 .. 1.6
    res = [_weights_and_residual(c)[1] for c in grid]
    sol = []
    for lo, hi, rlo, rhi in zip(grid[:-1], grid[1:], res[:-1], res[1:]):
        if rlo == 0 or (rlo < 0) != (rhi < 0):
            for _ in range(200):
                mid = (lo + hi) / 2
                rm = _weights_and_residual(mid)[1]
                if (rm < 0) == (rlo < 0):
                    lo, rlo = mid, rm
                else:
                    hi = mid
            c = (lo + hi) / 2
            w, r = _weights_and_residual(c)
            if abs(r) < mpmath.mpf(10) ** -30 and all(w[j] > 0 for j in range(len(SHELLS))):
                sol.append((c, [float(w[j]) for j in range(len(SHELLS))]))
    if len(sol) != 1:
        raise RuntimeError("expected exactly one positive-weight rule, got %d" % len(sol))
    c, wsh = sol[0]
    c = float(c)
    half = []  # one velocity of every opposite pair, with its shell weight
    for s, ws in zip(SHELLS[1:], wsh[1:]):
        for v in _orbit(*s):
            if (-v[0], -v[1]) not in [h[0] for h in half]:
                half.append((v, ws))
    e = [h[0] for h in half] + [(0, 0)] + [(-h[0][0], -h[0][1]) for h in reversed(half)]
    w = [h[1] for h in half] + [wsh[0]] + [h[1] for h in reversed(half)]
    return np.array(e, dtype=np.int64), np.array(w), float(c)


def lattice_scale() -> float:
    """The scale c (xi = c e) as written into the generated header."""
    import re
    with open(HEADER) as fh:
        return float(re.search(r"constexpr double kC = ([0-9.eE+-]+);", fh.read()).group(1))


def header_text():
    e, w, c = solve()
    lines = [
        "// Generated by paper_1808_04406_gb300/gen_d2q37.py -- do not edit.",
        "// 37-velocity degree-9 lattice: xi_i = kC * e_i, weights w_of(i) (sum 1),",
        "// opposite velocities at i and 36 - i, rest velocity at 18.",
        "#pragma once",
        "",
        "namespace lbm {",
        "namespace h37 {",
        "",
        "constexpr int kQ = 37;",
        "constexpr double kC = %.17g;" % c,
        "",
        "// velocity components and weights, usable in host and device code",
        "__host__ __device__ constexpr int ex_of(int i) {",
        "  constexpr int t[kQ] = {%s};" % ", ".join(str(int(v)) for v in e[:, 0]),
        "  return t[i];",
        "}",
        "__host__ __device__ constexpr int ey_of(int i) {",
        "  constexpr int t[kQ] = {%s};" % ", ".join(str(int(v)) for v in e[:, 1]),
        "  return t[i];",
        "}",
        "__host__ __device__ constexpr double w_of(int i) {",
        "  constexpr double t[kQ] = {",
    ]
    for k in range(0, 37, 3):
        lines.append("      " + ", ".join("%.17g" % x for x in w[k:k + 3]) + ",")
    lines += ["  };", "  return t[i];", "}", "", "}  // namespace h37", "}  // namespace lbm", ""]
    return "\n".join(lines)


def write():
    with open(HEADER, "w") as fh:
        fh.write(header_text())
    return HEADER


if __name__ == "__main__":
    print(write())
