"""Python side of the general Hermite-lattice CM-MRT oracle (TEST INFRASTRUCTURE ONLY).

The minimal square-symmetric rules of degree 7 (17 velocities) and 9 (37
velocities) with velocities inside |e_x|, |e_y| <= 3 come from
``oracle.quadrature.rules``; there are four of each.  They are labelled A..D in
the order ``rules`` returns them (by scale c, then shell list): the paper names
four rules of each kind (Sec. III.A, Fig. 2) but does not print them.  Degree-7
rules carry the Hermite expansion and the equilibrium to N = M = 3, degree-9
rules to N = M = 4.

Layout f[i, node] in the rule's own velocity order, node = x + nx * y; fields
rho[node], u[2, node] in Hermite units (xi = c e), theta[node].  Relaxation rates
omega[n] for orders n = 0..N (0 and 1 unused).
"""
import ctypes
import functools

import numpy as np
from numpy.polynomial.hermite_e import hermegauss

from . import quadrature

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_i64p = ctypes.POINTER(ctypes.c_int64)


def declare(L):
    L.hl_ctx_bytes.argtypes = []
    L.hl_ctx_bytes.restype = ctypes.c_size_t
    L.hl_setup.argtypes = [ctypes.c_void_p, ctypes.c_int, _ip, _dp, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                           _dp, _dp]
    L.hl_equilibrium_node.argtypes = [ctypes.c_void_p, ctypes.c_double, _dp, ctypes.c_double, _dp]
    L.hl_collide_node.argtypes = [ctypes.c_void_p, _dp, ctypes.c_int, _dp, _dp]
    L.hl_init.argtypes = [ctypes.c_void_p, ctypes.c_int64, _dp, _dp, _dp, _dp]
    L.hl_moments.argtypes = [ctypes.c_void_p, ctypes.c_int64, _dp, ctypes.c_int, _dp, _dp, _dp]
    L.hl_step.argtypes = [ctypes.c_void_p, _i64p, _dp, ctypes.c_int, _dp, _dp, ctypes.c_int64]
    for n in ("hl_setup", "hl_equilibrium_node", "hl_collide_node", "hl_init", "hl_moments", "hl_step"):
        getattr(L, n).restype = ctypes.c_int


def _p(a):
    return None if a is None else a.ctypes.data_as(_dp)


@functools.lru_cache(maxsize=None)
def rule_set(degree):
    """The four minimal rules of the degree, as a tuple of (label, e, w, c)."""
    return tuple(("ABCD"[k], e, w, c) for k, (e, w, c) in enumerate(quadrature.rules(degree)))


class Lattice:
    """One rule with its truncation order N (3 for degree 7, 4 for degree 9)."""

    def __init__(self, e, w, c, nmax):
        from . import lib
        self.L = lib()
        self.e = np.ascontiguousarray(e, dtype=np.int32).reshape(-1, 2)
        self.w = np.ascontiguousarray(w, dtype=np.float64)
        self.c = float(c)
        self.q = len(self.w)
        self.nmax = int(nmax)
        self.ctx = ctypes.create_string_buffer(int(self.L.hl_ctx_bytes()))
        x, gw = hermegauss(6)
        gw = gw / gw.sum()
        rc = self.L.hl_setup(self.ctx, self.q, self.e.reshape(-1).ctypes.data_as(_ip), _p(self.w), self.c, self.nmax,
                             len(x), _p(np.ascontiguousarray(x)), _p(np.ascontiguousarray(gw)))
        if rc:
            raise ValueError("bad lattice")

    @classmethod
    def named(cls, degree, label):
        for lab, e, w, c in rule_set(degree):
            if lab == label:
                return cls(e, w, c, 3 if degree == 7 else 4)
        raise KeyError(label)

    def omega_from_tau(self, tau_per_order):
        om = np.zeros(self.nmax + 1)
        t = list(tau_per_order)
        for n in range(2, self.nmax + 1):
            om[n] = 1.0 / (t[n - 2] if n - 2 < len(t) else 1.0)
        return om

    def equilibrium_node(self, rho, u, theta=1.0):
        f = np.zeros(self.q)
        self.L.hl_equilibrium_node(self.ctx, float(rho), _p(np.ascontiguousarray(u, dtype=np.float64)), float(theta),
                                   _p(f))
        return f

    def collide_node(self, omega, f, thermal=True):
        out = np.zeros(self.q)
        rc = self.L.hl_collide_node(self.ctx, _p(np.ascontiguousarray(omega, dtype=np.float64)), int(thermal),
                                    _p(np.ascontiguousarray(f, dtype=np.float64)), _p(out))
        if rc:
            raise ArithmeticError("singular relaxation system")
        return out

    def init(self, rho, u, theta=None):
        rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(-1)
        N = rho.size
        u = np.ascontiguousarray(u, dtype=np.float64).reshape(2, N)
        th = None if theta is None else np.ascontiguousarray(theta, dtype=np.float64).reshape(-1)
        f = np.zeros((self.q, N))
        self.L.hl_init(self.ctx, N, _p(rho), _p(u), _p(th), _p(f))
        return f

    def moments(self, f, thermal=True):
        f = np.ascontiguousarray(f, dtype=np.float64)
        N = f.shape[1]
        rho, u, th = np.zeros(N), np.zeros((2, N)), np.zeros(N)
        self.L.hl_moments(self.ctx, N, _p(f), int(thermal), _p(rho), _p(u), _p(th))
        return rho, u, th

    def step(self, dims, omega, f, nsteps=1, thermal=True):
        """Advance f (Q, N) in place by nsteps collide-then-stream steps."""
        assert f.dtype == np.float64 and f.flags.c_contiguous
        d = np.array(list(dims), dtype=np.int64)
        post = np.empty_like(f)
        rc = self.L.hl_step(self.ctx, d.ctypes.data_as(_i64p), _p(np.ascontiguousarray(omega, dtype=np.float64)),
                            int(thermal), _p(f), _p(post), int(nsteps))
        if rc:
            raise ArithmeticError("singular relaxation system")
        return f
