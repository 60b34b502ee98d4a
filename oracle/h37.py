"""Python side of the 37-velocity thermal CM-MRT oracle (TEST INFRASTRUCTURE ONLY).

Velocities, weights and scale come from ``oracle.quadrature.solve_d2q37`` and
the Maxwellian is integrated with numpy's Gauss-Hermite rule; both are handed
to the C oracle once.  Layout: f[i, node] in the oracle's velocity order
(``lattice()``), node = x + nx*y; fields rho[node], u[2, node], theta[node].
Relaxation rates omega[n] for orders n = 0..4 (0 and 1 unused).
"""
import ctypes

import numpy as np
from numpy.polynomial.hermite_e import hermegauss

from . import quadrature

H37_DEFINITIONAL, H37_CLOSED, H37_RBGK, H37_RAWMRT = 0, 1, 2, 3
Q = 37

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_i64p = ctypes.POINTER(ctypes.c_int64)
_state = {}


def declare(L):
    L.h37_setup.argtypes = [_ip, _dp, ctypes.c_double, ctypes.c_int, _dp, _dp]
    L.h37_hermite.argtypes = [_dp, _dp]
    L.h37_maxwellian_coefficients.argtypes = [ctypes.c_double, _dp, ctypes.c_double, _dp]
    L.h37_equilibrium_node.argtypes = [ctypes.c_double, _dp, ctypes.c_double, _dp]
    L.h37_collide_node.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, _dp, _dp]
    L.h37_init.argtypes = [ctypes.c_int64, _dp, _dp, _dp, _dp]
    L.h37_moments.argtypes = [ctypes.c_int64, _dp, ctypes.c_int, _dp, _dp, _dp]
    L.h37_step.argtypes = [_i64p, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, _dp, _dp, ctypes.c_int64]
    for n in ("h37_setup", "h37_hermite", "h37_maxwellian_coefficients", "h37_equilibrium_node",
              "h37_collide_node", "h37_init", "h37_moments", "h37_step"):
        getattr(L, n).restype = ctypes.c_int


def _p(a):
    return None if a is None else a.ctypes.data_as(_dp)


def _lib():
    from . import lib
    L = lib()
    if "ready" not in _state:
        e, w, c = quadrature.solve_d2q37()
        x, gw = hermegauss(6)
        gw = gw / gw.sum()
        ee = np.ascontiguousarray(e.reshape(-1), dtype=np.int32)
        L.h37_setup(ee.ctypes.data_as(_ip), _p(np.ascontiguousarray(w)), c, len(x), _p(np.ascontiguousarray(x)),
                    _p(np.ascontiguousarray(gw)))
        _state.update(ready=True, e=e, w=w, c=c)
    return L


def lattice():
    """(e[37, 2], w[37], c): xi_i = c e_i."""
    _lib()
    return _state["e"], _state["w"], _state["c"]


def omega_from_tau(tau_per_order):
    om = np.zeros(5)
    t = list(tau_per_order)
    for n in range(2, 5):
        om[n] = 1.0 / (t[n - 2] if n - 2 < len(t) else 1.0)
    return om


def hermite(xi):
    H = np.zeros(31)
    _lib().h37_hermite(_p(np.ascontiguousarray(xi, dtype=np.float64)), _p(H))
    return H


def maxwellian_coefficients(rho, u, theta):
    a = np.zeros(31)
    _lib().h37_maxwellian_coefficients(float(rho), _p(np.ascontiguousarray(u, dtype=np.float64)), float(theta),
                                       _p(a))
    return a


def equilibrium_node(rho, u, theta=1.0):
    f = np.zeros(Q)
    _lib().h37_equilibrium_node(float(rho), _p(np.ascontiguousarray(u, dtype=np.float64)), float(theta), _p(f))
    return f


def collide_node(omega, f, thermal=True, variant=H37_DEFINITIONAL, K=6.0):
    out = np.zeros(Q)
    rc = _lib().h37_collide_node(_p(np.ascontiguousarray(omega, dtype=np.float64)), int(thermal), variant, float(K),
                                 _p(np.ascontiguousarray(f, dtype=np.float64)), _p(out))
    if rc:
        raise ArithmeticError("singular relaxation system")
    return out


def init(rho, u, theta=None):
    rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(-1)
    N = rho.size
    u = np.ascontiguousarray(u, dtype=np.float64).reshape(2, N)
    th = None if theta is None else np.ascontiguousarray(theta, dtype=np.float64).reshape(-1)
    f = np.zeros((Q, N))
    _lib().h37_init(N, _p(rho), _p(u), _p(th), _p(f))
    return f


def moments(f, thermal=True):
    f = np.ascontiguousarray(f, dtype=np.float64)
    N = f.shape[1]
    rho, u, th = np.zeros(N), np.zeros((2, N)), np.zeros(N)
    _lib().h37_moments(N, _p(f), int(thermal), _p(rho), _p(u), _p(th))
    return rho, u, th


def step(dims, omega, f, nsteps=1, thermal=True, variant=H37_CLOSED, K=6.0):
    """Advance f (Q, N) in place by nsteps collide-then-stream steps."""
    assert f.dtype == np.float64 and f.flags.c_contiguous
    d = np.array(list(dims), dtype=np.int64)
    post = np.empty_like(f)
    rc = _lib().h37_step(d.ctypes.data_as(_i64p), _p(np.ascontiguousarray(omega, dtype=np.float64)), int(thermal),
                         variant, float(K), _p(f), _p(post), int(nsteps))
    if rc:
        raise ArithmeticError("singular relaxation system")
    return f
