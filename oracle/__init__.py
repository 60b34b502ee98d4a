"""FP64 CPU oracle of the CM-MRT lattice Boltzmann step (arXiv:1808.04406).

TEST INFRASTRUCTURE ONLY.  This package is the independent checker of the CUDA
library: only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline / reference leg may import it.  It shares no code with the CUDA
path and never imports the product package; the product never imports it.

Arrays follow the oracle's own layout: populations ``f[i, node]`` with
``node = x + nx*(y + ny*z)`` and velocity index ``i = sum_d (e_id + 1) 3^d``
(tensor-product lattices); fields ``rho[node]`` and ``u[d, node]``.

Relaxation rates: ``omega[n]`` is the rate of central-moment order ``n``
(Sec. II.C, Eq. omega); orders 0 and 1 are conserved and carry no rate.
"""
import ctypes

import numpy as np

from . import build as _build

ORC_DEFINITIONAL = 0
ORC_KRONECKER = 1
ORC_LBGK = 2

_lib = None


def lib():
    """Load (building first if needed) the compiled oracle."""
    global _lib
    if _lib is None:
        path = _build.build()
        _lib = ctypes.CDLL(path)
        _declare(_lib)
    return _lib


_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_i64p = ctypes.POINTER(ctypes.c_int64)


def _declare(L):
    L.orc_tp_weight.argtypes = [ctypes.c_int, _dp]
    L.orc_tp_velocities.argtypes = [ctypes.c_int, _ip]
    L.orc_tp_collide_node.argtypes = [ctypes.c_int, _dp, ctypes.c_int, _dp, _dp]
    L.orc_tp_collide_node_rates.argtypes = [ctypes.c_int, _dp, _dp, _dp]
    L.orc_tp_equilibrium_node.argtypes = [ctypes.c_int, ctypes.c_double, _dp, _dp]
    L.orc_tp_product_equilibrium_node.argtypes = [ctypes.c_int, ctypes.c_double, _dp, _dp]
    L.orc_tp_central_moments_node.argtypes = [ctypes.c_int, _dp, _dp, _dp]
    L.orc_tp_init.argtypes = [ctypes.c_int, ctypes.c_int64, _dp, _dp, _dp]
    L.orc_tp_moments.argtypes = [ctypes.c_int, ctypes.c_int64, _dp, _dp, _dp]
    L.orc_tp_step.argtypes = [ctypes.c_int, _i64p, _dp, ctypes.c_int, _dp, _dp, ctypes.c_int64]
    L.orc_num_threads.argtypes = []
    for name in ("orc_tp_collide_node", "orc_tp_collide_node_rates", "orc_tp_equilibrium_node", "orc_tp_init",
                 "orc_tp_step", "orc_tp_moments", "orc_tp_central_moments_node",
                 "orc_tp_product_equilibrium_node", "orc_tp_weight", "orc_tp_velocities",
                 "orc_num_threads"):
        getattr(L, name).restype = ctypes.c_int
    if hasattr(L, "h37_collide_node"):
        from . import h37 as _h37
        _h37.declare(L)
    if hasattr(L, "hl_collide_node"):
        from . import hlat as _hlat
        _hlat.declare(L)


def _p(a):
    return a.ctypes.data_as(_dp)


def _c(a, dtype=np.float64):
    return np.ascontiguousarray(a, dtype=dtype)


def num_threads() -> int:
    return lib().orc_num_threads()


def tp_Q(D: int) -> int:
    return 3 ** D


def omega_from_tau(D: int, tau_per_order) -> np.ndarray:
    """omega[n] = 1/tau_n for orders n = 2..2D; tau_per_order[0] is tau_2.
    Orders past the given list take tau = 1.  omega[0] = omega[1] = 0."""
    om = np.zeros(2 * D + 1)
    taus = list(tau_per_order)
    for n in range(2, 2 * D + 1):
        t = taus[n - 2] if n - 2 < len(taus) else 1.0
        om[n] = 1.0 / t
    return om


def tp_weights(D: int) -> np.ndarray:
    w = np.zeros(tp_Q(D))
    lib().orc_tp_weight(D, _p(w))
    return w


def tp_velocities(D: int) -> np.ndarray:
    e = np.zeros((tp_Q(D), D), dtype=np.int32)
    lib().orc_tp_velocities(D, e.ctypes.data_as(_ip))
    return e


def tp_collide_node(D: int, omega, f, variant=ORC_DEFINITIONAL) -> np.ndarray:
    om = _c(omega)
    f = _c(f)
    out = np.zeros(tp_Q(D))
    if lib().orc_tp_collide_node(D, _p(om), variant, _p(f), _p(out)):
        raise ArithmeticError("singular central-moment system")
    return out


def tp_collide_node_rates(D: int, omega_a, f) -> np.ndarray:
    """Collision with one rate per central moment a (Q entries)."""
    om = _c(omega_a)
    f = _c(f)
    out = np.zeros(tp_Q(D))
    if lib().orc_tp_collide_node_rates(D, _p(om), _p(f), _p(out)):
        raise ArithmeticError("singular central-moment system")
    return out


def tp_equilibrium_node(D: int, rho: float, u) -> np.ndarray:
    """f_eq = C(u)^{-1} kappa_eq, by solving the central-moment system."""
    u = _c(np.resize(np.asarray(u, dtype=np.float64), 3))
    out = np.zeros(tp_Q(D))
    if lib().orc_tp_equilibrium_node(D, float(rho), _p(u), _p(out)):
        raise ArithmeticError("singular central-moment system")
    return out


def tp_product_equilibrium_node(D: int, rho: float, u) -> np.ndarray:
    u = _c(np.resize(np.asarray(u, dtype=np.float64), 3))
    out = np.zeros(tp_Q(D))
    lib().orc_tp_product_equilibrium_node(D, float(rho), _p(u), _p(out))
    return out


def tp_central_moments_node(D: int, u, f) -> np.ndarray:
    u = _c(np.resize(np.asarray(u, dtype=np.float64), 3))
    f = _c(f)
    out = np.zeros(tp_Q(D))
    lib().orc_tp_central_moments_node(D, _p(u), _p(f), _p(out))
    return out


def tp_init(D: int, rho, u) -> np.ndarray:
    """Equilibrium populations f[i, node] for fields rho[node], u[d, node]."""
    rho = _c(rho).reshape(-1)
    N = rho.size
    u = _c(u).reshape(D, N)
    f = np.zeros((tp_Q(D), N))
    if lib().orc_tp_init(D, N, _p(rho), _p(u), _p(f)):
        raise ArithmeticError("singular central-moment system")
    return f


def tp_moments(D: int, f):
    f = _c(f)
    N = f.shape[1]
    rho = np.zeros(N)
    u = np.zeros((D, N))
    lib().orc_tp_moments(D, N, _p(f), _p(rho), _p(u))
    return rho, u


def tp_step(D: int, dims, omega, f, nsteps: int = 1, variant=ORC_KRONECKER) -> np.ndarray:
    """Advance f (shape (Q, N), modified in place and returned) by nsteps
    collide-then-stream steps on the periodic grid dims = (nx, ny[, nz])."""
    assert f.dtype == np.float64 and f.flags.c_contiguous
    d = np.array(list(dims) + [1] * (3 - len(dims)), dtype=np.int64)
    om = _c(omega)
    post = np.empty_like(f)
    if lib().orc_tp_step(D, d.ctypes.data_as(_i64p), _p(om), variant, _p(f), _p(post), int(nsteps)):
        raise ArithmeticError("singular central-moment system")
    return f
