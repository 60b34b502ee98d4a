"""Pins of the FP64 oracle on the tensor-product lattices D2Q9 and D3Q27.

Each test checks the oracle against something other than itself: a library
quadrature, the paper's binomial transform, the textbook LBGK special case,
conservation laws, the defining relaxation condition, or the Chapman-Enskog
transport coefficient of the linear viscous mode.  None of these tests needs a GPU.
"""
import itertools
from math import comb

import numpy as np
import pytest
from numpy.polynomial.hermite_e import hermegauss

from oracle import analysis
from paper_1808_04406_gb300 import inputs

CS2 = 1.0 / 3.0


def _dfact_moment(a):
    """Gaussian moment E[xi^a] for a unit-variance Gaussian: (a-1)!! for even a, else 0."""
    if a % 2:
        return 0.0
    r = 1.0
    for k in range(a - 1, 0, -2):
        r *= k
    return r


def _central_bruteforce(e, f, u, alpha):
    """sum_i f_i prod_d (e_id - u_d)^alpha_d by direct summation."""
    p = np.ones(len(f))
    for d, a in enumerate(alpha):
        p = p * (e[:, d] - u[d]) ** a
    return float(np.sum(f * p))


def _alphas(D):
    """Moment multi-indices in the oracle's order a = sum_d alpha_d 3^d."""
    return [tuple((a // 3 ** d) % 3 for d in range(D)) for a in range(3 ** D)]


def _near_eq(orc, D, rng, du=0.08, noise=2e-3):
    u = rng.uniform(-du, du, D)
    rho = 1.0 + rng.uniform(-0.05, 0.05)
    return orc.tp_product_equilibrium_node(D, rho, u) + rng.normal(0.0, noise, 3 ** D)


@pytest.mark.parametrize("D", [2, 3])
def test_weights_are_the_gauss_hermite_product_rule(orc, D):
    """Sec. II.A, Eq. quad: D1Q3^D is the product of the 3-point Gauss-Hermite rule
    (numpy's hermegauss), abscissas sqrt(3)*e, so c_s^2 = 1/3 in lattice units; it
    integrates every monomial of per-axis degree <= 5 exactly and fails at 6."""
    x, wg = hermegauss(3)
    wg = wg / wg.sum()
    order = np.argsort(x)  # -sqrt3, 0, +sqrt3 <-> e = -1, 0, 1
    w, e = orc.tp_weights(D), orc.tp_velocities(D)
    for i in range(3 ** D):
        expect = np.prod([wg[order[e[i, d] + 1]] for d in range(D)])
        assert w[i] == pytest.approx(expect, rel=1e-14)
        for d in range(D):
            assert np.sqrt(3.0) * e[i, d] == pytest.approx(x[order[e[i, d] + 1]], abs=1e-14)
    for alpha in itertools.product(range(6), repeat=D):
        got = np.sum(w * np.prod([e[:, d].astype(float) ** alpha[d] for d in range(D)], axis=0))
        expect = np.prod([CS2 ** (a / 2) * _dfact_moment(a) for a in alpha])
        assert got == pytest.approx(expect, abs=1e-15)
    got6 = np.sum(w * e[:, 0].astype(float) ** 6)
    assert abs(got6 - CS2 ** 3 * 15) > 0.1


@pytest.mark.parametrize("D", [2, 3])
def test_central_moments_follow_the_binomial_transform(orc, D):
    """Appendix, Eq. trans-a (monomial form): central moments about u equal
    sum_beta prod_d C(alpha_d, beta_d) (-u_d)^(alpha_d - beta_d) times raw moments."""
    rng = np.random.default_rng(1)
    e = orc.tp_velocities(D).astype(float)
    for _ in range(5):
        f = rng.uniform(0.0, 1.0, 3 ** D)
        u = rng.uniform(-0.3, 0.3, D)
        kap = orc.tp_central_moments_node(D, u, f)
        for a, alpha in enumerate(_alphas(D)):
            s = 0.0
            for beta in itertools.product(*[range(al + 1) for al in alpha]):
                c = np.prod([comb(alpha[d], beta[d]) * (-u[d]) ** (alpha[d] - beta[d]) for d in range(D)])
                raw = np.sum(f * np.prod([e[:, d] ** beta[d] for d in range(D)], axis=0))
                s += c * raw
            assert kap[a] == pytest.approx(s, abs=1e-14)


@pytest.mark.parametrize("D", [2, 3])
def test_equilibrium_has_maxwellian_moments(orc, D):
    """The equilibrium f_eq = C(u)^{-1} kappa_eq carries the isothermal Maxwellian's
    moments through second order (Sec. II, Eq. maxwellian with theta = c_s^2):
    sum f = rho, sum f e = rho u, sum f e_a e_b = rho (u_a u_b + c_s^2 delta_ab),
    and equals the LBGK product form rho prod_d g(e_d, u_d)."""
    rng = np.random.default_rng(2)
    e = orc.tp_velocities(D).astype(float)
    for _ in range(5):
        rho = rng.uniform(0.9, 1.1)
        u = rng.uniform(-0.1, 0.1, D)
        f = orc.tp_equilibrium_node(D, rho, u)
        assert np.all(f > 0)
        assert f.sum() == pytest.approx(rho, rel=1e-14)
        np.testing.assert_allclose(e.T @ f, rho * u, atol=1e-15)
        P = (e.T * f) @ e
        np.testing.assert_allclose(P, rho * (np.outer(u, u) + CS2 * np.eye(D)), atol=1e-15)
        np.testing.assert_allclose(f, orc.tp_product_equilibrium_node(D, rho, u), atol=1e-15)


@pytest.mark.parametrize("D", [2, 3])
def test_equal_rates_reduce_to_lbgk(orc, D):
    """Sec. II.C after Eq. regnmrt: with every relaxation time equal, CM-MRT is LBGK
    (Eq. lbgk) with the same equilibrium; distinct rates must differ from it."""
    rng = np.random.default_rng(3)
    for tau in (0.51, 0.6, 1.0, 1.7):
        om = orc.omega_from_tau(D, [tau] * (2 * D - 1))
        for _ in range(4):
            f = _near_eq(orc, D, rng)
            a = orc.tp_collide_node(D, om, f, orc.ORC_DEFINITIONAL)
            b = orc.tp_collide_node(D, om, f, orc.ORC_LBGK)
            np.testing.assert_allclose(a, b, atol=2e-15)
    om = orc.omega_from_tau(D, [0.6, 0.9] + [1.0] * (2 * D - 3))
    f = _near_eq(orc, D, rng)
    assert np.abs(orc.tp_collide_node(D, om, f) - orc.tp_collide_node(D, om, f, orc.ORC_LBGK)).max() > 1e-6
    # grid-level: several steps of both agree
    dims = (6, 5, 4)[:D]
    rho, u = inputs.random_noise(dims, seed=7)
    om = orc.omega_from_tau(D, [0.7] * (2 * D - 1))
    f1 = orc.tp_init(D, rho, u)
    f2 = f1.copy()
    orc.tp_step(D, dims, om, f1, 5, orc.ORC_DEFINITIONAL)
    orc.tp_step(D, dims, om, f2, 5, orc.ORC_LBGK)
    np.testing.assert_allclose(f1, f2, atol=1e-14)


@pytest.mark.parametrize("D", [2, 3])
def test_equilibrium_is_a_fixed_point_and_mass_momentum_are_conserved(orc, D):
    """Sec. II.B: f^(0) is unchanged by collision (M <= N); Sec. II.C: the zeroth and
    first moments of Omega vanish, so mass and momentum are conserved exactly."""
    rng = np.random.default_rng(4)
    e = orc.tp_velocities(D).astype(float)
    om = orc.omega_from_tau(D, [0.55, 0.8, 1.2, 1.9, 0.7][: 2 * D - 1])
    for _ in range(5):
        rho = rng.uniform(0.9, 1.1)
        u = rng.uniform(-0.1, 0.1, D)
        feq = orc.tp_equilibrium_node(D, rho, u)
        for v in (orc.ORC_DEFINITIONAL, orc.ORC_KRONECKER):
            np.testing.assert_allclose(orc.tp_collide_node(D, om, feq, v), feq, atol=3e-16)
        f = _near_eq(orc, D, rng)
        fs = orc.tp_collide_node(D, om, f)
        assert fs.sum() == pytest.approx(f.sum(), abs=1e-15)
        np.testing.assert_allclose(e.T @ fs, e.T @ f, atol=1e-15)


@pytest.mark.parametrize("D", [2, 3])
def test_relaxation_condition_eq_omega(orc, D):
    """Eq. omega, for every order: each central moment of Omega equals -omega_n times
    the same central moment of f^(1) = f - f^(0) (brute-force moments)."""
    rng = np.random.default_rng(5)
    e = orc.tp_velocities(D).astype(float)
    taus = [0.55, 0.8, 1.3, 1.9, 0.7][: 2 * D - 1]
    om = orc.omega_from_tau(D, taus)
    for _ in range(5):
        f = _near_eq(orc, D, rng, noise=5e-3)
        rho = f.sum()
        u = (e.T @ f) / rho
        f1 = f - orc.tp_product_equilibrium_node(D, rho, u)
        Om = orc.tp_collide_node(D, om, f) - f
        for alpha in _alphas(D):
            n = sum(alpha)
            kO = _central_bruteforce(e, Om, u, alpha)
            k1 = _central_bruteforce(e, f1, u, alpha)
            if n <= 1:
                assert abs(kO) < 1e-15 and abs(k1) < 1e-15
            else:
                assert kO == pytest.approx(-om[n] * k1, abs=1e-15, rel=1e-11)


@pytest.mark.parametrize("D", [2, 3])
def test_definitional_and_kronecker_variants_agree(orc, D):
    rng = np.random.default_rng(6)
    om = orc.omega_from_tau(D, [0.52, 1.1, 0.8, 1.5, 1.2][: 2 * D - 1])
    for _ in range(10):
        f = _near_eq(orc, D, rng, du=0.2, noise=1e-2)
        a = orc.tp_collide_node(D, om, f, orc.ORC_DEFINITIONAL)
        b = orc.tp_collide_node(D, om, f, orc.ORC_KRONECKER)
        np.testing.assert_allclose(a, b, atol=1e-15)


@pytest.mark.parametrize("D", [2, 3])
def test_streaming_moves_population_i_by_e_i(orc, D):
    """Sec. II.A, Eq. lbgk left side: f_i(x + xi_i, t + 1).  With zero collision rates
    the step is pure streaming: each population plane is rolled by its velocity."""
    dims = (5, 4, 3)[:D]
    rng = np.random.default_rng(8)
    N = int(np.prod(dims))
    w = orc.tp_weights(D)
    e = orc.tp_velocities(D)
    f = w[:, None] * (1.0 + 0.1 * rng.uniform(size=(3 ** D, N)))
    g = orc.tp_step(D, dims, np.zeros(2 * D + 1), f.copy(), 1)
    shape = tuple(reversed(dims))  # arrays are [z, y, x]
    for i in range(3 ** D):
        plane = f[i].reshape(shape)
        shift = tuple(int(e[i, d]) for d in reversed(range(D)))
        # zero rates make the collision the identity up to the rounding of C^-1 C
        np.testing.assert_allclose(g[i].reshape(shape), np.roll(plane, shift, axis=tuple(range(D))), rtol=1e-13)


def _shear_rate(orc, D, dims, taus, u0, steps, every):
    rho, u = inputs.shear_wave(dims, amplitude=1e-4, u0=u0, mode=1, k_axis=0, u_axis=1)
    om = orc.omega_from_tau(D, taus)
    f = orc.tp_init(D, rho, u)
    ts, amps = [], []
    mode = [1] + [0] * (D - 1)
    for s in range(0, steps + 1, every):
        if s:
            orc.tp_step(D, dims, om, f, every)
        _, uu = orc.tp_moments(D, f)
        ts.append(s)
        amps.append(analysis.mode_amplitude(uu[1], dims, mode))
    return analysis.fit_decay_rate(ts, amps)


@pytest.mark.parametrize("D,dims", [(2, (64, 1)), (3, (64, 1, 1))])
@pytest.mark.parametrize("tau2,u0", [(0.6, 0.0), (0.8, 0.0), (0.8, 0.1), (0.53, 0.05)])
def test_shear_wave_gives_chapman_enskog_viscosity(orc, D, dims, tau2, u0):
    """Eq. dr, viscous mode: |A| decays at nu k^2 exactly, with nu = c_s^2 (tau_2 - 1/2)
    (Eq. sigma with tau -> tau_2), independent of a base flow perpendicular to k
    (Sec. III.A, Galilean test) and of the higher-order rates."""
    k = 2 * np.pi / dims[0]
    nu = CS2 * (tau2 - 0.5)
    steps = int(round(0.7 / (nu * k * k)))
    steps = max(50, min(steps, 1500))
    gamma = _shear_rate(orc, D, dims, [tau2, 0.9, 1.3, 0.75, 1.1][: 2 * D - 1], u0, steps, max(1, steps // 25))
    # the finite-k lattice correction is O(k^2): below 0.2 % at 64 nodes per wavelength
    assert gamma / (k * k) == pytest.approx(nu, rel=3e-3)


@pytest.mark.parametrize("D,dims", [(2, (64, 1)), (3, (64, 1, 1))])
def test_shear_viscosity_is_independent_of_a_perpendicular_base_flow(orc, D, dims):
    """Sec. III.A, Galilean test: with the base flow u0 perpendicular to k the measured
    viscosity does not depend on u0 (central moments remove the u0 dependence)."""
    taus = [0.7, 0.6, 1.4, 0.8, 1.2][: 2 * D - 1]
    rates = [_shear_rate(orc, D, dims, taus, u0, 600, 50) for u0 in (0.0, 0.05, 0.1)]
    assert max(rates) - min(rates) < 1e-8 * rates[0]


def test_taylor_green_2d_decays_at_the_analytic_rate(orc):
    """2D Taylor-Green vortex (incompressible NS solution): the velocity field keeps its
    shape and decays as exp(-2 nu k^2 t), kinetic energy as exp(-4 nu k^2 t).
    D2Q9, 64^2, u0 = 0.02, tau_2 = 0.6 (nu = 1/30), higher orders tau = 1."""
    n, u0, tau2 = 64, 0.02, 0.6
    rho, u = inputs.taylor_green_2d(n, n, u0=u0)
    nu = CS2 * (tau2 - 0.5)
    k = 2 * np.pi / n
    f = orc.tp_init(2, rho, u)
    steps = 600
    orc.tp_step(2, (n, n), orc.omega_from_tau(2, [tau2, 1.0, 1.0]), f, steps)
    _, uu = orc.tp_moments(2, f)
    expect = u * np.exp(-2 * nu * k * k * steps)
    err = np.abs(uu - expect).max() / np.abs(expect).max()
    assert err < 3e-3
    ke = 0.5 * np.sum(uu ** 2) / (0.5 * np.sum(u ** 2))
    assert ke == pytest.approx(np.exp(-4 * nu * k * k * steps), rel=3e-3)
