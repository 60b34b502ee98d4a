"""GPU parity of caller-supplied Hermite lattices (the minimal 17- and
37-velocity rules of Sec. III.A, Fig. 2) against the general FP64 oracle.

Populations are matched by velocity vector (the library keeps the caller's
order); velocities crossing the C ABI are in lattice units, the oracle's in
Hermite units (u_H = c u).  Tolerances: FP64 <= 2e-14 per step (as the
37-velocity lattice), FP32 <= 1e-5 relative on the fields after 1000 steps
(correctly rounded transforms, the FP32 default)."""
import numpy as np
import pytest

from oracle import hlat
from paper_1808_04406_gb300 import gen_d2q37, gen_rules, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lbm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1808_04406_gb300 import build as libbuild
    libbuild.build()
    from paper_1808_04406_gb300 import lbm as L
    L.load()
    return L


RULES = ["E7-A", "E7-B", "E7-C", "E7-D", "E9-A", "E9-B", "E9-C", "E9-D"]


def _pair(name, order=None):
    e, w, c, n = gen_rules.rule(name)
    n = n if order is None else order
    degree = int(name[1])
    lab = name[-1]
    eo, wo, co = [(x[1], x[2], x[3]) for x in hlat.rule_set(degree) if x[0] == lab][0]
    lat = hlat.Lattice(eo, wo, co, n)
    idx = {tuple(v): i for i, v in enumerate(eo)}
    perm = np.array([idx[tuple(v)] for v in e])  # library velocity k -> oracle velocity perm[k]
    return (e, w, c, n), lat, perm


def _fields(dims, seed):
    rho, u = inputs.random_smooth(dims, seed=seed, du=0.03, drho=0.01)
    rng = np.random.default_rng(seed + 7)
    theta = 1.1 + 0.02 * np.cos(2 * np.pi * np.arange(int(np.prod(dims))) / 29.0 + rng.uniform())
    return rho, u, theta


TAUS = [0.58, 0.7, 0.62]


@pytest.mark.parametrize("name", RULES)
@pytest.mark.parametrize("thermal", [True, False])
@pytest.mark.parametrize("dims", [(13, 7), (3, 4)])
def test_fp64_steps_match_the_oracle(lbm, name, thermal, dims):
    rule, lat, perm = _pair(name)
    rho, u, theta = _fields(dims, seed=5)
    if not thermal:
        theta = np.ones_like(theta)
    flags = lbm.LBM_THERMAL if thermal else 0
    sim = lbm.HermiteSimulation(rule, dims, TAUS, storage="f64", flags=flags, theta_ref=1.1)
    sim.init_fields(rho, u, theta)
    f = lat.init(rho, u * rule[2], theta)
    np.testing.assert_allclose(sim.populations(), f[perm], atol=1e-15)
    om = lat.omega_from_tau(TAUS)
    for _ in range(3):
        sim.step(1)
        lat.step(dims, om, f, 1, thermal)
        assert np.abs(sim.populations() - f[perm]).max() <= 2e-14
    grho, gu, gth = sim.moments(with_theta=True)
    orho, ou, oth = lat.moments(f, thermal)
    np.testing.assert_allclose(grho, orho, atol=1e-14)
    np.testing.assert_allclose(gu, ou / rule[2], atol=1e-14)
    np.testing.assert_allclose(gth, oth if thermal else 1.0, atol=1e-13)


def test_order_three_on_a_37_velocity_rule(lbm):
    rule, lat, perm = _pair("E9-B", order=3)
    dims = (8, 6)
    rho, u, theta = _fields(dims, seed=9)
    sim = lbm.HermiteSimulation(rule, dims, TAUS, storage="f64", flags=lbm.LBM_THERMAL, theta_ref=1.1)
    sim.init_fields(rho, u, theta)
    f = lat.init(rho, u * rule[2], theta)
    om = lat.omega_from_tau(TAUS)
    for _ in range(2):
        sim.step(1)
        lat.step(dims, om, f, 1, True)
    assert np.abs(sim.populations() - f[perm]).max() <= 2e-14


@pytest.mark.parametrize("name", ["E7-D", "E9-C"])
def test_fp32_long_run_parity(lbm, name):
    """FP32 storage with the correctly rounded transforms (the default): u,
    theta and rho - 1 within 1e-5 of the FP64 oracle after 1000 steps."""
    rule, lat, perm = _pair(name)
    dims = (34, 20)
    taus = [0.5 + 0.02, 0.5 + 0.04, 0.52]
    rho, u, theta = _fields(dims, seed=11)
    sim = lbm.HermiteSimulation(rule, dims, taus, storage="f32", flags=lbm.LBM_THERMAL, theta_ref=1.1)
    sim.init_fields(rho, u, theta)
    sim.step(1000)
    f = lat.init(rho, u * rule[2], theta)
    lat.step(dims, lat.omega_from_tau(taus), f, 1000, True)
    grho, gu, gth = sim.moments(with_theta=True)
    orho, ou, oth = lat.moments(f, True)
    rel = lambda a, b: np.abs(a - b).max() / np.abs(b).max()
    assert rel(gu, ou / rule[2]) <= 1e-5
    assert rel(gth, oth) <= 1e-5
    assert rel(grho, orho) <= 1e-5
    assert rel(grho - 1, orho - 1) <= 1e-5


def test_e9_a_with_order_four_is_the_built_in_37_velocity_lattice(lbm):
    """The same rule through the caller-supplied path and through the compiled-in
    tables: the same collision (Hermite space, K = 6), projections summed in a
    different order."""
    rule = gen_rules.rule("E9-A")
    dims = (11, 9)
    rho, u, theta = _fields(dims, seed=13)
    a = lbm.HermiteSimulation(rule, dims, TAUS, storage="f64", flags=lbm.LBM_THERMAL, theta_ref=1.2)
    b = lbm.Simulation("D2Q37", dims, TAUS, storage="f64", flags=lbm.LBM_THERMAL, theta_ref=1.2)
    for s in (a, b):
        s.init_fields(rho, u, theta)
        s.step(5)
    e_lib, _, _ = gen_d2q37.solve()
    idx = {tuple(v): i for i, v in enumerate(rule[0])}
    perm = np.array([idx[tuple(v)] for v in e_lib])
    np.testing.assert_allclose(a.populations()[perm], b.populations(), rtol=0, atol=5e-14)


def test_rejects_rules_shapes_and_storage_it_cannot_take(lbm):
    e, w, c, n = gen_rules.rule("E7-B")
    with pytest.raises(lbm.LBMError):
        lbm.HermiteSimulation((e, w, c, 4), (8, 8), TAUS)  # degree 7 cannot carry N = 4
    with pytest.raises(lbm.LBMError):
        lbm.HermiteSimulation((e, w, c * 1.01, 3), (8, 8), TAUS)  # not exact any more
    with pytest.raises(lbm.LBMError):
        lbm.HermiteSimulation((e, w, c, 3), (8, 8), TAUS, storage="f16")
    with pytest.raises(lbm.LBMError):
        lbm.HermiteSimulation((e, w, c, 3), (2, 8), TAUS)
    with pytest.raises(lbm.LBMError):
        lbm.HermiteSimulation((e, w, c, 3), (8, 8), TAUS, flags=lbm.LBM_K72)


@pytest.mark.parametrize("name", ["E7-C", "E9-A"])
def test_shear_viscosity_from_the_device_fit(lbm, name):
    """nu = theta (tau_2 - 1/2) within 1 % at 64 nodes per wavelength (mode 1)."""
    rule = gen_rules.rule(name)
    n, nu = 64, 0.1
    taus = [0.5 + nu, 0.5 + nu, 0.5 + nu]
    rho, u = inputs.shear_wave((n, n), amplitude=1e-4, mode=1, k_axis=0, u_axis=1)
    sim = lbm.HermiteSimulation(rule, (n, n), taus, storage="f64", flags=lbm.LBM_THERMAL, theta_ref=1.0)
    sim.init_fields(rho, u, np.ones(n * n))
    k = 2 * np.pi / n
    steps = int(0.7 / (nu * k * k / rule[2] ** 2))
    fit, _ = sim.mode_history(2, (1, 0), 40, max(1, steps // 39))
    nu_m = fit[0] * rule[2] ** 2 / (k * k)
    assert nu_m == pytest.approx(nu, rel=1e-2)
