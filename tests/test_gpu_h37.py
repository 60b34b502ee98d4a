"""GPU parity of the 37-velocity thermal CM-MRT (Hermite N = M = 4) against the
FP64 oracle, and the paper's linear-mode measurements (Sec. III.A) on the GPU.

The library orders the 37 velocities so that opposite ones sit at i and 36 - i;
the oracle has its own order, so populations are compared by velocity vector.
Velocities crossing the C ABI are in lattice units; the oracle works in the
paper's (Hermite) units, u_H = c u with xi = c e.
"""
import numpy as np
import pytest

import oracle
import oracle.h37 as H
from paper_1808_04406_gb300 import gen_d2q37, inputs

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
    oracle.lib()
    return L


def _perm():
    """perm[k] = oracle index of the library's velocity k."""
    e_lib, _, _ = gen_d2q37.solve()
    e_orc, _, _ = H.lattice()
    idx = {tuple(v): i for i, v in enumerate(e_orc)}
    return np.array([idx[tuple(v)] for v in e_lib])


def _sim(lbm, dims, taus, storage="f64", thermal=True, flags=0, theta_ref=1.2):
    f = flags | (lbm.LBM_THERMAL if thermal else 0)
    return lbm.Simulation("D2Q37", dims, taus, storage=storage, flags=f, theta_ref=theta_ref)


def _fields(dims, seed):
    rho, u = inputs.random_smooth(dims, seed=seed, du=0.03, drho=0.01)
    rng = np.random.default_rng(seed + 100)
    theta = 1.2 + 0.02 * np.cos(2 * np.pi * np.arange(int(np.prod(dims))) / 37.0 + rng.uniform())
    return rho, u, theta


TAUS = [0.5 + 0.1 / 1.2, 0.5 + 0.2 / 1.2, 0.9]


@pytest.mark.parametrize("thermal", [True, False])
@pytest.mark.parametrize("dims", [(133, 7), (3, 3), (5, 4)])
def test_fp64_steps_match_the_oracle_both_parities(lbm, dims, thermal):
    rho, u, theta = _fields(dims, seed=3)
    if not thermal:
        theta = np.ones_like(theta)
    sim = _sim(lbm, dims, TAUS, "f64", thermal)
    sim.init_fields(rho, u, theta)
    c = H.lattice()[2]
    f = H.init(rho, u * c, theta)
    P = _perm()
    np.testing.assert_allclose(sim.populations(), f[P], atol=1e-15)
    om = H.omega_from_tau(TAUS)
    for s in range(1, 4):
        sim.step(1)
        H.step(dims, om, f, 1, thermal, H.H37_CLOSED)
        assert np.abs(sim.populations() - f[P]).max() <= 2e-14
    grho, gu, gth = sim.moments(with_theta=True)
    orho, ou, oth = H.moments(f, thermal)
    np.testing.assert_allclose(grho, orho, atol=1e-14)
    np.testing.assert_allclose(gu, ou / c, atol=1e-14)
    np.testing.assert_allclose(gth, oth if thermal else np.ones_like(oth), atol=1e-13)


def _long_run(lbm, dims, storage, steps, flags=0):
    """rho, u, theta relative errors against the FP64 oracle after `steps` steps:
    D2Q37 thermal CM-MRT, nu = 0.02, kappa = 0.04, tau_4 = tau_2 (with tau_4 far
    from tau_2 this flow diverges: the (omega_4 - omega_2) delta coupling of
    Eq. mrt)."""
    taus = [0.5 + 0.02 / 1.2, 0.5 + 0.04 / 1.2, 0.5 + 0.02 / 1.2]
    rho, u, theta = _fields(dims, seed=5)
    sim = _sim(lbm, dims, taus, storage, flags=flags)
    sim.init_fields(rho, u, theta)
    c = H.lattice()[2]
    f = H.init(rho, u * c, theta)
    out, done = [], 0
    rel = lambda a, b: np.abs(a - b).max() / np.abs(b).max()
    for n in ([steps] if np.isscalar(steps) else steps):
        sim.step(n - done)
        H.step(dims, H.omega_from_tau(taus), f, n - done, True, H.H37_CLOSED)
        done = n
        grho, gu, gth = sim.moments(with_theta=True)
        orho, ou, oth = H.moments(f, True)
        out.append({"u": rel(gu, ou / c), "rho": rel(grho, orho), "theta": rel(gth, oth),
                    "rho-1": rel(grho - 1, orho - 1)})
    return out


@pytest.mark.parametrize("storage,steps,tol,tol_dr,dims", [
    ("f64", 400, 1e-12, 1e-11, (130, 40)), ("f32", 1000, 1e-5, 1e-5, (130, 40)),
    ("f32", 1000, 1e-5, 1e-5, (132, 40)), ("f32", 1000, 1e-5, 1e-5, (66, 21))])
def test_long_run_parity_on_a_ragged_grid(lbm, storage, steps, tol, tol_dr, dims):
    """130 x 40 (two 128-wide x tiles, ragged) and other shapes: rho, u, theta
    within the tolerance of the FP64 oracle after 400 (FP64) or 1000 (FP32)
    steps, and rho - 1 on its own.  FP32 storage computes the two Hermite
    transforms (Eqs. an, fi) correctly rounded (compensated products and sums,
    constants as FP32 pairs): measured ~4e-7 on u and ~3e-6 on rho - 1, flat in
    time.  In FP64, rho - 1 relative to its own small maximum (~1e-3) carries
    the rounding of rho ~ 1 itself (measured 3e-12), hence 1e-11 there."""
    (e,) = _long_run(lbm, dims, storage, steps)
    for k in ("u", "rho", "theta"):
        assert e[k] <= tol, (k, e)
    assert e["rho-1"] <= tol_dr, e


def test_plain_fp32_transforms_drift_linearly_and_the_correctly_rounded_ones_do_not(lbm):
    """The stated error of the LBM_FAST_TRANSFORMS option (plain FP32 Hermite
    transforms, the two-node sweep).  With the constants rounded once to FP32
    the two transforms are not exact inverses (the momentum row of the round
    trip is off by ~8e-9 per step), and every sum rounds at each term; the
    errors recur every step on this slowly varying flow, so the velocity error
    grows linearly: ~1.1e-5 relative after 1000 steps, ~2.4e-5 after 2000.  The
    correctly rounded transforms of the default FP32 path stay below 1e-6 on u
    over the same run, so the drift is FP32 rounding in the transforms, not the
    model (which the FP64 path matches to 1e-12)."""
    dims = (132, 40)
    fast = _long_run(lbm, dims, "f32", [500, 1000, 2000], lbm.LBM_FAST_TRANSFORMS)
    exact = _long_run(lbm, dims, "f32", [500, 1000, 2000])
    assert fast[1]["u"] <= 2e-5 and fast[2]["u"] <= 4e-5
    # linear growth: doubling the steps roughly doubles the plain error ...
    assert 1.5 <= fast[2]["u"] / fast[1]["u"] <= 2.6
    # ... while the correctly rounded error stays flat and > 10x smaller
    for k in range(3):
        assert exact[k]["u"] <= 1e-6
    for k in (1, 2):
        assert exact[k]["u"] * 10 <= fast[k]["u"]
    assert exact[2]["u"] <= 2.0 * exact[0]["u"]


@pytest.mark.parametrize("storage,bits,sr", [("f16", 11, False), ("bf16", 8, False), ("f16", 11, True),
                                             ("bf16", 8, True)])
def test_low_precision_offsets_one_step_bound(lbm, storage, bits, sr):
    """FP16 / BF16 offsets (f - f_ref)/w, FP32 collision: one step from the GPU's
    own state matches the oracle within half an ulp of the stored offset (one
    ulp with stochastic rounding, which rounds to either neighbour)."""
    dims = (40, 9)
    rho, u, theta = _fields(dims, seed=7)
    sim = _sim(lbm, dims, TAUS, storage, flags=lbm.LBM_STOCHASTIC_ROUND if sr else 0)
    sim.init_fields(rho, u, theta)
    P = _perm()
    inv = np.argsort(P)
    w_lib = gen_d2q37.solve()[1][:, None]
    om = H.omega_from_tau(TAUS)
    for _ in range(2):
        f_lib = sim.populations()
        f = np.ascontiguousarray(f_lib[inv])
        H.step(dims, om, f, 1, True, H.H37_CLOSED)
        sim.step(1)
        g = sim.populations()
        fo = f[P]
        fref = H.equilibrium_node(1.0, np.zeros(2), 1.2)[P][:, None]
        s = (fo - fref) / w_lib
        bound = w_lib * 2.0 ** -bits * np.abs(s) * (2.1 if sr else 1.05) + 2e-7
        assert np.all(np.abs(g - fo) <= bound)


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("flags,thermal", [(0, True), (0, False), ("K72", True), ("RAW", True)])
def test_two_node_kernel_matches_the_one_node_kernel(lbm, monkeypatch, storage, flags, thermal):
    """The packed FP32x2 two-node sweep (even nx) against the one-node sweep on
    the same state: both are FP32 evaluations of the same formulas, in a different
    rounding order, so after 2 steps (both parities) they agree to a few FP32 ulps
    (FP16 / BF16: a stored value may round to a neighbouring code)."""
    dims = (36, 11)
    fl = {"K72": lbm.LBM_K72, "RAW": lbm.LBM_RAW_MRT}.get(flags, 0)
    if storage == "f32":
        fl |= lbm.LBM_FAST_TRANSFORMS  # the two-node sweep runs the plain FP32 transforms
    rho, u, theta = _fields(dims, seed=9)
    out = []
    for mode in ("scalar", "pair"):
        if mode == "scalar":
            monkeypatch.setenv("LBM_H37_SWEEP", "scalar")
        else:
            monkeypatch.delenv("LBM_H37_SWEEP", raising=False)
        sim = _sim(lbm, dims, TAUS, storage, thermal, fl)
        sim.init_fields(rho, u, theta if thermal else np.ones_like(theta))
        sim.step(2)
        out.append(sim.populations())
    w_lib = gen_d2q37.solve()[1][:, None]
    ulp = {"f32": 2.0 ** -23 * 64, "f16": 2.0 ** -10 * 2, "bf16": 2.0 ** -7 * 2}[storage]
    err = np.abs(out[0] - out[1]) / w_lib
    assert err.max() <= ulp * max(1.0, np.abs((out[0] - w_lib) / w_lib).max()), err.max()


@pytest.mark.parametrize("flag,variant,K", [("K72", "closed", 72.0), ("RAW", "raw", 6.0)])
def test_model_options_match_the_oracle(lbm, flag, variant, K):
    dims = (17, 6)
    rho, u, theta = _fields(dims, seed=9)
    flags = lbm.LBM_K72 if flag == "K72" else lbm.LBM_RAW_MRT
    sim = _sim(lbm, dims, TAUS, "f64", True, flags)
    sim.init_fields(rho, u, theta)
    c = H.lattice()[2]
    f = H.init(rho, u * c, theta)
    v = H.H37_CLOSED if variant == "closed" else H.H37_RAWMRT
    for _ in range(2):
        sim.step(1)
        H.step(dims, H.omega_from_tau(TAUS), f, 1, True, v, K)
        assert np.abs(sim.populations() - f[_perm()]).max() <= 2e-14


def test_mass_momentum_energy_conserved_on_the_gpu(lbm):
    dims = (64, 16)
    rho, u, theta = _fields(dims, seed=11)
    sim = _sim(lbm, dims, TAUS, "f64")
    sim.init_fields(rho, u, theta)

    def totals():
        r, uu, th = sim.moments(with_theta=True)
        c = H.lattice()[2]
        uh = uu * c
        return np.array([r.sum(), (r * uh[0]).sum(), (r * uh[1]).sum(), (r * ((uh ** 2).sum(0) + 2 * th)).sum()])

    t0 = totals()
    sim.step(7)
    np.testing.assert_allclose(totals(), t0, rtol=1e-13, atol=1e-12)


@pytest.mark.parametrize("storage,dims,sr", [("f16", (64, 18), False), ("f32", (38, 11), False),
                                             ("bf16", (64, 18), True), ("f32", (33, 7), False), ("f64", (20, 6), False)])
def test_step_totals_are_those_of_the_state_the_step_advanced_from(lbm, storage, dims, sr):
    """lbm_step_totals on the 37-velocity lattice = lbm_reduce just before
    lbm_step(1), and the same step (bit-identical populations afterwards).  The
    two-node kernel accumulates the totals itself (even nx, 16/32-bit storage,
    also with stochastic rounding); odd nx and FP64 reduce, then sweep."""
    rho, u, theta = _fields(dims, seed=21)
    flags = lbm.LBM_STOCHASTIC_ROUND if sr else 0
    a = _sim(lbm, dims, TAUS, storage, flags=flags)
    b = _sim(lbm, dims, TAUS, storage, flags=flags)
    for s in (a, b):
        s.init_fields(rho, u, theta)
    n = int(np.prod(dims))
    exact = storage == "f64" or dims[0] % 2
    for _ in range(4):
        want = b.reduce()
        b.step(1)
        got = a.step_totals()
        if exact:
            np.testing.assert_array_equal(got, want)
        else:
            np.testing.assert_allclose(got, want, rtol=1e-6, atol=1e-8 * n)
    np.testing.assert_array_equal(a.populations(), b.populations())
    assert a.status() == 0


def test_step_totals_async_equal_the_synchronous_ones(lbm):
    """On the 37-velocity lattice (FP16, fused totals): K lbm_step_totals_async
    calls with no wait in between give, after one synchronisation, the totals of
    K lbm_step_totals bit for bit and the same populations."""
    dims = (64, 18)
    rho, u, theta = _fields(dims, seed=22)
    a = _sim(lbm, dims, TAUS, "f16")
    c = _sim(lbm, dims, TAUS, "f16")
    for s in (a, c):
        s.init_fields(rho, u, theta)
    K = 5
    want = np.stack([a.step_totals() for _ in range(K)])
    out = torch.zeros((K, 5), dtype=torch.float64).pin_memory()
    for k in range(K):
        c.step_totals_async(out.data_ptr() + 40 * k)
    assert c.status() == 0
    np.testing.assert_array_equal(out.numpy(), want)
    np.testing.assert_array_equal(c.populations(), a.populations())


def _decay(lbm, n, pr, kind, storage="f16", mode=10, amp=1e-3, u0=0.0, flags=0):
    if storage.endswith("+sr"):
        storage, flags = storage[:-3], flags | lbm.LBM_STOCHASTIC_ROUND
    theta0, nu = 1.2, 0.1
    kap = nu / pr
    taus = [0.5 + nu / theta0, 0.5 + kap / theta0, 1.0]
    dims = (n, n)
    if kind == "thermal":
        rho, u, th = inputs.thermal_wave(dims, amplitude=amp, theta0=theta0, mode=mode, u0=u0)
        field = 3
    else:
        rho, u = inputs.shear_wave(dims, amplitude=amp, u0=u0, mode=mode, k_axis=0, u_axis=1)
        th = np.full(rho.size, theta0)
        field = 2
    sim = _sim(lbm, dims, taus, storage, True, flags, theta_ref=theta0)
    sim.init_fields(rho, u, th)
    c = H.lattice()[2]
    k = 2 * np.pi * mode / n
    D = nu if kind == "viscous" else kap
    steps = int(0.7 / (D * k * k / c ** 2))
    n_rec = 40
    fit, _ = sim.mode_history(field, (mode, 0), n_rec, max(1, steps // (n_rec - 1)))
    sim.close()
    return fit[0] * c ** 2 / (k * k), D


# Stated errors of the 1024^2, mode-10 measurement against theta0 (tau - 1/2):
# FP32 (and FP64) storage carry only the lattice's O(k^2) error of the viscous
# mode (+0.40 %, as in the oracle at ~100 nodes per wavelength; kappa within
# 0.4 %, largest at Pr = 2 where tau_3 is closest to 1/2).  FP16 offsets add
# quantization error: the half-ulp of a stored offset (2^-12 relative) is as
# large as a slow mode's decay per step, and round-to-nearest then stalls the
# decay.  Measured at Pr = 0.5: nu +1.1 %, kappa +2.0 .. +2.3 %, Pr -0.8 .. -1.2 %;
# at Pr = 2 (kappa k^2 / c^2 = 1.3e-4 per step) kappa comes out 23 % low, so
# round-to-nearest FP16 offsets are only checked for Pr <= 0.71 here; BF16 with
# round-to-nearest freezes both modes.  With LBM_STOCHASTIC_ROUND ("+sr") the
# stored offsets are unbiased and FP16 and BF16 reach the FP32 figures at every
# Pr (measured: nu +0.42 .. +0.48 %, kappa -0.02 .. +0.37 %).
@pytest.mark.parametrize("storage,pr,tol_nu,tol_ka,tol_pr", [
    ("f32", 0.5, 6e-3, 6e-3, 8e-3), ("f32", 0.71, 6e-3, 6e-3, 8e-3), ("f32", 2.0, 6e-3, 6e-3, 8e-3),
    ("f16", 0.5, 1.5e-2, 3e-2, 2e-2), ("f16", 0.71, 1.5e-2, 3e-2, 2e-2),
    ("f16+sr", 0.5, 8e-3, 8e-3, 1e-2), ("f16+sr", 2.0, 8e-3, 8e-3, 1e-2),
    ("bf16+sr", 0.71, 8e-3, 8e-3, 1e-2), ("bf16+sr", 2.0, 8e-3, 8e-3, 1e-2)])
def test_thermal_and_shear_wave_decay_1024(lbm, pr, storage, tol_nu, tol_ka, tol_pr):
    """The thermal configuration: 1024^2 periodic, FP32 collision, FP64 on-device
    fits; temperature and shear waves at mode 10 (~102 nodes per wavelength),
    amplitude 1e-3, Pr in {0.5, 0.71, 2}; FP16 offset storage and FP32 storage."""
    nu_m, nu = _decay(lbm, 1024, pr, "viscous", storage=storage)
    ka_m, ka = _decay(lbm, 1024, pr, "thermal", storage=storage)
    assert nu_m == pytest.approx(nu, rel=tol_nu)
    assert ka_m == pytest.approx(ka, rel=tol_ka)
    assert nu_m / ka_m == pytest.approx(pr, rel=tol_pr)


def test_galilean_invariance_fig3_on_the_gpu(lbm):
    """Fig. 3 on the GPU (FP64 storage, 64 x 4): superposed viscous and thermal
    waves on a base flow u0 perpendicular to k.  CM-MRT kappa is flat in u0, the
    raw-moment MRT's kappa error grows with u0."""
    c = H.lattice()[2]

    def kappa(u0, flags):
        dims = (64, 4)
        rho, u, th = inputs.thermal_wave(dims, amplitude=1e-4, theta0=1.2, mode=1, shear_amplitude=1e-4 / c,
                                         u0=u0 / c)
        sim = _sim(lbm, dims, [0.5 + 0.1 / 1.2, 0.5 + 0.2 / 1.2, 1.0], "f64", True, flags)
        sim.init_fields(rho, u, th)
        k = 2 * np.pi / 64
        steps = int(0.8 / (0.2 * k * k / c ** 2))
        fit, _ = sim.mode_history(3, (1, 0), 21, steps // 20)
        return fit[0] * c ** 2 / (k * k)

    cm = [kappa(u0, 0) for u0 in (0.0, 0.1, 0.2)]
    raw = [kappa(u0, lbm.LBM_RAW_MRT) for u0 in (0.0, 0.1, 0.2)]
    assert abs(cm[2] / cm[0] - 1) < 1e-4
    assert raw[2] / raw[0] - 1 > 10 * abs(cm[2] / cm[0] - 1) and raw[2] / raw[0] - 1 > 5e-3


def test_d2q37_argument_checks(lbm):
    with pytest.raises(lbm.LBMError):
        lbm.Simulation("D2Q37", (2, 8), TAUS)
    with pytest.raises(lbm.LBMError):
        lbm.Simulation("D2Q9", (8, 8), [0.6], flags=lbm.LBM_THERMAL)
    with pytest.raises(lbm.LBMError):
        lbm.Simulation("D2Q37", (8, 8), TAUS, theta_ref=-1.0)
    sim = _sim(lbm, (8, 8), TAUS)
    with pytest.raises(lbm.LBMError):
        sim.mode_amplitude(5, (1, 0))


@pytest.mark.parametrize("storage,dims", [("f16", (36, 11)), ("bf16", (35, 9))])
def test_stochastic_rounding_is_deterministic(lbm, storage, dims):
    """The rounding bits come from a counter-based stream of (step, node,
    population): two runs from the same state agree bit for bit, and differ from
    round-to-nearest."""
    rho, u, theta = _fields(dims, seed=13)
    out = []
    for flags in (lbm.LBM_STOCHASTIC_ROUND, lbm.LBM_STOCHASTIC_ROUND, 0):
        sim = _sim(lbm, dims, TAUS, storage, flags=flags)
        sim.init_fields(rho, u, theta)
        sim.step(5)
        out.append(sim.raw_populations().view(torch.int16).cpu().numpy().copy())
    assert np.array_equal(out[0], out[1])
    assert not np.array_equal(out[0], out[2])


def test_full_size_thermal_1024_fp16_one_step_bound(lbm):
    """The thermal configuration at full size, in the launch the benchmark times:
    1024^2, temperature and shear waves at mode 10, theta0 1.2, Pr 0.71, FP16
    offsets, two-node FP32x2 kernel.  After 7 steps, each of two more steps (both
    parities) from the GPU's own state equals the oracle's step on the whole grid
    within half an ulp of the stored FP16 offset (as on small grids)."""
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    n = bench.THERMAL_N
    t2 = 0.5 + 0.1 / bench.THERMAL_THETA0
    taus = [t2, 0.5 + (t2 - 0.5) / bench.THERMAL_PR, t2]
    rho, u, th = inputs.thermal_wave((n, n), amplitude=1e-3, theta0=bench.THERMAL_THETA0, mode=10,
                                     shear_amplitude=1e-3)
    sim = _sim(lbm, (n, n), taus, "f16", theta_ref=bench.THERMAL_THETA0)
    sim.init_fields(rho, u, th)
    sim.step(7)
    P = _perm()
    inv = np.argsort(P)
    w_lib = gen_d2q37.solve()[1][:, None]
    om = H.omega_from_tau(taus)
    fref = H.equilibrium_node(1.0, np.zeros(2), bench.THERMAL_THETA0)[P][:, None]
    for _ in range(2):
        f = np.ascontiguousarray(sim.populations()[inv])
        H.step((n, n), om, f, 1, True, H.H37_CLOSED)
        sim.step(1)
        g = sim.populations()
        fo = f[P]
        bound = w_lib * 2.0 ** -11 * np.abs((fo - fref) / w_lib) * 1.05 + 2e-7
        assert np.all(np.abs(g - fo) <= bound), np.max(np.abs(g - fo) / bound)
    assert sim.status() == 0
