"""Linear-mode measurements on the GPU (Sec. III.A): the on-device FP64 decay
fit and the Chapman-Enskog viscosity with a translating base flow.

The shear-wave sweep is the 64^3 part of the D3Q27 FP32 configuration: a
viscous mode u_y = u0 + A sin(2 pi x / 64) with base flow u0 in 0..0.1 along y
(perpendicular to k, as in the paper's Galilean test) and tau_2 in
{0.55, 0.6, 0.8}.  Eq. dr: the viscous mode decays at exactly nu k^2, with
nu = c_s^2 (tau_2 - 1/2) (Eq. sigma with tau -> tau_2).
"""
import numpy as np
import pytest

import oracle
from oracle import analysis
from paper_1808_04406_gb300 import inputs

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


def _shear_sim(lbm, dims, tau2, u0, storage="f32", amplitude=1e-3):
    rho, u = inputs.shear_wave(dims, amplitude=amplitude, u0=u0, mode=1, k_axis=0, u_axis=1)
    taus = [tau2, 1.0, tau2, 1.0, tau2][: 2 * len(dims) - 1]
    sim = lbm.Simulation("D3Q27" if len(dims) == 3 else "D2Q9", dims, taus, storage=storage)
    sim.init_fields(rho, u)
    return sim, taus


def test_device_fit_matches_host_fit_of_the_same_records(lbm):
    dims = (48, 6, 4)
    sim, _ = _shear_sim(lbm, dims, 0.6, 0.05)
    fit, amps = sim.mode_history(2, (1, 0, 0), 40, 25)
    t = np.arange(40) * 25.0
    assert fit[0] == pytest.approx(analysis.fit_decay_rate(t, amps), rel=1e-10)
    ph = np.unwrap(np.angle(amps))
    slope = np.polyfit(t, ph, 1)[0]
    assert fit[1] == pytest.approx(slope, abs=1e-12)
    # the fitted intercept sits within the start-up transient of the first record
    assert np.exp(fit[2]) == pytest.approx(abs(amps[0]), rel=1e-2)
    assert sim.step_count == 39 * 25


def test_mode_history_matches_the_oracle_history(lbm):
    """The recorded amplitudes follow the oracle's (FP64) run of the same wave."""
    dims = (32, 4, 2)
    tau2 = 0.7
    sim, taus = _shear_sim(lbm, dims, tau2, 0.03, storage="f64")
    _, amps = sim.mode_history(2, (1, 0, 0), 6, 20)
    rho, u = inputs.shear_wave(dims, amplitude=1e-3, u0=0.03, mode=1, k_axis=0, u_axis=1)
    f = oracle.tp_init(3, rho, u)
    om = oracle.omega_from_tau(3, taus)
    ref = []
    for r in range(6):
        if r:
            oracle.tp_step(3, dims, om, f, 20)
        _, uu = oracle.tp_moments(3, f)
        ref.append(analysis.mode_amplitude(uu[1], dims, (1, 0, 0)))
    np.testing.assert_allclose(amps, np.array(ref), rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("tau2", [0.55, 0.6, 0.8])
def test_shear_wave_sweep_galilean_invariant_viscosity_64cubed(lbm, tau2):
    """D3Q27 FP32 64^3: nu from the device fit equals c_s^2 (tau_2 - 1/2) within
    0.3 % (the O(k^2) lattice correction at 64 nodes per wavelength, as in the
    oracle's pin), and its spread over u0 = 0 .. 0.1 is below 0.1 %."""
    dims = (64, 64, 64)
    k = 2 * np.pi / 64
    nu = (tau2 - 0.5) / 3.0
    steps = int(0.7 / (nu * k * k))
    n_rec = 50
    stride = max(1, steps // (n_rec - 1))
    nus = []
    for u0 in (0.0, 0.02, 0.04, 0.06, 0.08, 0.1):
        sim, _ = _shear_sim(lbm, dims, tau2, u0)
        fit, _ = sim.mode_history(2, (1, 0, 0), n_rec, stride)
        nus.append(fit[0] / (k * k))
        sim.close()
    nus = np.array(nus)
    assert np.all(np.abs(nus / nu - 1) < 3e-3), nus / nu - 1
    assert (nus.max() - nus.min()) / nu < 1e-3


def test_mode_history_rejects_bad_arguments(lbm):
    sim, _ = _shear_sim(lbm, (8, 4, 2), 0.6, 0.0)
    for args in [(2, (1, 0, 0), 1, 5), (2, (1, 0, 0), 5000, 5), (2, (1, 0, 0), 10, 0), (7, (1, 0, 0), 10, 1)]:
        with pytest.raises(lbm.LBMError) as ei:
            sim.mode_history(*args)
        assert ei.value.code == lbm.LBM_EINVAL
