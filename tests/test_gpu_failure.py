"""Failure detection on the GPU without a fault: the bounded device wait of the
tensor-core sweeps runs out on purpose (an mbarrier nothing arrives at, nothing
asynchronous in flight), the kernel returns, the library reports LBM_ETIMEOUT,
and the context stays usable."""
import numpy as np
import pytest

import oracle
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
    oracle.lib()
    return L


@pytest.mark.parametrize("polls", [1, 1000])
def test_bounded_wait_gives_up_and_reports_timeout(lbm, polls):
    dims = (16, 8, 6)
    taus = [0.6, 0.9, 0.6, 1.0, 0.6]
    rho, u = inputs.random_smooth(dims, seed=2, du=0.04)
    sim = lbm.Simulation("D3Q27", dims, taus, storage="f32")
    sim.init_fields(rho, u)
    sim.step(2)
    assert sim.status() == lbm.LBM_OK
    lbm.lbm_selftest_wait_timeout(sim.handle, polls)
    assert sim.status() == lbm.LBM_ETIMEOUT
    assert b"gave up" in lbm.load().lbm_last_error()
    with pytest.raises(lbm.LBMError) as ei:
        sim.moments()
    assert ei.value.code == lbm.LBM_ETIMEOUT
    # the context still works: re-initialising clears the flag, and the steps
    # that follow match the oracle
    sim.init_fields(rho, u)
    assert sim.status() == lbm.LBM_OK
    sim.step(3)
    assert sim.status() == lbm.LBM_OK
    f = oracle.tp_init(3, rho, u)
    oracle.tp_step(3, dims, oracle.omega_from_tau(3, taus), f, 3)
    assert np.abs(sim.populations() - f).max() <= 2e-7


def test_selftest_rejects_bad_arguments(lbm):
    sim = lbm.Simulation("D2Q9", (8, 8), [0.6], storage="f32")
    for polls in (0, -1, (1 << 20) + 1):
        with pytest.raises(lbm.LBMError) as ei:
            lbm.lbm_selftest_wait_timeout(sim.handle, polls)
        assert ei.value.code == lbm.LBM_EINVAL
    assert lbm.load().lbm_selftest_wait_timeout(None, 10) == lbm.LBM_EINVAL
