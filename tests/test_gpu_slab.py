"""Slab decomposition on the GPU: the library's sweeps restricted to a slab's
planes (lbm_set_active_planes) plus the plane exchange of
paper_1808_04406_gb300/slab.py reproduce the single-domain run bit for bit.

All slabs of a grid run in one process on the one GPU (slab.LocalGroup: one
device copy per population and plane, on the sweeps' stream); the same
exchange schedule runs between processes over gloo in tests/test_slab_cpu.py.
A slab's nodes take the same kernels, pairing and arithmetic as in the whole
grid, so every population must be identical."""
import numpy as np
import pytest

from paper_1808_04406_gb300 import inputs, slab

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


TAUS = [0.53, 1.0, 0.53, 1.0, 0.53]


def _whole(lbm, dims, storage, rho, u, steps):
    sim = lbm.Simulation("D3Q27", dims, TAUS, storage=storage)
    sim.init_fields(rho, u)
    sim.step(steps)
    return sim


@pytest.mark.parametrize("dims,storage", [((40, 12, 13), "f32"), ((40, 12, 13), "bf16"), ((21, 10, 11), "f32"),
                                          ((22, 6, 9), "f64")])
@pytest.mark.parametrize("world", [1, 2, 3])
@pytest.mark.parametrize("steps", [6, 7])
def test_slabs_equal_the_single_domain_run_bit_for_bit(lbm, dims, storage, world, steps):
    rho, u = inputs.random_smooth(dims, seed=41, du=0.05, drho=0.02)
    ref = _whole(lbm, dims, storage, rho, u, steps)
    f_ref = ref.populations().reshape(27, dims[2], -1)
    t_ref = ref.reduce()
    runs = [slab.SlabRun.create(dims, TAUS, storage, r, world) for r in range(world)]
    for run in runs:
        run.sim.init_fields(*run.local_fields(rho, u))
    group = slab.LocalGroup(runs)
    group.step(steps)
    group.refresh_ghosts()  # odd parity: boundary nodes read populations from the ghost planes
    totals = np.zeros(5)
    for run in runs:
        assert run.sim.status() == lbm.LBM_OK
        own = run.owned(run.sim.populations(), 27).reshape(27, run.nzl, -1)
        np.testing.assert_array_equal(own, f_ref[:, run.z0:run.z0 + run.nzl])
        totals += run.sim.reduce()  # the slab's own planes only
    np.testing.assert_allclose(totals, t_ref, rtol=1e-12, atol=1e-9)


def test_one_rank_slab_run_exchanges_with_itself(lbm):
    dims = (32, 8, 10)
    rho, u = inputs.random_smooth(dims, seed=43, du=0.05)
    ref = _whole(lbm, dims, "f32", rho, u, 9)
    run = slab.SlabRun.create(dims, TAUS, "f32", 0, 1)
    run.sim.init_fields(*run.local_fields(rho, u))
    run.step(9)
    run.refresh_ghosts()
    np.testing.assert_array_equal(run.owned(run.sim.populations(), 27), ref.populations())


def test_active_planes_reject_bad_ranges_and_other_lattices(lbm):
    sim = lbm.Simulation("D3Q27", (8, 4, 6), TAUS, storage="f32")
    for z_lo, cnt in [(-1, 2), (0, 0), (5, 2), (0, 7)]:
        with pytest.raises(lbm.LBMError) as ei:
            sim.set_active_planes(z_lo, cnt)
        assert ei.value.code == lbm.LBM_EINVAL
    sim.set_active_planes(1, 4)
    sim.set_active_planes(0, 6)  # the whole grid again
    d2 = lbm.Simulation("D2Q9", (8, 4), [0.6], storage="f32")
    with pytest.raises(lbm.LBMError) as ei:
        d2.set_active_planes(0, 1)
    assert ei.value.code == lbm.LBM_EINVAL
