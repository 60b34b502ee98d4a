"""lbm_reduce_noalloc: grid totals for callers that cannot allocate device memory.

Such callers (a plugin whose host application's memory manager owns the whole
device, or a time-critical loop that cannot pay for cudaMalloc's implicit
synchronisation) hold a population buffer but no workspace.  The entry point
uses a fixed scratch array inside the library instead.  This file is collected
last on purpose; it creates its own simulation, so it also passes alone.
"""
import numpy as np
import pytest

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


@pytest.mark.parametrize("lattice,dims,storage", [
    ("D3Q27", (37, 21, 11), "f32"),
    ("D2Q9", (300, 45), "f64"),
])
def test_noalloc_reduce_matches_workspace_reduce_on_two_calls(lbm, lattice, dims, storage):
    taus = [0.57, 0.9, 1.2, 0.8, 1.1]
    rho, u = inputs.random_smooth(dims, seed=21, du=0.05, drho=0.02)
    sim = lbm.Simulation(lattice, dims, taus, storage=storage)
    sim.init_fields(rho, u)
    sim.step(3)
    stream = sim.stream.cuda_stream
    first = None
    for call in range(2):  # two calls in a row, then one at the other AA parity
        ref = sim.reduce()
        got = lbm.lbm_reduce_noalloc(sim.lattice, dims, sim.storage, sim.pop.data_ptr(), sim.pop.numel(),
                                     sim.step_count, stream)
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)
        if first is None:
            first = got
        else:
            np.testing.assert_array_equal(got, first)  # the shared array holds no stale state
    sim.step(1)
    ref = sim.reduce()
    got = lbm.lbm_reduce_noalloc(sim.lattice, dims, sim.storage, sim.pop.data_ptr(), sim.pop.numel(),
                                 sim.step_count, stream)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_noalloc_reduce_rejects_sizes_beyond_its_limits(lbm):
    dims = (16, 8, 4)
    sim = lbm.Simulation("D3Q27", dims, [0.6], storage="f32")
    rho, u = inputs.random_noise(dims, seed=1)
    sim.init_fields(rho, u)
    ptr, nbytes = sim.pop.data_ptr(), sim.pop.numel()
    with pytest.raises(lbm.LBMError) as ei:
        lbm.lbm_reduce_noalloc(sim.lattice, dims, sim.storage, ptr, nbytes - 256, 0)
    assert ei.value.code == lbm.LBM_ESIZE
    with pytest.raises(lbm.LBMError) as ei:
        lbm.lbm_reduce_noalloc(sim.lattice, (4096, 4096, 256), sim.storage, ptr, nbytes, 0)
    assert ei.value.code == lbm.LBM_EINVAL
    with pytest.raises(lbm.LBMError) as ei:
        lbm.lbm_reduce_noalloc(sim.lattice, dims, sim.storage, 0, nbytes, 0)
    assert ei.value.code == lbm.LBM_EINVAL
