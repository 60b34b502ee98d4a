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
    _check_both_parities(lbm, sim, dims)


def test_noalloc_reduce_on_the_thermal_37_velocity_lattice_in_fp16(lbm):
    """The 37-velocity lattice goes through its own reduction; FP16 offsets taken
    from the equilibrium at theta_ref = 1.2, thermal model.  The entry point has
    no theta_ref argument: the totals (mass, momentum, kinetic energy) do not
    depend on the offsets' base temperature."""
    dims = (40, 18)
    rho, u = inputs.random_smooth(dims, seed=23, du=0.03, drho=0.01)
    theta = 1.2 + 0.02 * np.cos(2 * np.pi * np.arange(int(np.prod(dims))) / 13.0)
    sim = lbm.Simulation("D2Q37", dims, [0.58, 0.66, 0.58], storage="f16", flags=lbm.LBM_THERMAL, theta_ref=1.2)
    sim.init_fields(rho, u, theta)
    sim.step(2)
    _check_both_parities(lbm, sim, dims)


def _check_both_parities(lbm, sim, dims):
    """Two calls in a row at one AA parity, then one at the other: each equals
    lbm_reduce on the same state bit for bit (same kernels, grid and summation
    order), so the shared array carries nothing from one call to the next."""
    stream = sim.stream.cuda_stream
    for parity in range(2):
        ref = sim.reduce()
        for call in range(2):
            got = lbm.lbm_reduce_noalloc(sim.lattice, dims, sim.storage, sim.pop.data_ptr(), sim.pop.numel(),
                                         sim.step_count, stream)
            np.testing.assert_array_equal(got, ref)
        sim.step(1)
