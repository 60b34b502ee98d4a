"""Slab decomposition of a D3Q27 grid along z (paper_1808_04406_gb300/slab.py)
on CPU: the plane bookkeeping, and whole runs split over 1, 2 and 3 gloo ranks
that equal the single-domain FP64 oracle bit for bit.

The sweeps in these tests are a test-side AA sweeper whose per-node collision
is the oracle's (tests/slab_aa_cpu.py), so that the only thing under test is
the decomposition: which planes each rank sweeps, which nine populations cross
each face, and when they move.  The oracle streams by pulling from a second
array over the whole periodic grid; any missing, extra or misplaced plane copy
changes some node's collision input, which the exact comparison catches."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

import oracle  # noqa: E402
from paper_1808_04406_gb300 import inputs, slab  # noqa: E402

DIMS = (6, 5, 7)
TAUS = [0.56, 0.9, 0.56, 1.0, 0.56]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _fields():
    return inputs.random_smooth(DIMS, seed=31, du=0.05, drho=0.02)


def _oracle(steps):
    rho, u = _fields()
    f = oracle.tp_init(3, rho, u)
    oracle.tp_step(3, DIMS, oracle.omega_from_tau(3, TAUS), f, steps)
    return f


def test_split_covers_the_grid_once():
    for nz, world in [(7, 1), (7, 2), (7, 3), (8, 4), (5, 5)]:
        parts = slab.split(nz, world)
        assert [z0 for z0, _ in parts] == list(np.cumsum([0] + [c for _, c in parts])[:-1])
        assert sum(c for _, c in parts) == nz and max(c for _, c in parts) - min(c for _, c in parts) <= 1
    for nz, world in [(3, 4), (3, 0)]:
        with pytest.raises(ValueError):
            slab.split(nz, world)


def test_up_and_down_populations_are_the_nine_crossing_each_face():
    e = oracle.tp_velocities(3)
    assert slab.UP == tuple(j for j in range(27) if e[j, 2] == 1)
    assert slab.DOWN == tuple(j for j in range(27) if e[j, 2] == -1)


@pytest.mark.parametrize("nzl", [1, 2, 5])
def test_every_send_meets_one_receive_with_the_same_populations(nzl):
    """Before the odd sweep owned boundary planes go to ghost planes; after it
    ghost planes go back to owned boundary planes; the receiving side of each
    message is the opposite one."""
    for phase in ("pre", "post"):
        sends, recvs = slab.messages(nzl, phase)
        assert len(sends) == len(recvs) == 2
        for to, pops, pl in sends:
            match = [r for r in recvs if r[0] != to and r[1] == pops]
            assert len(match) == 1
            ghost = {0, nzl + 1}
            if phase == "pre":
                assert pl not in ghost and match[0][2] in ghost
            else:
                assert pl in ghost and match[0][2] not in ghost


def _make_rank(rank, world):
    from slab_aa_cpu import OracleAASim
    z0, nzl = slab.split(DIMS[2], world)[rank]
    sim = OracleAASim((DIMS[0], DIMS[1], nzl + 2), oracle.omega_from_tau(3, TAUS), 1, nzl, torch)
    return sim


def _init(run):
    rho, u = _fields()
    lr, lu = run.local_fields(rho, u)
    run.sim.init_natural(oracle.tp_init(3, lr, lu))


@pytest.mark.parametrize("steps", [4, 5])
def test_one_slab_with_ghost_planes_equals_the_periodic_oracle(steps):
    """World 1: the slab is its own neighbour (a local copy per plane)."""
    run = slab.SlabRun(_make_rank(0, 1), DIMS, 0, 1)
    _init(run)
    run.step(steps)
    from slab_aa_cpu import natural_from_aa
    P = run.owned(run.sim.raw_populations().numpy(), 27)
    np.testing.assert_array_equal(natural_from_aa(P, DIMS, steps & 1), _oracle(steps))


def _gloo_rank(rank, world, port, steps, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        run = slab.SlabRun(_make_rank(rank, world), DIMS, rank, world, slab.TorchTransport(dist))
        _init(run)
        run.step(steps)
        q.put((rank, run.z0, run.owned(run.sim.raw_populations().numpy(), 27)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,steps", [(2, 5), (3, 4), (3, 5)])
def test_gloo_slabs_equal_the_single_domain_oracle_bit_for_bit(world, steps):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_gloo_rank, args=(r, world, port, steps, q)) for r in range(world)]
    for p in procs:
        p.start()
    parts = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    nx, ny, nz = DIMS
    P = np.empty((27, nz, nx * ny))
    for rank, z0, own in sorted(parts, key=lambda t: t[0]):
        nzl = own.shape[1] // (nx * ny)
        P[:, z0:z0 + nzl] = own.reshape(27, nzl, nx * ny)
    from slab_aa_cpu import natural_from_aa
    np.testing.assert_array_equal(natural_from_aa(P.reshape(27, -1), DIMS, steps & 1), _oracle(steps))
