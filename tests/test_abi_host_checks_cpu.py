"""Host-side size queries and argument checks of the batch calls, the
caller-supplied Hermite-lattice calls and the closure-training calls, on CPU.

Every case here is either a size query (host-only by contract) or fails the
create call's validation, which runs before any CUDA call.  The buffer
addresses passed are fake and are never dereferenced."""
import ctypes

import numpy as np
import pytest

from paper_1808_04406_gb300 import build as libbuild
from paper_1808_04406_gb300 import lbm

FAKE = 1 << 20  # a 256-byte aligned address that validation rejects before use
ESIZE = {lbm.LBM_F64: 8, lbm.LBM_F32: 4, lbm.LBM_F16: 2, lbm.LBM_BF16: 2}


@pytest.fixture(scope="module")
def L():
    libbuild.build()
    return lbm.load()


def _dims(runs):
    return np.ascontiguousarray(np.array([[nx, ny, nz] for nx, ny, nz in runs], dtype=np.int64).reshape(-1))


def _batch_query(L, runs, storage, lattice=lbm.LBM_D2Q9):
    d = _dims(runs)
    pb, wb = ctypes.c_size_t(), ctypes.c_size_t()
    rc = L.lbm_batch_query_bytes(lattice, len(runs), d.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), storage,
                                 ctypes.byref(pb), ctypes.byref(wb))
    return rc, pb.value, wb.value


def _round(v, m):
    return (v + m - 1) // m * m


@pytest.mark.parametrize("storage", [lbm.LBM_F64, lbm.LBM_F32, lbm.LBM_F16, lbm.LBM_BF16])
def test_batch_population_bytes_are_the_runs_slices(L, storage):
    """Each run owns 9 nx ny values rounded up to 64 elements; the buffer is their
    sum in the storage type, rounded to 256 bytes."""
    runs = [(64, 64, 1), (65, 3, 1), (1, 1, 1), (511, 7, 1), (2, 65535, 1)]
    rc, pb, wb = _batch_query(L, runs, storage)
    assert rc == lbm.LBM_OK
    elems = sum(_round(9 * nx * ny, 64) for nx, ny, _ in runs)
    assert pb == _round(elems * ESIZE[storage], 256)
    assert wb % 256 == 0 and wb > 0
    # the workspace grows with the number of runs (status, run table, totals)
    rc2, _, wb2 = _batch_query(L, runs * 4, storage)
    assert rc2 == lbm.LBM_OK and wb2 > wb


@pytest.mark.parametrize("lattice,runs,storage", [
    (lbm.LBM_D3Q27, [(8, 8, 1)], lbm.LBM_BF16),          # batches are D2Q9 only
    (lbm.LBM_D2Q9, [(8, 8, 2)], lbm.LBM_BF16),           # nz must be 1
    (lbm.LBM_D2Q9, [(8, 8, 1), (0, 8, 1)], lbm.LBM_BF16),  # empty run
    (lbm.LBM_D2Q9, [(8, 70000, 1)], lbm.LBM_BF16),        # ny beyond the launch limit
    (lbm.LBM_D2Q9, [(30000, 16000, 1)], lbm.LBM_BF16),    # 9 nx ny >= 2^32
    (lbm.LBM_D2Q9, [(8, 8, 1)], 9),                      # unknown storage
])
def test_batch_query_rejects_bad_runs(L, lattice, runs, storage):
    rc, _, _ = _batch_query(L, runs, storage, lattice)
    assert rc == lbm.LBM_EINVAL
    assert L.lbm_last_error()


def test_batch_query_rejects_no_runs(L):
    pb, wb = ctypes.c_size_t(), ctypes.c_size_t()
    d = _dims([(8, 8, 1)])
    rc = L.lbm_batch_query_bytes(lbm.LBM_D2Q9, 0, d.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), lbm.LBM_BF16,
                                 ctypes.byref(pb), ctypes.byref(wb))
    assert rc == lbm.LBM_EINVAL


def test_batch_create_rejects_bad_arguments_before_any_cuda_call(L):
    runs = [(16, 8, 1), (9, 5, 1)]
    d = _dims(runs)
    dp = d.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    _, pb, wb = _batch_query(L, runs, lbm.LBM_BF16)
    taus = np.ascontiguousarray([0.6, 0.7], dtype=np.float64)
    tp = taus.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    h = ctypes.c_void_p()

    def create(n_tau=1, pop=FAKE, pop_bytes=pb, work=FAKE, work_bytes=wb, out=True):
        return L.lbm_batch_create(lbm.LBM_D2Q9, len(runs), dp, tp, n_tau, lbm.LBM_BF16, pop, pop_bytes, work,
                                  work_bytes, ctypes.byref(h) if out else None)

    assert create(out=False) == lbm.LBM_EINVAL
    assert create(pop_bytes=pb - 1) == lbm.LBM_ESIZE
    assert create(work_bytes=wb - 256) == lbm.LBM_ESIZE
    assert create(pop=FAKE + 16) == lbm.LBM_EINVAL
    assert create(pop=None) == lbm.LBM_EINVAL
    assert create(n_tau=0) == lbm.LBM_EINVAL
    assert h.value is None


def test_batch_create_reports_a_failed_host_allocation_as_eoom(L, monkeypatch):
    """A host allocation that fails while the batch's bookkeeping is built comes
    back as LBM_EOOM, not as a C++ exception through the C boundary.  The failure
    is injected on the host (LBM_FAULT_HOST_ALLOC names the call); it is raised
    after the arguments are validated and before any CUDA call, and the handle
    allocated before it is freed."""
    runs = [(16, 8, 1), (9, 5, 1)]
    d = _dims(runs)
    dp = d.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    _, pb, wb = _batch_query(L, runs, lbm.LBM_BF16)
    taus = np.ascontiguousarray([0.6, 0.7], dtype=np.float64)
    tp = taus.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    h = ctypes.c_void_p()
    monkeypatch.setenv("LBM_FAULT_HOST_ALLOC", "lbm_batch_create")
    for _ in range(3):
        rc = L.lbm_batch_create(lbm.LBM_D2Q9, len(runs), dp, tp, 1, lbm.LBM_BF16, FAKE, pb, FAKE, wb, ctypes.byref(h))
        assert rc == lbm.LBM_EOOM
        assert b"host allocation failed" in L.lbm_last_error()
        assert h.value is None
    # validation still comes first: a bad argument is reported as such
    rc = L.lbm_batch_create(lbm.LBM_D2Q9, len(runs), dp, tp, 0, lbm.LBM_BF16, FAKE, pb, FAKE, wb, ctypes.byref(h))
    assert rc == lbm.LBM_EINVAL


def test_hermite_query_bytes(L):
    for q in (17, 37):
        for storage in (lbm.LBM_F64, lbm.LBM_F32):
            pb, wb = lbm.lbm_hermite_query_bytes(q, (40, 24), storage)
            assert pb == _round(q * 40 * 24 * ESIZE[storage], 256)
            assert wb % 256 == 0 and wb > 0
    for q, dims in [(0, (8, 8)), (38, (8, 8)), (17, (2, 8)), (17, (8, 8, 2))]:
        with pytest.raises(lbm.LBMError) as ei:
            lbm.lbm_hermite_query_bytes(q, dims, lbm.LBM_F64)
        assert ei.value.code == lbm.LBM_EINVAL


@pytest.fixture(scope="module")
def rule17():
    """A 17-velocity degree-7 rule from the oracle's quadrature solver."""
    from oracle import quadrature
    e, w, c = quadrature.rules(7)[0]
    return np.asarray(e), np.asarray(w, dtype=np.float64), float(c)


def test_create_hermite_checks_the_rule_before_any_cuda_call(L, rule17):
    e, w, c = rule17
    dims = (16, 12)
    pb, wb = lbm.lbm_hermite_query_bytes(len(w), dims, lbm.LBM_F64)

    def create(e=e, w=w, c=c, order=3, storage=lbm.LBM_F64, flags=0, theta_ref=1.0, taus=(0.6,), pop_bytes=pb):
        return lbm.lbm_create_hermite(e, w, c, order, dims, list(taus), storage, flags, theta_ref, FAKE, pop_bytes,
                                      FAKE, wb)

    cases = [
        dict(order=4),                     # 17 velocities carry order 3 only
        dict(c=0.0), dict(c=float("inf")),
        dict(storage=lbm.LBM_F16),         # FP64 / FP32 only
        dict(flags=lbm.LBM_K72),           # only LBM_THERMAL applies
        dict(theta_ref=0.0),
    ]
    for kw in cases:
        with pytest.raises(lbm.LBMError) as ei:
            create(**kw)
        assert ei.value.code == lbm.LBM_EINVAL, kw
    # a weight moved by 1e-6 breaks exactness to degree 2N = 6: rejected as such
    w_bad = w.copy()
    w_bad[1] += 1e-6
    with pytest.raises(lbm.LBMError) as ei:
        create(w=w_bad)
    assert ei.value.code == lbm.LBM_EINVAL and "exact" in str(ei.value)
    # a scale off by 1e-6 likewise
    with pytest.raises(lbm.LBMError) as ei:
        create(c=c * (1 + 1e-6))
    assert ei.value.code == lbm.LBM_EINVAL and "exact" in str(ei.value)
    # the exact rule passes every check up to the buffer sizes
    with pytest.raises(lbm.LBMError) as ei:
        create(pop_bytes=pb - 1)
    assert ei.value.code == lbm.LBM_ESIZE


def test_mlp_workspace_size_and_argument_checks(L):
    """lbm_mlp_work_bytes is host arithmetic; the training calls reject bad
    arguments (sizes, alignment, rate range, optimiser settings) before any
    CUDA call."""
    assert lbm.lbm_mlp_work_bytes(0) == 0 and lbm.lbm_mlp_work_bytes(-3) == 0
    sizes = [lbm.lbm_mlp_work_bytes(b) for b in (1, 64, 65, 4096, 65536)]
    assert sizes[0] > lbm.MLP_PARAMS * 4 and all(a <= b for a, b in zip(sizes, sizes[1:]))
    n = 4096
    wb = lbm.lbm_mlp_work_bytes(n)
    cw = [1.0] * 6

    def loss_grad(n=n, work=FAKE, work_bytes=wb, lo=0.0, hi=2.0):
        return lbm.lbm_mlp_loss_grad(FAKE, FAKE, n, cw, FAKE, FAKE, work, work_bytes, omega_lo=lo, omega_hi=hi)

    for kw, code in [(dict(n=0), lbm.LBM_EINVAL), (dict(work_bytes=wb - 1), lbm.LBM_ESIZE),
                     (dict(work=FAKE + 64), lbm.LBM_EINVAL), (dict(work=None), lbm.LBM_EINVAL),
                     (dict(lo=1.5, hi=1.0), lbm.LBM_EINVAL), (dict(hi=2.5), lbm.LBM_EINVAL)]:
        with pytest.raises(lbm.LBMError) as ei:
            loss_grad(**kw)
        assert ei.value.code == code, kw

    def train(iters=10, batch=64, lr=1e-3, t0=0, m=FAKE):
        return lbm.lbm_mlp_train(FAKE, FAKE, n, cw, FAKE, m, FAKE, iters, batch, lr, 0, t0, None, FAKE,
                                 lbm.lbm_mlp_work_bytes(max(batch, 1)))

    for kw in [dict(batch=0), dict(lr=0.0), dict(lr=float("nan")), dict(iters=-1), dict(t0=-1), dict(m=None)]:
        with pytest.raises(lbm.LBMError) as ei:
            train(**kw)
        assert ei.value.code == lbm.LBM_EINVAL, kw


# ---- lbm_reduce_noalloc: every rejection happens before any CUDA call ----------

def _noalloc(L, lattice, dims, storage, ptr, nbytes, step):
    d = (ctypes.c_int64 * 3)(*(list(dims) + [1] * (3 - len(dims))))
    out = (ctypes.c_double * 5)()
    return L.lbm_reduce_noalloc(lattice, d, storage, ctypes.c_void_p(ptr), nbytes, step, None, out)


def test_noalloc_reduce_rejects_bad_arguments_before_any_cuda_call(L):
    dims = (16, 8, 4)
    nbytes = 27 * 16 * 8 * 4 * 4
    cases = [
        (lbm.LBM_D3Q27, dims, lbm.LBM_F32, FAKE, nbytes - 256, 0, lbm.LBM_ESIZE),   # buffer too small
        (lbm.LBM_D3Q27, (4096, 4096, 256), lbm.LBM_F32, FAKE, nbytes, 0, lbm.LBM_EINVAL),  # N >= 2^31
        (lbm.LBM_D3Q27, dims, lbm.LBM_F32, 0, nbytes, 0, lbm.LBM_EINVAL),           # NULL populations
        (lbm.LBM_D3Q27, dims, lbm.LBM_F32, FAKE + 8, nbytes, 0, lbm.LBM_EINVAL),    # not 256-byte aligned
        (lbm.LBM_D3Q27, dims, lbm.LBM_F32, FAKE + 4, nbytes, 0, lbm.LBM_EINVAL),
        (lbm.LBM_D3Q27, dims, lbm.LBM_F32, FAKE, nbytes, -1, lbm.LBM_EINVAL),       # negative step
        (lbm.LBM_D2Q37, (2, 9), lbm.LBM_F16, FAKE, 1 << 20, 0, lbm.LBM_EINVAL),     # 37 velocities need nx >= 3
        (9, dims, lbm.LBM_F32, FAKE, nbytes, 0, lbm.LBM_EINVAL),                    # unknown lattice
        (lbm.LBM_D3Q27, dims, 7, FAKE, nbytes, 0, lbm.LBM_EINVAL),                  # unknown storage
    ]
    for lattice, d, st, ptr, nb, step, want in cases:
        assert _noalloc(L, lattice, d, st, ptr, nb, step) == want, (lattice, d, st, ptr, nb, step)
        assert L.lbm_last_error()


def test_noalloc_reduce_null_output_is_rejected(L):
    d = (ctypes.c_int64 * 3)(16, 8, 4)
    rc = L.lbm_reduce_noalloc(lbm.LBM_D3Q27, d, lbm.LBM_F32, ctypes.c_void_p(FAKE), 1 << 24, 0, None, None)
    assert rc == lbm.LBM_EINVAL


# ---- lbm_alu_probe: shape and pointer checks run before the launch ------------

@pytest.mark.parametrize("kind,iters,blocks,threads", [
    (3, 16, 1, 256), (-1, 16, 1, 256),            # unknown kind
    (lbm.LBM_PROBE_F32, 0, 1, 256),               # no iterations
    (lbm.LBM_PROBE_F32X2, 16, 0, 256),            # no blocks
    (lbm.LBM_PROBE_F64, 16, 1, 100),              # not a multiple of a warp
    (lbm.LBM_PROBE_F64, 16, 1, 2048),             # above the block limit
])
def test_alu_probe_rejects_bad_shapes(L, kind, iters, blocks, threads):
    flops = ctypes.c_double()
    assert L.lbm_alu_probe(kind, iters, blocks, threads, ctypes.c_void_p(FAKE), None,
                           ctypes.byref(flops)) == lbm.LBM_EINVAL
    assert L.lbm_last_error()


def test_alu_probe_rejects_null_pointers(L):
    flops = ctypes.c_double()
    assert L.lbm_alu_probe(0, 16, 1, 256, None, None, ctypes.byref(flops)) == lbm.LBM_EINVAL
    assert L.lbm_alu_probe(0, 16, 1, 256, ctypes.c_void_p(FAKE), None, None) == lbm.LBM_EINVAL


def test_selftest_wait_timeout_rejects_a_null_handle(L):
    assert L.lbm_selftest_wait_timeout(None, 10) == lbm.LBM_EINVAL
    assert L.lbm_last_error()


def test_sweep_kernel_name_of_a_null_handle_is_null(L):
    assert L.lbm_sweep_kernel(None) is None


def test_bulk_batch_init_rejects_a_null_handle(L):
    assert L.lbm_batch_init_runs(None, None, None, lbm.LBM_DTYPE_F64, 0) == lbm.LBM_EINVAL
    assert L.lbm_last_error()
