"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every symbol include/lbm.h declares, sizes its buffers, and rejects bad
arguments before touching the device."""
import os
import re

import pytest

from paper_1808_04406_gb300 import build as libbuild
from paper_1808_04406_gb300 import lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    libbuild.build()
    return lbm.load()


def _declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", text))
    return names


def test_library_exports_every_declared_symbol(L):
    declared = _declared_symbols()
    assert "lbm_step" in declared and "lbm_create" in declared
    for name in declared:
        assert hasattr(L, name), name
    assert declared == set(lbm.EXPORTS)


def test_every_export_has_its_prototype_after_load(L):
    """ctypes passes arguments of an undeclared function as C ints, which would
    garble 64-bit sizes and pointers: load() declares every entry point."""
    assert [n for n in lbm.EXPORTS if getattr(L, n).argtypes is None] == []


def test_binding_constants_match_the_header():
    """Every LBM_* integer constant the header defines has the same value in the
    Python binding (lattices, storage types, flags, dtypes, status codes)."""
    text = open(os.path.join(ROOT, "include", "lbm.h")).read()
    defs = dict(re.findall(r"#define\s+(LBM_[A-Z0-9_]+)\s+\(?(-?(?:0x[0-9a-fA-F]+|\d+))u?\)?", text))
    assert "LBM_OK" in defs and "LBM_EOOM" in defs
    for name, val in defs.items():
        assert hasattr(lbm, name), name
        assert getattr(lbm, name) == int(val, 0), (name, val)


def test_query_bytes_sizes(L):
    pb, wb = lbm.lbm_query_bytes(lbm.LBM_D3Q27, (256, 256, 256), lbm.LBM_F32)
    assert pb == 27 * 256 ** 3 * 4
    assert wb >= 32 << 20


def test_query_bytes_rounds_to_256(L):
    pb, wb = lbm.lbm_query_bytes(lbm.LBM_D2Q9, (5, 7), lbm.LBM_BF16)
    assert pb % 256 == 0 and pb >= 9 * 35 * 2
    assert wb % 256 == 0


@pytest.mark.parametrize("lattice,dims,storage", [
    (7, (4, 4, 1), lbm.LBM_F32),          # unknown lattice
    (lbm.LBM_D2Q9, (4, 4, 2), lbm.LBM_F32),  # 2D with nz != 1
    (lbm.LBM_D3Q27, (0, 4, 4), lbm.LBM_F32),  # empty grid
    (lbm.LBM_D3Q27, (4, 70000, 4), lbm.LBM_F32),  # ny beyond the launch limit
    (lbm.LBM_D3Q27, (4096, 4096, 256), lbm.LBM_F32),  # N >= 2^31
    (lbm.LBM_D3Q27, (4, 4, 4), 9),  # unknown storage
])
def test_query_bytes_rejects_bad_shapes(L, lattice, dims, storage):
    with pytest.raises(lbm.LBMError) as ei:
        lbm.lbm_query_bytes(lattice, dims, storage)
    assert ei.value.code == lbm.LBM_EINVAL


def test_create_rejects_bad_arguments_before_any_cuda_call(L):
    dims = (8, 8, 8)
    pb, wb = lbm.lbm_query_bytes(lbm.LBM_D3Q27, dims, lbm.LBM_F32)
    fake = 1 << 20  # never dereferenced: every case fails validation first
    with pytest.raises(lbm.LBMError) as ei:
        lbm.lbm_create(lbm.LBM_D3Q27, dims, [0.5], lbm.LBM_F32, fake, pb, fake, wb)
    assert ei.value.code == lbm.LBM_EINVAL and "tau" in str(ei.value)
    with pytest.raises(lbm.LBMError) as ei:
        lbm.lbm_create(lbm.LBM_D3Q27, dims, [0.6, float("nan")], lbm.LBM_F32, fake, pb, fake, wb)
    assert ei.value.code == lbm.LBM_EINVAL
    with pytest.raises(lbm.LBMError) as ei:
        lbm.lbm_create(lbm.LBM_D3Q27, dims, [0.6], lbm.LBM_F32, fake, pb - 1, fake, wb)
    assert ei.value.code == lbm.LBM_ESIZE
    with pytest.raises(lbm.LBMError) as ei:
        lbm.lbm_create(lbm.LBM_D3Q27, dims, [0.6], lbm.LBM_F32, fake + 8, pb, fake, wb)
    assert ei.value.code == lbm.LBM_EINVAL and "aligned" in str(ei.value)
    with pytest.raises(lbm.LBMError) as ei:
        lbm.lbm_create(lbm.LBM_D3Q27, dims, [0.6], lbm.LBM_F32, 0, pb, fake, wb)
    assert ei.value.code == lbm.LBM_EINVAL


def test_null_handle_is_rejected(L):
    assert L.lbm_step(None, 1) == lbm.LBM_EINVAL
    assert L.lbm_step_count(None) == -1
    assert "NULL handle" in lbm.lbm_last_error()


def test_last_error_is_per_thread(L):
    """lbm_last_error holds the message of the calling thread's last failure: two
    threads failing in different ways, interleaved, each read back their own."""
    import threading
    out = {}
    barrier = threading.Barrier(2)

    def fail(key, lattice, dims):
        msgs = []
        for _ in range(200):
            barrier.wait()
            with pytest.raises(lbm.LBMError) as ei:
                lbm.lbm_query_bytes(lattice, dims, lbm.LBM_F32)
            msgs.append(str(ei.value))
        out[key] = msgs

    t1 = threading.Thread(target=fail, args=("lattice", 7, (4, 4, 1)))
    t2 = threading.Thread(target=fail, args=("empty", lbm.LBM_D3Q27, (0, 4, 4)))
    for t in (t1, t2):
        t.start()
    for t in (t1, t2):
        t.join()
    assert len(set(out["lattice"])) == 1 and len(set(out["empty"])) == 1
    assert out["lattice"][0] != out["empty"][0]
