"""Thin Python binding of the C ABI in ``include/lbm.h`` (ctypes).

The functions ``lbm_*`` below marshal arguments to the library calls of the same
names; every step of the computation runs in the library's CUDA kernels.
PyTorch only provides the device memory (population buffer and workspace) and
the stream.  If ``liblbm.so`` has not been built this module raises on first
use: there is no CPU fallback.

``Simulation`` bundles a handle with its torch-allocated buffers.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbm.so")

LBM_D2Q9, LBM_D3Q27, LBM_D2Q37, LBM_HERMITE = 1, 2, 3, 4
LBM_THERMAL, LBM_K72, LBM_RAW_MRT, LBM_STOCHASTIC_ROUND, LBM_FAST_TRANSFORMS = 1, 2, 4, 8, 16
LBM_F64, LBM_F32, LBM_F16, LBM_BF16 = 0, 1, 2, 3
LBM_DTYPE_F64, LBM_DTYPE_F32 = 0, 1
LBM_OK, LBM_EINVAL, LBM_ECUDA, LBM_EDIVERGED, LBM_ESIZE, LBM_ETIMEOUT, LBM_EOOM = 0, -1, -2, -3, -4, -5, -6

LATTICES = {"D2Q9": LBM_D2Q9, "D3Q27": LBM_D3Q27, "D2Q37": LBM_D2Q37}
STORAGES = {"f64": LBM_F64, "f32": LBM_F32, "f16": LBM_F16, "bf16": LBM_BF16}
LATTICE_D = {LBM_D2Q9: 2, LBM_D3Q27: 3, LBM_D2Q37: 2}
LATTICE_Q = {LBM_D2Q9: 9, LBM_D3Q27: 27, LBM_D2Q37: 37}

# every symbol declared in include/lbm.h
EXPORTS = (
    "lbm_query_bytes", "lbm_create", "lbm_create_ex", "lbm_destroy", "lbm_set_stream", "lbm_set_tau",
    "lbm_init_fields", "lbm_step", "lbm_moments", "lbm_get_populations", "lbm_set_populations",
    "lbm_reduce", "lbm_step_totals", "lbm_step_totals_async", "lbm_mode_amplitude", "lbm_step_count", "lbm_status", "lbm_last_error",
    "lbm_reduce_noalloc", "lbm_mode_history", "lbm_alu_probe", "lbm_selftest_wait_timeout",
    "lbm_set_active_planes", "lbm_sweep_kernel",
)


class LBMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("lbm error %d: %s" % (code, msg))
        self.code = code


_lib = None
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_szp = ctypes.POINTER(ctypes.c_size_t)
_i64p = ctypes.POINTER(ctypes.c_int64)
_dp = ctypes.POINTER(ctypes.c_double)


def load():
    """Load liblbm.so (built by ``__graft_entry__.build()``); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("CUDA library %s is missing: run __graft_entry__.build() first" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        L.lbm_query_bytes.argtypes = [ctypes.c_int, _i64p, ctypes.c_int, _szp, _szp]
        L.lbm_create.argtypes = [ctypes.c_int, _i64p, _dp, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_size_t,
                                 _vp, ctypes.c_size_t, ctypes.POINTER(_vp)]
        L.lbm_create_ex.argtypes = [ctypes.c_int, _i64p, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_uint,
                                    ctypes.c_double, _vp, ctypes.c_size_t, _vp, ctypes.c_size_t,
                                    ctypes.POINTER(_vp)]
        L.lbm_destroy.argtypes = [_vp]
        L.lbm_destroy.restype = None
        L.lbm_set_stream.argtypes = [_vp, _vp]
        L.lbm_set_tau.argtypes = [_vp, _dp, ctypes.c_int]
        L.lbm_init_fields.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_int, ctypes.c_int]
        L.lbm_step.argtypes = [_vp, _i64]
        L.lbm_moments.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_int, ctypes.c_int]
        L.lbm_get_populations.argtypes = [_vp, _vp, ctypes.c_int]
        L.lbm_set_populations.argtypes = [_vp, _vp, ctypes.c_int]
        L.lbm_reduce.argtypes = [_vp, _dp]
        L.lbm_step_totals.argtypes = [_vp, _dp]
        L.lbm_step_totals_async.argtypes = [_vp, _vp]
        L.lbm_mode_amplitude.argtypes = [_vp, ctypes.c_int, _i64p, _dp]
        L.lbm_step_count.argtypes = [_vp]
        L.lbm_step_count.restype = ctypes.c_int64
        L.lbm_status.argtypes = [_vp]
        L.lbm_reduce_noalloc.argtypes = [ctypes.c_int, _i64p, ctypes.c_int, _vp, ctypes.c_size_t, _i64,
                                         _vp, _dp]
        L.lbm_mode_history.argtypes = [_vp, ctypes.c_int, _i64p, ctypes.c_int, _i64, _dp, _dp]
        L.lbm_selftest_wait_timeout.argtypes = [_vp, ctypes.c_int]
        L.lbm_set_active_planes.argtypes = [_vp, _i64, _i64]
        L.lbm_sweep_kernel.argtypes = [_vp]
        L.lbm_sweep_kernel.restype = ctypes.c_char_p
        L.lbm_alu_probe.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp, _dp]
        L.lbm_last_error.argtypes = []
        L.lbm_last_error.restype = ctypes.c_char_p
        _lib = L
        # the other groups' prototypes too, so that every entry point of the
        # object returned here is safe to call directly (ctypes would otherwise
        # pass undeclared 64-bit arguments as C ints)
        _batch_lib()
        _closure_lib()
        _hermite_lib()
    return _lib


def _check(rc):
    if rc != LBM_OK:
        raise LBMError(rc, load().lbm_last_error().decode())
    return rc


def _dims3(dims):
    d = list(int(x) for x in dims) + [1] * (3 - len(dims))
    return (ctypes.c_int64 * 3)(*d)


def _taus(tau_per_order):
    t = [float(x) for x in tau_per_order]
    return (ctypes.c_double * max(1, len(t)))(*t), len(t)


# ---- raw C-ABI wrappers (same names as the C functions) ----------------------

def lbm_query_bytes(lattice, dims, storage):
    pb, wb = ctypes.c_size_t(), ctypes.c_size_t()
    _check(load().lbm_query_bytes(lattice, _dims3(dims), storage, ctypes.byref(pb), ctypes.byref(wb)))
    return pb.value, wb.value


def lbm_create(lattice, dims, tau_per_order, storage, pop_ptr, pop_bytes, work_ptr, work_bytes):
    h = _vp()
    arr, n = _taus(tau_per_order)
    _check(load().lbm_create(lattice, _dims3(dims), arr, n, storage, _vp(pop_ptr), pop_bytes,
                             _vp(work_ptr), work_bytes, ctypes.byref(h)))
    return h


def lbm_create_ex(lattice, dims, tau_per_order, storage, flags, theta_ref, pop_ptr, pop_bytes, work_ptr,
                  work_bytes):
    h = _vp()
    arr, n = _taus(tau_per_order)
    _check(load().lbm_create_ex(lattice, _dims3(dims), arr, n, storage, int(flags), float(theta_ref),
                                _vp(pop_ptr), pop_bytes, _vp(work_ptr), work_bytes, ctypes.byref(h)))
    return h


def lbm_destroy(h):
    load().lbm_destroy(h)


def lbm_set_stream(h, stream_ptr):
    _check(load().lbm_set_stream(h, _vp(stream_ptr)))


def lbm_set_tau(h, tau_per_order):
    arr, n = _taus(tau_per_order)
    _check(load().lbm_set_tau(h, arr, n))


def lbm_init_fields(h, rho_ptr, u_ptr, theta_ptr, dtype, on_device):
    _check(load().lbm_init_fields(h, _vp(rho_ptr), _vp(u_ptr), _vp(theta_ptr), dtype, int(on_device)))


def lbm_step(h, n):
    _check(load().lbm_step(h, int(n)))


def lbm_moments(h, rho_ptr, u_ptr, theta_ptr, dtype, on_device):
    return _check(load().lbm_moments(h, _vp(rho_ptr), _vp(u_ptr), _vp(theta_ptr), dtype, int(on_device)))


def lbm_get_populations(h, f_ptr, on_device):
    _check(load().lbm_get_populations(h, _vp(f_ptr), int(on_device)))


def lbm_set_populations(h, f_ptr, on_device):
    _check(load().lbm_set_populations(h, _vp(f_ptr), int(on_device)))


def lbm_step_totals_async(h, out_ptr):
    """One step; its totals land in host memory out_ptr[0..5) (doubles, ideally
    pinned) once the handle's stream has passed it.  Returns without waiting."""
    _check(load().lbm_step_totals_async(h, _vp(out_ptr)))


def lbm_reduce(h):
    out = (ctypes.c_double * 5)()
    _check(load().lbm_reduce(h, out))
    return np.array(out[:])


def lbm_reduce_noalloc(lattice, dims, storage, pop_ptr, pop_bytes, step, stream_ptr=None):
    """Grid totals of a population buffer without a handle or any allocation
    (for callers that cannot call cudaMalloc); same out[5] as lbm_reduce."""
    out = (ctypes.c_double * 5)()
    _check(load().lbm_reduce_noalloc(lattice, _dims3(dims), storage, _vp(pop_ptr), pop_bytes, int(step),
                                     _vp(stream_ptr), out))
    return np.array(out[:])


LBM_PROBE_F32, LBM_PROBE_F32X2, LBM_PROBE_F64 = 0, 1, 2


def lbm_set_active_planes(h, z_lo, z_count):
    """Restrict the sweeps and totals of a D3Q27 handle to planes z_lo .. z_lo + z_count - 1."""
    _check(load().lbm_set_active_planes(h, int(z_lo), int(z_count)))


def lbm_sweep_kernel(h):
    """Name of the sweep kernel lbm_step launches for this handle."""
    name = load().lbm_sweep_kernel(h)
    if name is None:
        raise LBMError(LBM_EINVAL, "NULL handle")
    return name.decode()


def lbm_selftest_wait_timeout(h, polls):
    """Enqueue the bounded-wait self-test (a wait that runs out on purpose)."""
    _check(load().lbm_selftest_wait_timeout(h, int(polls)))


def lbm_alu_probe(kind, iters, blocks, threads, sink_ptr, stream_ptr=None):
    """Enqueue one FMA-throughput probe kernel; returns the FLOPs it performs
    (the caller times it on the stream)."""
    flops = ctypes.c_double()
    _check(load().lbm_alu_probe(int(kind), int(iters), int(blocks), int(threads), _vp(sink_ptr), _vp(stream_ptr),
                                ctypes.byref(flops)))
    return flops.value


def lbm_mode_amplitude(h, field, mode):
    out = (ctypes.c_double * 2)()
    _check(load().lbm_mode_amplitude(h, int(field), _dims3(list(mode)), out))
    return complex(out[0], out[1])


def lbm_mode_history(h, field, mode, n_records, stride, want_amplitudes=True):
    """Record n_records amplitudes every `stride` steps and fit them on the device:
    returns (fit[4], amplitudes[n_records] complex or None)."""
    fit = (ctypes.c_double * 4)()
    amps = (ctypes.c_double * (2 * n_records))() if want_amplitudes else None
    _check(load().lbm_mode_history(h, int(field), _dims3(list(mode)), int(n_records), int(stride),
                                   amps, fit))
    a = None
    if amps is not None:
        arr = np.array(amps[:])
        a = arr[0::2] + 1j * arr[1::2]
    return np.array(fit[:]), a


def lbm_step_count(h):
    return int(load().lbm_step_count(h))


def lbm_status(h):
    return int(load().lbm_status(h))


def lbm_last_error():
    return load().lbm_last_error().decode()


# ---- convenience object -------------------------------------------------------

def _np_ptr(a):
    return a.ctypes.data


class Simulation:
    """A periodic CM-MRT simulation on one GPU with torch-owned buffers.

    lattice: "D2Q9" | "D3Q27" | "D2Q37"; dims: (nx, ny) or (nx, ny, nz);
    tau_per_order: [tau_2, tau_3, ...] (later orders default to 1);
    storage: "f64" | "f32" | "f16" | "bf16"; flags (D2Q37): LBM_THERMAL |
    LBM_K72 | LBM_RAW_MRT | LBM_STOCHASTIC_ROUND; theta_ref (D2Q37): offset base
    temperature.
    Velocities are in lattice units.
    """

    def __init__(self, lattice, dims, tau_per_order, storage="f32", device=None, stream=None, flags=0,
                 theta_ref=1.0):
        import torch
        self.torch = torch
        self.lattice = LATTICES[lattice] if isinstance(lattice, str) else int(lattice)
        self.storage = STORAGES[storage] if isinstance(storage, str) else int(storage)
        self.D = LATTICE_D[self.lattice]
        self.Q = LATTICE_Q[self.lattice]
        self.flags = int(flags)
        self.dims = tuple(int(x) for x in dims)
        if len(self.dims) != self.D:
            raise ValueError("dims must have %d entries" % self.D)
        self.N = int(np.prod(self.dims))
        self.device = torch.device(device if device is not None else "cuda")
        if self.device.type != "cuda":
            raise RuntimeError("Simulation runs on a CUDA device only")
        pb, wb = lbm_query_bytes(self.lattice, self.dims, self.storage)
        self.pop = torch.empty(pb, dtype=torch.uint8, device=self.device)
        self.work = torch.empty(wb, dtype=torch.uint8, device=self.device)
        self.handle = lbm_create_ex(self.lattice, self.dims, tau_per_order, self.storage, self.flags, theta_ref,
                                    self.pop.data_ptr(), pb, self.work.data_ptr(), wb)
        self.set_stream(stream)

    def set_stream(self, stream=None):
        torch = self.torch
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.stream = s
        lbm_set_stream(self.handle, s.cuda_stream)

    def close(self):
        if getattr(self, "handle", None):
            lbm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # fields -----------------------------------------------------------------
    def init_fields(self, rho, u, theta=None):
        """rho[N], u[D, N] (lattice units) and optional theta[N], as numpy arrays
        (host) or torch tensors (host or device)."""
        torch = self.torch
        if isinstance(rho, torch.Tensor):
            dt = LBM_DTYPE_F64 if rho.dtype == torch.float64 else LBM_DTYPE_F32
            tdt = torch.float64 if dt == LBM_DTYPE_F64 else torch.float32
            rho = rho.to(tdt).contiguous()
            u = u.to(tdt).contiguous()
            th = None if theta is None else theta.to(tdt).contiguous()
            lbm_init_fields(self.handle, rho.data_ptr(), u.data_ptr(), 0 if th is None else th.data_ptr(), dt,
                            rho.is_cuda)
            return
        rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(-1)
        u = np.ascontiguousarray(u, dtype=np.float64).reshape(self.D, -1)
        th = None if theta is None else np.ascontiguousarray(theta, dtype=np.float64).reshape(-1)
        lbm_init_fields(self.handle, _np_ptr(rho), _np_ptr(u), 0 if th is None else _np_ptr(th), LBM_DTYPE_F64, 0)

    def step(self, n=1):
        lbm_step(self.handle, n)

    def moments(self, on_device=False, dtype="f64", with_theta=False):
        """(rho[N], u[D, N]) or, with_theta, (rho, u, theta); numpy (host) or torch (device)."""
        torch = self.torch
        cdt = LBM_DTYPE_F64 if dtype == "f64" else LBM_DTYPE_F32
        if on_device:
            tdt = torch.float64 if dtype == "f64" else torch.float32
            rho = torch.empty(self.N, dtype=tdt, device=self.device)
            u = torch.empty(self.D, self.N, dtype=tdt, device=self.device)
            th = torch.empty(self.N, dtype=tdt, device=self.device) if with_theta else None
            lbm_moments(self.handle, rho.data_ptr(), u.data_ptr(), 0 if th is None else th.data_ptr(), cdt, 1)
        else:
            ndt = np.float64 if dtype == "f64" else np.float32
            rho = np.empty(self.N, dtype=ndt)
            u = np.empty((self.D, self.N), dtype=ndt)
            th = np.empty(self.N, dtype=ndt) if with_theta else None
            lbm_moments(self.handle, _np_ptr(rho), _np_ptr(u), 0 if th is None else _np_ptr(th), cdt, 0)
        return (rho, u, th) if with_theta else (rho, u)

    def populations(self, on_device=False):
        if on_device:
            f = self.torch.empty(self.Q, self.N, dtype=self.torch.float64, device=self.device)
            lbm_get_populations(self.handle, f.data_ptr(), 1)
            return f
        f = np.empty((self.Q, self.N))
        lbm_get_populations(self.handle, _np_ptr(f), 0)
        return f

    def set_populations(self, f):
        torch = self.torch
        if isinstance(f, torch.Tensor) and f.is_cuda:
            f = f.to(torch.float64).contiguous()
            lbm_set_populations(self.handle, f.data_ptr(), 1)
            return
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(self.Q, self.N)
        lbm_set_populations(self.handle, _np_ptr(f), 0)

    def reduce(self):
        return lbm_reduce(self.handle)

    def step_totals(self):
        """One step; returns the FP64 totals of the state it advanced from."""
        out = np.zeros(5)
        _check(load().lbm_step_totals(self.handle, out.ctypes.data_as(_dp)))
        return out

    def step_totals_async(self, out_ptr):
        """One step without waiting; its totals go to host out_ptr[0..5) (see
        lbm_step_totals_async)."""
        lbm_step_totals_async(self.handle, out_ptr)

    def mode_amplitude(self, field, mode):
        return lbm_mode_amplitude(self.handle, field, mode)

    def mode_history(self, field, mode, n_records, stride):
        return lbm_mode_history(self.handle, field, mode, n_records, stride)

    def sweep_kernel(self):
        """Name of the sweep kernel that step() launches with the current settings."""
        return lbm_sweep_kernel(self.handle)

    def set_active_planes(self, z_lo, z_count):
        """Sweep and reduce planes z_lo .. z_lo + z_count - 1 only (D3Q27 slabs)."""
        lbm_set_active_planes(self.handle, z_lo, z_count)

    def set_closure(self, params, norm, omega_lo=0.0, omega_hi=2.0):
        """Relax orders 3..6 at rates in [omega_lo, omega_hi] from the network
        (device FP32 tensors: the 5894 parameters and the 40-value feature
        standardisation); None clears."""
        if params is None:
            lbm_set_closure(self.handle, 0, 0)
            return
        params = params.float().contiguous()
        norm = norm.float().contiguous()
        lbm_set_closure(self.handle, params.data_ptr(), norm.data_ptr(), omega_lo, omega_hi)

    def status(self):
        return lbm_status(self.handle)

    @property
    def step_count(self):
        return lbm_step_count(self.handle)

    def raw_populations(self):
        """The storage buffer viewed in its element type, shape (Q, N) (AA layout)."""
        torch = self.torch
        dt = {LBM_F64: torch.float64, LBM_F32: torch.float32, LBM_F16: torch.float16,
              LBM_BF16: torch.bfloat16}[self.storage]
        n = self.Q * self.N
        return self.pop.view(dt)[:n].view(self.Q, self.N)


# ---- batches of independent runs ---------------------------------------------

BATCH_EXPORTS = (
    "lbm_batch_query_bytes", "lbm_batch_create", "lbm_batch_destroy", "lbm_batch_set_stream",
    "lbm_batch_init_run", "lbm_batch_init_runs", "lbm_batch_step", "lbm_batch_use_graph", "lbm_batch_set_tiles", "lbm_batch_set_launch", "lbm_batch_get_launch",
    "lbm_batch_autotune", "lbm_batch_status", "lbm_batch_reduce", "lbm_batch_moments",
    "lbm_batch_get_populations", "lbm_batch_step_count",
)
EXPORTS = EXPORTS + BATCH_EXPORTS


def _declare_batch(L):
    L.lbm_batch_query_bytes.argtypes = [ctypes.c_int, ctypes.c_int, _i64p, ctypes.c_int, _szp, _szp]
    L.lbm_batch_create.argtypes = [ctypes.c_int, ctypes.c_int, _i64p, _dp, ctypes.c_int, ctypes.c_int, _vp,
                                   ctypes.c_size_t, _vp, ctypes.c_size_t, ctypes.POINTER(_vp)]
    L.lbm_batch_destroy.argtypes = [_vp]
    L.lbm_batch_destroy.restype = None
    L.lbm_batch_set_stream.argtypes = [_vp, _vp]
    L.lbm_batch_init_run.argtypes = [_vp, ctypes.c_int, _vp, _vp, ctypes.c_int, ctypes.c_int]
    L.lbm_batch_init_runs.argtypes = [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_int]
    L.lbm_batch_step.argtypes = [_vp, _i64]
    L.lbm_batch_use_graph.argtypes = [_vp, ctypes.c_int]
    L.lbm_batch_set_tiles.argtypes = [_vp, ctypes.c_int, ctypes.c_int]
    L.lbm_batch_set_launch.argtypes = [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    L.lbm_batch_get_launch.argtypes = [_vp] + [ctypes.POINTER(ctypes.c_int)] * 5
    L.lbm_batch_autotune.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    L.lbm_batch_status.argtypes = [_vp, ctypes.POINTER(ctypes.c_int)]
    L.lbm_batch_reduce.argtypes = [_vp, _dp]
    L.lbm_batch_moments.argtypes = [_vp, ctypes.c_int, _vp, _vp, ctypes.c_int, ctypes.c_int]
    L.lbm_batch_get_populations.argtypes = [_vp, ctypes.c_int, _vp, ctypes.c_int]
    L.lbm_batch_step_count.argtypes = [_vp]
    L.lbm_batch_step_count.restype = ctypes.c_int64


def _batch_lib():
    L = load()
    if not getattr(L, "_batch_declared", False):
        _declare_batch(L)
        L._batch_declared = True
    return L


def _dims_array(dims_list):
    flat = []
    for d in dims_list:
        d = list(int(x) for x in d) + [1] * (3 - len(d))
        flat += d
    return (ctypes.c_int64 * len(flat))(*flat)


class Batch:
    """Independent periodic D2Q9 runs advanced together (one launch per step).

    dims_list: [(nx, ny), ...]; taus: per-run [tau_2, tau_3, tau_4] lists;
    storage as for Simulation.  Buffers are torch-owned.
    """

    def __init__(self, dims_list, taus, storage="bf16", device=None, stream=None):
        import torch
        self.torch = torch
        L = _batch_lib()
        self.dims = [tuple(int(x) for x in d) for d in dims_list]
        self.n_runs = len(self.dims)
        self.storage = STORAGES[storage] if isinstance(storage, str) else int(storage)
        self.device = torch.device(device if device is not None else "cuda")
        n_tau = max(len(t) for t in taus)
        tv = np.ones((self.n_runs, n_tau))
        for r, t in enumerate(taus):
            tv[r, :len(t)] = t
        tv = np.ascontiguousarray(tv)
        d = _dims_array(self.dims)
        pb, wb = ctypes.c_size_t(), ctypes.c_size_t()
        _check(L.lbm_batch_query_bytes(LBM_D2Q9, self.n_runs, d, self.storage, ctypes.byref(pb), ctypes.byref(wb)))
        self.pop = torch.empty(pb.value, dtype=torch.uint8, device=self.device)
        self.work = torch.empty(wb.value, dtype=torch.uint8, device=self.device)
        h = _vp()
        _check(L.lbm_batch_create(LBM_D2Q9, self.n_runs, d, tv.ctypes.data_as(_dp), n_tau, self.storage,
                                  _vp(self.pop.data_ptr()), pb.value, _vp(self.work.data_ptr()), wb.value,
                                  ctypes.byref(h)))
        self.handle = h
        # a stream of its own: CUDA-graph capture is not allowed on the default stream
        s = stream if stream is not None else torch.cuda.Stream(device=self.device)
        self.stream = s
        _check(L.lbm_batch_set_stream(h, _vp(s.cuda_stream)))

    def close(self):
        if getattr(self, "handle", None):
            _batch_lib().lbm_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_run(self, run, rho, u):
        rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(-1)
        u = np.ascontiguousarray(u, dtype=np.float64).reshape(2, -1)
        _check(_batch_lib().lbm_batch_init_run(self.handle, int(run), _vp(_np_ptr(rho)), _vp(_np_ptr(u)),
                                               LBM_DTYPE_F64, 0))

    def init_runs(self, fields):
        """Initialise every run from fields[r] = (rho, u) in one call.  Torch
        tensors (CUDA, or page-locked host memory) are read where they are, by
        one kernel; numpy arrays go run by run through staged copies."""
        torch = self.torch
        keep = []
        on_device = 1 if all(isinstance(r, torch.Tensor) and r.is_cuda for r, _ in fields) else 0
        for rho, u in fields:
            if isinstance(rho, torch.Tensor):
                rho = rho.to(torch.float64).contiguous()
                u = u.to(torch.float64).contiguous()
                keep.append((rho, u, rho.data_ptr(), u.data_ptr()))
            else:
                rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(-1)
                u = np.ascontiguousarray(u, dtype=np.float64).reshape(2, -1)
                keep.append((rho, u, _np_ptr(rho), _np_ptr(u)))
        if len(keep) != self.n_runs:
            raise ValueError("need fields for each of the %d runs" % self.n_runs)
        rp = (_vp * self.n_runs)(*[k[2] for k in keep])
        up = (_vp * self.n_runs)(*[k[3] for k in keep])
        _check(_batch_lib().lbm_batch_init_runs(self.handle, rp, up, LBM_DTYPE_F64, on_device))

    def step(self, n=1):
        _check(_batch_lib().lbm_batch_step(self.handle, int(n)))

    def use_graph(self, enable=True):
        _check(_batch_lib().lbm_batch_use_graph(self.handle, int(bool(enable))))

    def set_tiles(self, threads, rows):
        _check(_batch_lib().lbm_batch_set_tiles(self.handle, int(threads), int(rows)))

    def set_launch(self, split=0, depth=1, staged=1):
        _check(_batch_lib().lbm_batch_set_launch(self.handle, int(bool(split)), int(depth), int(staged)))

    def launch(self):
        """(threads, rows, split, depth, staged) of the current launch mode."""
        v = [ctypes.c_int() for _ in range(5)]
        _check(_batch_lib().lbm_batch_get_launch(self.handle, *[ctypes.byref(x) for x in v]))
        return tuple(x.value for x in v)

    def autotune(self, steps_per_trial=10):
        t, r = ctypes.c_int(), ctypes.c_int()
        _check(_batch_lib().lbm_batch_autotune(self.handle, int(steps_per_trial), ctypes.byref(t), ctypes.byref(r)))
        return t.value, r.value

    def status(self):
        out = (ctypes.c_int * self.n_runs)()
        _check(_batch_lib().lbm_batch_status(self.handle, out))
        return np.array(out[:])

    def reduce(self):
        out = np.zeros(5 * self.n_runs)
        _check(_batch_lib().lbm_batch_reduce(self.handle, out.ctypes.data_as(_dp)))
        return out.reshape(self.n_runs, 5)

    def moments(self, run):
        N = int(np.prod(self.dims[run]))
        rho, u = np.empty(N), np.empty((2, N))
        _check(_batch_lib().lbm_batch_moments(self.handle, int(run), _vp(_np_ptr(rho)), _vp(_np_ptr(u)),
                                              LBM_DTYPE_F64, 0))
        return rho, u

    def populations(self, run):
        N = int(np.prod(self.dims[run]))
        f = np.empty((9, N))
        _check(_batch_lib().lbm_batch_get_populations(self.handle, int(run), _vp(_np_ptr(f)), 0))
        return f

    @property
    def step_count(self):
        return int(_batch_lib().lbm_batch_step_count(self.handle))


# ---- learned closure ------------------------------------------------------------

CLOSURE_EXPORTS = ("lbm_set_closure", "lbm_closure_filter", "lbm_closure_rescale", "lbm_closure_dataset",
                   "lbm_mlp_work_bytes", "lbm_mlp_loss_grad", "lbm_mlp_train")
EXPORTS = EXPORTS + CLOSURE_EXPORTS
MLP_PARAMS = LBM_MLP_PARAMS = 5894


def _closure_lib():
    L = load()
    if not getattr(L, "_closure_declared", False):
        _d = ctypes.c_double
        L.lbm_set_closure.argtypes = [_vp, _vp, _vp, _d, _d]
        L.lbm_closure_filter.argtypes = [_vp, ctypes.c_int, _vp]
        L.lbm_closure_rescale.argtypes = [_i64p, _vp, _d, _vp]
        L.lbm_closure_dataset.argtypes = [_i64p, _vp, _vp, ctypes.c_double, _vp, _vp, _vp, _vp]
        L.lbm_mlp_work_bytes.argtypes = [_i64]
        L.lbm_mlp_work_bytes.restype = ctypes.c_size_t
        L.lbm_mlp_loss_grad.argtypes = [_vp, _vp, _i64, _dp_f, _d, _d, _vp, _vp, _dp, _vp, ctypes.c_size_t, _vp]
        L.lbm_mlp_train.argtypes = [_vp, _vp, _i64, _dp_f, _d, _d, _vp, _vp, _vp, _i64, _i64, ctypes.c_double,
                                    ctypes.c_uint64, _i64, _vp, _vp, ctypes.c_size_t, _vp]
        L._closure_declared = True
    return L


_dp_f = ctypes.POINTER(ctypes.c_float)


def lbm_set_closure(h, params_ptr, norm_ptr, omega_lo=0.0, omega_hi=2.0):
    _check(_closure_lib().lbm_set_closure(h, _vp(params_ptr), _vp(norm_ptr), float(omega_lo), float(omega_hi)))


def lbm_closure_rescale(dims, f_ptr, scale, stream_ptr=None):
    _check(_closure_lib().lbm_closure_rescale(_dims3(dims), _vp(f_ptr), float(scale), _vp(stream_ptr)))


def lbm_closure_filter(h, m, out_ptr):
    _check(_closure_lib().lbm_closure_filter(h, int(m), _vp(out_ptr)))


def lbm_closure_dataset(dims, ft_ptr, ft1_ptr, tau2, norm_ptr, X_ptr, abc_ptr, stream_ptr=None):
    _check(_closure_lib().lbm_closure_dataset(_dims3(dims), _vp(ft_ptr), _vp(ft1_ptr), float(tau2), _vp(norm_ptr),
                                              _vp(X_ptr), _vp(abc_ptr), _vp(stream_ptr)))


def lbm_mlp_work_bytes(batch):
    return int(_closure_lib().lbm_mlp_work_bytes(int(batch)))


def lbm_mlp_loss_grad(X_ptr, abc_ptr, n, cw, params_ptr, grad_ptr, work_ptr, work_bytes, stream_ptr=None,
                      omega_lo=0.0, omega_hi=2.0):
    cwa = (ctypes.c_float * 6)(*[float(c) for c in cw])
    loss = ctypes.c_double()
    _check(_closure_lib().lbm_mlp_loss_grad(_vp(X_ptr), _vp(abc_ptr), int(n), cwa, float(omega_lo), float(omega_hi),
                                            _vp(params_ptr), _vp(grad_ptr), ctypes.byref(loss), _vp(work_ptr),
                                            int(work_bytes), _vp(stream_ptr)))
    return loss.value


def lbm_mlp_train(X_ptr, abc_ptr, n, cw, params_ptr, m_ptr, v_ptr, iters, batch, lr, seed, t0, loss_ptr, work_ptr,
                  work_bytes, stream_ptr=None, omega_lo=0.0, omega_hi=2.0):
    cwa = (ctypes.c_float * 6)(*[float(c) for c in cw])
    _check(_closure_lib().lbm_mlp_train(_vp(X_ptr), _vp(abc_ptr), int(n), cwa, float(omega_lo), float(omega_hi),
                                        _vp(params_ptr), _vp(m_ptr), _vp(v_ptr), int(iters), int(batch), float(lr),
                                        int(seed), int(t0), _vp(loss_ptr), _vp(work_ptr), int(work_bytes),
                                        _vp(stream_ptr)))


# ---- caller-supplied Hermite lattices ----------------------------------------

HERMITE_EXPORTS = ("lbm_hermite_query_bytes", "lbm_create_hermite")
EXPORTS = EXPORTS + HERMITE_EXPORTS


def _hermite_lib():
    L = load()
    if not getattr(L, "_hermite_declared", False):
        L.lbm_hermite_query_bytes.argtypes = [ctypes.c_int, _i64p, ctypes.c_int, _szp, _szp]
        L.lbm_create_hermite.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), _dp, ctypes.c_double,
                                         ctypes.c_int, _i64p, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_uint,
                                         ctypes.c_double, _vp, ctypes.c_size_t, _vp, ctypes.c_size_t,
                                         ctypes.POINTER(_vp)]
        L._hermite_declared = True
    return L


def lbm_hermite_query_bytes(q, dims, storage):
    pb, wb = ctypes.c_size_t(), ctypes.c_size_t()
    _check(_hermite_lib().lbm_hermite_query_bytes(int(q), _dims3(dims), int(storage), ctypes.byref(pb),
                                                  ctypes.byref(wb)))
    return pb.value, wb.value


def lbm_create_hermite(e, w, c, order, dims, tau_per_order, storage, flags, theta_ref, pop_ptr, pop_bytes,
                       work_ptr, work_bytes):
    ee = np.ascontiguousarray(np.asarray(e, dtype=np.int32).reshape(-1))
    ww = np.ascontiguousarray(w, dtype=np.float64)
    taus = np.ascontiguousarray(tau_per_order, dtype=np.float64)
    h = _vp()
    _check(_hermite_lib().lbm_create_hermite(len(ww), ee.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                             ww.ctypes.data_as(_dp), float(c), int(order), _dims3(dims),
                                             taus.ctypes.data_as(_dp), len(taus), int(storage), int(flags),
                                             float(theta_ref), _vp(pop_ptr), int(pop_bytes), _vp(work_ptr),
                                             int(work_bytes), ctypes.byref(h)))
    return h


class HermiteSimulation(Simulation):
    """A periodic CM-MRT simulation on a caller-supplied 2D Hermite lattice.

    rule: a name "E7-A" .. "E7-D" (17 velocities, N = 3) or "E9-A" .. "E9-D"
    (37 velocities, N = 4) from ``gen_rules``, or a tuple (e[Q, 2], w[Q], c, N).
    Populations are in the rule's velocity order; velocities in lattice units.
    """

    def __init__(self, rule, dims, tau_per_order, storage="f64", device=None, stream=None, flags=0,
                 theta_ref=1.0):
        import torch
        if isinstance(rule, str):
            from .gen_rules import rule as _rule
            rule = _rule(rule)
        e, w, c, order = rule
        self.torch = torch
        self.lattice = LBM_HERMITE
        self.storage = STORAGES[storage] if isinstance(storage, str) else int(storage)
        self.D = 2
        self.Q = len(w)
        self.e = np.asarray(e, dtype=np.int32).reshape(-1, 2)
        self.w = np.asarray(w, dtype=np.float64)
        self.c = float(c)
        self.order = int(order)
        self.flags = int(flags)
        self.dims = tuple(int(x) for x in dims)
        if len(self.dims) != 2:
            raise ValueError("dims must have 2 entries")
        self.N = int(np.prod(self.dims))
        self.device = torch.device(device if device is not None else "cuda")
        if self.device.type != "cuda":
            raise RuntimeError("HermiteSimulation runs on a CUDA device only")
        pb, wb = lbm_hermite_query_bytes(self.Q, self.dims, self.storage)
        self.pop = torch.empty(pb, dtype=torch.uint8, device=self.device)
        self.work = torch.empty(wb, dtype=torch.uint8, device=self.device)
        self.handle = lbm_create_hermite(self.e, self.w, self.c, self.order, self.dims, tau_per_order, self.storage,
                                         self.flags, theta_ref, self.pop.data_ptr(), pb, self.work.data_ptr(), wb)
        self.set_stream(stream)
