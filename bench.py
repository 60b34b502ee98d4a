"""Benchmark: CM-MRT lattice Boltzmann sweep throughput on GB300.

Workload (one step = one fused stream+collide sweep over the whole grid):
  D3Q27 CM-MRT, FP32 offset storage, 256^3 triply periodic Taylor-Green vortex,
  Re = 1600, Ma = 0.1 (U0 = 0.1 c_s), tau_2 from nu = U0 (n / 2 pi) / Re, orders
  4 and 6 at tau_2, orders 3 and 5 at tau = 1.  Populations (1.81 GB) exceed L2,
  so no L2 flush is needed.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
instead, on a bounded sample of the same workload.
"""
import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CM-MRT MLUPS & % of HBM roofline; learned vs plain GPU time at equal error"
UNIT = "MLUPS"
N_SIDE = 256
RE, MA = 1600.0, 0.1
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "tp_pair_d3q27_f32_tgv.md")
PROFILE_SUMMARIES = {st: os.path.join(ROOT, "profiles", "tp_pair_d3q27_%s_tgv.md" % st) for st in ("f32", "f16", "bf16")}


def workload_params(n=N_SIDE):
    """U0 = Ma c_s; tau_2 = 1/2 + 3 nu with nu = U0 (n / 2 pi) / Re.  Even orders
    (4, 6) relax with tau_2 and odd orders (3, 5) with tau = 1: any setting with
    tau_4 or tau_6 different from tau_2 diverges within a few hundred steps on this
    flow (the 4th and 6th central monomials contain traces of the 2nd)."""
    U0 = MA / np.sqrt(3.0)
    nu = U0 * (n / (2 * np.pi)) / RE
    t2 = 0.5 + 3.0 * nu
    return U0, [t2, 1.0, t2, 1.0, t2]


STORAGE_BYTES = {"f32": 4, "f16": 2, "bf16": 2}
STORAGE_NAMES = {"f32": "FP32 offset storage", "f16": "FP16 offsets (f - w)/w",
                 "bf16": "BF16 offsets (f - w)/w"}
PASSES = 5  # timed passes of K steps; value from the median pass


def config(n=N_SIDE, storage="f32"):
    U0, taus = workload_params(n)
    b = STORAGE_BYTES[storage]
    return {
        "workload": "D3Q27 CM-MRT Taylor-Green vortex %d^3 periodic, Re %g, Ma %g, %s, FP32 collision, "
                    "AA in-place fused stream+collide; tau = [tau2, 1, tau2, 1, tau2]"
                    % (n, RE, MA, STORAGE_NAMES[storage]),
        "lattice": "D3Q27", "grid": [n, n, n], "storage": storage, "tau_per_order": taus,
        "bytes_per_lup": 2 * 27 * b,
        "l2": "inputs larger than L2 (populations %.2f GB), no flush" % (27 * n ** 3 * b / 1e9),
    }


# Learned-closure coarse run: decaying isotropic turbulence, 128^3, k0 = 4, u_rms 0.04,
# Re_lambda 100 of the 512^3 fine run in acoustic scaling (nu_coarse = nu_fine / 4).
LEARNED_N, LEARNED_K0, LEARNED_URMS, LEARNED_RE = 128, 4.0, 0.04, 100.0
# Rate range of the network's outputs, chosen on a validation seed (2) that the
# reported run (seed 0) does not use: the lower bound sits 0.1 above the first one
# that diverged there (0.4), the upper bound where a lower one only did worse.
LEARNED_RANGE = (0.5, 1.98)
MLP_FLOPS_PER_NODE = 2 * (32 * 64 + 64 * 64 + 64 * 8)  # padded GEMMs issued per node


def learned_network(taus, device):
    """A network for the timing workload: seeded random hidden layers with a small
    output layer around the plain model's rates (orders 3, 5 near 1, orders 4, 6
    near omega_2), so the run stays stable while every node still evaluates the
    full network."""
    import torch
    from paper_1808_04406_gb300 import closure as C
    P = C.init_params(1, device)
    lo, hi = LEARNED_RANGE
    om = [1.02, 1.02, 1.0 / taus[0], 1.0 / taus[0], 1.02, 1.0 / taus[0]]
    q = torch.tensor([(min(max(o, lo + 1e-3), hi - 1e-3) - lo) / (hi - lo) for o in om], device=device)
    P[5888 - 6 * 64:5888] *= 0.05  # W3
    P[5888:] = torch.log(q / (1 - q))  # b3
    return P


def learned_params(n=LEARNED_N):
    from paper_1808_04406_gb300 import closure as C
    nu = C.taylor_scale_viscosity(4 * n, LEARNED_K0, LEARNED_URMS, LEARNED_RE) / 4.0
    t2 = 0.5 + 3.0 * nu
    return [t2, 1.0, t2, 1.0, t2]


PAIR_SOURCES = ("tp_pair.cu", "sweep_body.cuh", "pair_io.cuh", "tp_common.cuh", "f32x2.cuh", "lbm_internal.cuh")
KERNEL_LABELS = {
    "tp_pair_kernel": "tp_pair_kernel<3, %s> (two nodes per thread, packed FP32x2)",
    "tp_pair_zrun_kernel": "tp_pair_zrun_kernel<%s> (two nodes per thread, packed FP32x2; each thread walks 8 "
                           "planes with the next plane's loads in flight)",
    "tp_sweep_kernel": "tp_sweep_kernel<3, %s> (one node per thread)",
}
BATCH_PROFILE = os.path.join(ROOT, "profiles", "batch_sweep_d2q9_bf16.md")
BATCH_SOURCES = ("batch.cu", "batch_stage.cuh", "sweep_body.cuh", "pair_io.cuh", "tp_common.cuh", "f32x2.cuh",
                 "tc05.cuh", "lbm_internal.cuh")


def kernel_source_hash(names=PAIR_SOURCES):
    h = hashlib.sha256()
    for name in names:
        with open(os.path.join(ROOT, "paper_1808_04406_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(summary=PROFILE_SUMMARY, names=PAIR_SOURCES):
    """DRAM bytes per sweep launch from the committed ncu summary, or None when the
    kernel source changed since the counters were taken."""
    try:
        text = open(summary).read()
    except OSError:
        return None
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    hm = re.search(r"kernel_source_hash:\s*([0-9a-f]+)", text)
    if not m or not hm or hm.group(1) != kernel_source_hash(names):
        return None
    return float(m.group(1))


def measured_peak_bf16():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["bf16_tflops"])
    except (OSError, KeyError, ValueError):
        return 1900.0


def measured_peak_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except OSError:
            pass
        finally:
            try:
                os.unlink(self.path)
            except OSError:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


class NvmlSampler:
    """SM clock and clock-event reasons read through NVML (the driver's own
    library, by ctypes) every `period` seconds on a host thread, so that a timed
    region of a few milliseconds still holds samples; reads only.  mark(label)
    brackets a pass by host time (each pass ends with a device synchronise, so
    its host interval covers its GPU work).  Falls back to no samples when NVML
    cannot be loaded."""
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown"}

    def __init__(self, cuda_index=0, period=0.002):
        self.period = period
        self.samples = []  # (host time, sm MHz, reasons bitmask)
        self.passes = []   # (label, t0, t1)
        self.lib = None
        self.handle = None
        self.max_mhz = None
        self._stop = False
        try:
            import ctypes
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                return
            h = ctypes.c_void_p()
            bus = self._pci_bus_id(cuda_index)
            rc = (lib.nvmlDeviceGetHandleByPciBusId_v2(bus.encode(), ctypes.byref(h)) if bus
                  else lib.nvmlDeviceGetHandleByIndex_v2(cuda_index, ctypes.byref(h)))
            if rc != 0:
                return
            mx = ctypes.c_uint()
            if lib.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0:
                self.max_mhz = float(mx.value)
            self.lib, self.handle, self.ct = lib, h, ctypes
        except OSError:
            self.lib = None

    @staticmethod
    def _pci_bus_id(cuda_index):
        try:
            import torch
            p = torch.cuda.get_device_properties(cuda_index)
            return "%08x:%02x:%02x.0" % (p.pci_domain_id, p.pci_bus_id, p.pci_device_id)
        except (AttributeError, RuntimeError, AssertionError):
            return None

    def _read(self):
        ct = self.ct
        mhz, reasons = ct.c_uint(), ct.c_ulonglong()
        if self.lib.nvmlDeviceGetClockInfo(self.handle, 1, ct.byref(mhz)) != 0:
            return None
        if self.lib.nvmlDeviceGetCurrentClocksThrottleReasons(self.handle, ct.byref(reasons)) != 0:
            reasons.value = 0
        return time.perf_counter(), float(mhz.value), int(reasons.value)

    def _loop(self):
        while not self._stop:
            s = self._read()
            if s:
                self.samples.append(s)
            time.sleep(self.period)

    def __enter__(self):
        if self.lib is not None:
            import threading
            self.thread = threading.Thread(target=self._loop, daemon=True)
            self.thread.start()
        return self

    def __exit__(self, *exc):
        self._stop = True
        if self.lib is not None:
            self.thread.join(timeout=2)

    def mark(self, label, t0, t1):
        self.passes.append((label, t0, t1))

    def _stats(self, rows):
        if not rows:
            return {"sm_mhz": None, "samples": 0, "reasons": []}
        bits = 0
        for r in rows:
            bits |= r[2]
        return {"sm_mhz": statistics.median(r[1] for r in rows), "samples": len(rows),
                "reasons": sorted(v for k, v in self.REASONS.items() if bits & k)}

    def summary(self):
        if self.lib is None:
            return None
        inside = [r for r in self.samples if any(a <= r[0] <= b for _, a, b in self.passes)]
        out = dict(self._stats(inside), sm_max_mhz=self.max_mhz, source="NVML every %g ms" % (1e3 * self.period))
        out["per_pass"] = [dict(self._stats([r for r in self.samples if a <= r[0] <= b]), label=lab)
                           for lab, a, b in self.passes]
        return out


def merge_clocks(smi, nvml):
    """The nvidia-smi record of the timed region with the NVML one beside it;
    NVML's reasons are added to the top-level list so that no reason is lost."""
    if nvml is None:
        return smi
    out = dict(smi)
    out["reasons"] = sorted(set(smi.get("reasons") or []) - {"unsampled"} | set(nvml["reasons"]))
    if out.get("sm_mhz") is None:
        out["sm_mhz"] = nvml["sm_mhz"]
        out["sm_max_mhz"] = nvml["sm_max_mhz"]
    out["nvml"] = nvml
    return out


def cpu_baseline_sample(n=64, steps=100):
    """Time the FP64 oracle on a bounded sample of the workload: a TGV of side n with
    the same Re and Ma, `steps` steps, all host cores (OpenMP)."""
    import oracle
    from paper_1808_04406_gb300 import inputs
    U0, taus = workload_params(n)
    rho, u = inputs.taylor_green_3d(n, U0)
    f = oracle.tp_init(3, rho, u)
    om = oracle.omega_from_tau(3, taus)
    oracle.tp_step(3, (n, n, n), om, f, 1)  # warm
    t0 = time.perf_counter()
    oracle.tp_step(3, (n, n, n), om, f, steps)
    dt = time.perf_counter() - t0
    return {"value": n ** 3 * steps / dt / 1e6, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": "D3Q27 TGV %d^3 (Re %g, Ma %g), %d steps, FP64 oracle (Kronecker variant), %.1f s"
                      % (n, RE, MA, steps, dt)}


def cpu_baseline_learned(n=12):
    """The FP64 oracle's learned step (features, network, per-node collision,
    stream) on a bounded sample: one step of an n^3 grid of smooth random flow."""
    import oracle
    from oracle import closure as OC
    from paper_1808_04406_gb300 import inputs
    rho, u = inputs.random_smooth((n, n, n), seed=0, du=0.04)
    f = oracle.tp_init(3, rho, u)
    taus = learned_params()
    P = OC.init_params(1)
    norm = (np.zeros(20), np.ones(20))
    t = time.perf_counter()
    steps = 0
    while time.perf_counter() - t < 10.0:
        f = OC.learned_step(f, (n, n, n), taus[0], P, norm, *LEARNED_RANGE)
        steps += 1
    dt = time.perf_counter() - t
    return {"value": n ** 3 * steps / dt / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "%d learned steps of a %d^3 grid (FP64 features, network, definitional per-node collision)"
                      % (steps, n)}


def run_reference(args, rank, world):
    """Reference arm: the CPU oracle as it stands, one bounded sample per step."""
    if rank != 0:
        return
    import oracle
    from paper_1808_04406_gb300 import inputs
    n = 48
    U0, taus = workload_params(n)
    rho, u = inputs.taylor_green_3d(n, U0)
    f = oracle.tp_init(3, rho, u)
    om = oracle.omega_from_tau(3, taus)
    for _ in range(args.warmup):
        oracle.tp_step(3, (n, n, n), om, f, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.tp_step(3, (n, n, n), om, f, 1)
    dt = time.perf_counter() - t0
    v = n ** 3 * args.steps / dt / 1e6
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference", "config": config(),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": "each step: one FP64 oracle step of a D3Q27 TGV %d^3 sample" % n},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def e2e_legs(sim, steps, init, final, sync=None, advance=None):
    """The end-to-end leg, through the public API, in two forms (seconds each):
    init() from pinned host fields, `steps` steps that each return the FP64
    totals of the state they advanced from, final() fields to host.
      pipelined: lbm_step_totals_async copies every step's totals into pinned
        host memory on the stream (no host wait per step); final() synchronises
        and the host then checks the totals of all steps (mass drift);
      blocking: lbm_step_totals, the host waiting for each step's totals.
    Returns (pipelined s, blocking s, largest |total mass - first| seen)."""
    import torch
    tot = torch.zeros((steps, 5), dtype=torch.float64).pin_memory()
    base = tot.data_ptr()
    sync = sync or torch.cuda.synchronize
    # one untimed pass through the same calls first (its first host-memory
    # accesses and launches are not part of the steady state being measured)
    init()
    for k in range(min(steps, 2)):
        if advance is None:
            sim.step_totals_async(base + 40 * k)
        else:
            advance(1, lambda k=k: sim.step_totals_async(base + 40 * k))
    final()
    sync()
    t0 = time.perf_counter()
    init()
    for k in range(steps):
        if advance is None:
            sim.step_totals_async(base + 40 * k)
        else:
            advance(1, lambda k=k: sim.step_totals_async(base + 40 * k))
    final()
    torch.cuda.synchronize()
    m = tot[:, 0].numpy()
    drift = float(np.abs(m - m[0]).max())
    pipelined = time.perf_counter() - t0
    sync()
    t0 = time.perf_counter()
    init()
    for _ in range(steps):
        if advance is None:
            sim.step_totals()
        else:
            advance(1, sim.step_totals)
    final()
    torch.cuda.synchronize()
    blocking = time.perf_counter() - t0
    return pipelined, blocking, drift


E2E_DEFINITION = ("(after one untimed pass) init from pinned host fields + K x (step whose FP64 totals of the state it advanced from are "
                  "copied to pinned host memory on the stream, no host wait per step) + final fields to host "
                  "(synchronises) + host check of the K totals; blocking_value: the same with the host waiting "
                  "for each step's totals")


def max_over_ranks(value, dist, device):
    """The largest of the ranks' values, returned on every rank (the slowest rank's
    time bounds a whole-job throughput); the value itself when there is one rank."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world, units_per_rank, steps, seconds):
    """Whole-job throughput of `world` independent replicas in millions of units per
    second: every rank's units over the slowest rank's time."""
    return world * units_per_rank * steps / seconds / 1e6


def run_gpu(args, rank, world, dist):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1808_04406_gb300 import inputs
    from paper_1808_04406_gb300.lbm import Simulation

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    learned = args.workload == "learned128"
    storage = "f32" if learned else (args.storage or "f32")
    if storage not in STORAGE_BYTES:
        raise SystemExit("--storage must be one of f32, f16, bf16 for this workload")
    if learned:
        n = LEARNED_N
        taus = learned_params(n)
        rho, u = inputs.isotropic_turbulence_3d(n, 0, k0=LEARNED_K0, u_rms=LEARNED_URMS)
    else:
        n = args.n
        U0, taus = workload_params(n)
    slab_run = None
    if args.decomp == "slab" and not learned:
        # one grid of n x n x (n world) planes split into slabs along z, one per
        # rank, with the halo exchange of slab.py (NCCL between the ranks' GPUs)
        from paper_1808_04406_gb300 import slab as SL
        gdims = (n, n, n * world)
        z0, nzl = SL.split(gdims[2], world)[rank]
        planes = [(z0 - 1 + k) % gdims[2] for k in range(nzl + 2)]
        rho, u = inputs.taylor_green_3d_planes(n, U0, gdims[2], planes)
    elif not learned:
        rho, u = inputs.taylor_green_3d(n, U0)
    rho_t = torch.tensor(rho, dtype=torch.float32).pin_memory()
    u_t = torch.tensor(u, dtype=torch.float32).pin_memory()
    del rho, u
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        if args.decomp == "slab" and not learned:
            slab_run = SL.SlabRun.create(gdims, taus, storage, rank, world,
                                         transport=SL.TorchTransport(dist) if world > 1 else None,
                                         device=dev, stream=stream)
            sim = slab_run.sim
        else:
            sim = Simulation("D3Q27", (n, n, n), taus, storage=storage, device=dev, stream=stream)
        sim.init_fields(rho_t.to(dev), u_t.to(dev))
        if learned:
            norm = torch.cat([torch.zeros(20), torch.ones(20)]).to(dev)
            sim.set_closure(learned_network(taus, dev), norm, *LEARNED_RANGE)
    sweep_name = sim.sweep_kernel()
    N = n ** 3

    def advance(k=1, sweep=None):
        """k steps: plain sweeps, or slab sweeps with the halo exchange around odd ones."""
        if slab_run is None:
            if sweep is None:
                sim.step(k)
            else:
                for _ in range(k):
                    sweep()
        else:
            with torch.cuda.stream(stream):
                slab_run.step(k, sweep)

    def barrier():
        if dist is not None:
            dist.barrier()

    # warm-up
    advance(args.warmup)
    torch.cuda.synchronize()
    # timed region: PASSES passes of exactly K sweeps, each pass bracketed by a
    # barrier and a synchronise on both sides, each sweep by events on its stream;
    # value is taken from the median pass
    passes = []
    launch_ms = []
    with ClockSampler(local) as clk, NvmlSampler(local) as nv:
        for p in range(PASSES):
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(args.steps)]
            t_start = torch.cuda.Event(enable_timing=True)
            t_end = torch.cuda.Event(enable_timing=True)
            barrier()
            torch.cuda.synchronize()
            h0 = time.perf_counter()
            t_start.record(stream)
            for a, b in evs:
                a.record(stream)
                advance(1)
                b.record(stream)
            t_end.record(stream)
            torch.cuda.synchronize()
            nv.mark(p, h0, time.perf_counter())
            barrier()
            passes.append(max_over_ranks(t_start.elapsed_time(t_end), dist, dev))
            launch_ms += [a.elapsed_time(b) for a, b in evs]
    total_ms = statistics.median(passes)
    status = sim.status()

    # end to end through the public API with host buffers (e2e_legs)
    # the fields of every node the handle holds (a slab's grid includes its two ghost planes)
    out_rho = torch.empty(sim.N, dtype=torch.float32).pin_memory()
    out_u = torch.empty(3, sim.N, dtype=torch.float32).pin_memory()
    from paper_1808_04406_gb300 import lbm as L

    def e2e_sync():
        barrier()
        torch.cuda.synchronize()

    def e2e_final():
        if slab_run is not None:
            with torch.cuda.stream(stream):
                slab_run.refresh_ghosts()
        L.lbm_moments(sim.handle, out_rho.data_ptr(), out_u.data_ptr(), 0, L.LBM_DTYPE_F32, 0)

    e_dt, e_blk, e_drift = e2e_legs(sim, args.steps, lambda: sim.init_fields(rho_t, u_t), e2e_final, e2e_sync,
                                    advance=advance)
    e_dt = max_over_ranks(e_dt, dist, dev)
    e_blk = max_over_ranks(e_blk, dist, dev)
    h2d = (rho_t.numel() + u_t.numel()) * 4
    d2h = (out_rho.numel() + out_u.numel()) * 4

    if rank != 0:
        return
    value = replica_throughput(world, N, args.steps, total_ms * 1e-3)
    avg_launch_s = statistics.mean(launch_ms) * 1e-3
    first_odd = args.warmup & 1
    par = {"even": [t for k, t in enumerate(launch_ms) if (k + first_odd) % 2 == 0],
           "odd": [t for k, t in enumerate(launch_ms) if (k + first_odd) % 2 == 1]}
    bytes_per_launch = 2 * 27 * STORAGE_BYTES[storage] * N
    peak, peak_kind = measured_peak_hbm()
    achieved = bytes_per_launch / avg_launch_s / 1e9
    if learned:
        cfg = {"workload": "D3Q27 CM-MRT with the learned closure fused into the sweep: decaying isotropic "
                           "turbulence %d^3, E(k) ~ k^4 exp(-2 (k/k0)^2), k0 %g, u_rms %g, Re_lambda %g of the "
                           "%d^3 fine run in acoustic scaling; FP32 offsets; 20-64-64-6 BF16 network (tcgen05), "
                           "rates of orders 3..6 in [%g, %g]" % (n, LEARNED_K0, LEARNED_URMS, LEARNED_RE, 4 * n,
                                                                 LEARNED_RANGE[0], LEARNED_RANGE[1]),
               "lattice": "D3Q27", "grid": [n, n, n], "storage": "f32", "tau_per_order": taus,
               "bytes_per_lup": 216, "mlp_flops_per_lup": MLP_FLOPS_PER_NODE,
               "l2": "populations %.0f MB fit in L2; each sweep still reads and writes all of them once"
                     % (27 * N * 4 / 1e6)}
        kname = "learned_tc_kernel (one node per thread; network on tcgen05, M = 128 tiles, TMEM accumulators)"
    else:
        cfg = config(n, storage)
        kname = KERNEL_LABELS[sweep_name] % storage
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(cfg, parallelism=("slab decomposition along z, halo exchange over NCCL"
                                         if slab_run is not None and world > 1 else
                                         "replicas" if world > 1 else "single GPU"),
                       **({"global_grid": [n, n, n * world], "slab": [n, n, n]} if slab_run is not None else {})),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": (None if learned or sweep_name not in ("tp_pair_kernel", "tp_pair_zrun_kernel")
                                 else profiled_traffic(PROFILE_SUMMARIES[storage])),
                     "peak_kind": peak_kind, "kernel": kname,
                     "algorithmic_bytes_per_launch": bytes_per_launch,
                     "mean_launch_ms": {k: statistics.mean(v) for k, v in par.items() if v}},
        "e2e": {"value": replica_throughput(world, N, args.steps, e_dt), "unit": UNIT,
                "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps + 40,
                "blocking_value": replica_throughput(world, N, args.steps, e_blk), "mass_drift": e_drift,
                "definition": E2E_DEFINITION},
        "gpu_launches": args.steps,
        "passes": {"count": PASSES, "steps_each": args.steps, "ms": passes,
                   "spread": (max(passes) - min(passes)) / statistics.median(passes),
                   "note": "value and ms_per_step from the median pass; gpu_launches per pass"},
        "clocks": merge_clocks(clk.summary(), nv.summary()),
        "status": status,
    }
    if learned:
        tflops = MLP_FLOPS_PER_NODE * N / avg_launch_s / 1e12
        bf16_peak = measured_peak_bf16()
        line["roofline"]["tensor"] = {"achieved": tflops, "peak": bf16_peak, "unit": "TFLOP/s",
                                      "frac": tflops / bf16_peak if bf16_peak else None,
                                      "note": "BF16 tensor-core FLOPs of the fused network per launch (padded "
                                              "GEMMs: K 32 / 80, N 64 / 64 / 16 counted as 20-64-64-8)"}
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_learned() if learned else cpu_baseline_sample()
    if (world == 1 and not learned and slab_run is None and storage == "f32" and n == N_SIDE
            and not args.no_secondary):
        line["secondary"] = run_secondary(args)
    print(json.dumps(line), flush=True)


# The other configurations, measured by the default run in child processes after
# its own timed region (each with its own warm-up, timing and clock samples), so
# that one run records them all.  Each entry: the child's arguments and a compact
# copy of its JSON line.
SECONDARY = (
    ("tgv256 FP16 offsets", ["--storage", "f16"]),
    ("tgv256 BF16 offsets", ["--storage", "bf16"]),
    ("thermal1024 FP16 offsets", ["--workload", "thermal1024", "--steps", "1000", "--warmup", "20"]),
    ("batch512 BF16 offsets", ["--workload", "batch512", "--steps", "20", "--warmup", "5"]),
    ("learned128", ["--workload", "learned128", "--steps", "200", "--warmup", "5"]),
    ("closure: learned vs plain GPU time at equal spectrum error", ["--workload", "closure"]),
)
SECONDARY_TIMEOUT_S = 600


def compact_line(d):
    r = d.get("roofline", {})
    e = d.get("e2e") or {}
    c = d.get("clocks") or {}
    out = {"value": d.get("value"), "unit": d.get("unit"), "ms_per_step": d.get("ms_per_step"),
           "steps": d.get("steps"), "dtype": d.get("dtype"), "workload": (d.get("config") or {}).get("workload"),
           "roofline": {k: r.get(k) for k in ("bound", "frac", "achieved", "peak", "unit", "peak_kind", "kernel",
                                              "traffic")},
           "e2e": e.get("value"), "clocks": {"sm_mhz": c.get("sm_mhz"), "sm_max_mhz": c.get("sm_max_mhz"),
                                             "reasons": c.get("reasons")},
           "status": d.get("status")}
    for k in ("hbm", "alu", "tensor"):
        if isinstance(r.get(k), dict):
            out["roofline"][k] = {kk: r[k].get(kk) for kk in ("bound", "frac", "achieved", "peak", "unit")}
    if "passes" in d:
        out["passes_spread"] = d["passes"].get("spread")
    res = d.get("result")
    if isinstance(res, dict):  # the learned-versus-plain experiment
        keep = ("n", "steps", "gpu_ms", "status", "spectrum_error")
        out["result"] = {k: {kk: (res.get(k) or {}).get(kk) for kk in keep} for k in ("plain_coarse", "plain_medium")}
        out["result"]["learned"] = [
            {kk: r.get(kk) for kk in keep + ("omega_lo", "omega_hi", "apriori_gain", "plain_gpu_ms_at_equal_error",
                                              "time_ratio_at_equal_error")} for r in res.get("learned", [])]
    return out


def run_secondary(args):
    res = []
    for name, extra in SECONDARY:
        cmd = [sys.executable, os.path.abspath(__file__), "--no-cpu-baseline", "--no-secondary"]
        if "--steps" not in extra:
            cmd += ["--steps", str(args.steps), "--warmup", str(args.warmup)]
        cmd += extra
        entry = {"name": name, "args": cmd[2:]}
        t0 = time.perf_counter()
        try:
            p = subprocess.run(cmd, capture_output=True, text=True, timeout=SECONDARY_TIMEOUT_S)
            lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
            if p.returncode == 0 and lines:
                entry.update(compact_line(json.loads(lines[-1])))
            else:
                entry["error"] = "exit %d: %s" % (p.returncode, (p.stderr or p.stdout).strip()[-300:])
        except subprocess.TimeoutExpired:
            entry["error"] = "no result within %d s" % SECONDARY_TIMEOUT_S
        entry["wall_s"] = round(time.perf_counter() - t0, 1)
        res.append(entry)
    return res


def run_batch(args):
    """Batched workload: 512 independent D2Q9 CM-MRT decaying-turbulence runs,
    sides uniform in 64..512 (seed 0), E(k) ~ k^-3 random-phase velocity at
    Ma 0.1 (seed = run index), Re log-uniform in [1e3, 1e5] (tau_2 = 1/2 + 3 nu,
    nu = u_rms s / Re), orders 3-4 at tau = 1, BF16 offsets; one launch per step
    for the whole batch (shared-memory band sweep or tile sweep, whichever the
    autotuner finds faster; two-step CUDA graph)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1808_04406_gb300 import inputs
    from paper_1808_04406_gb300.lbm import Batch
    torch.cuda.set_device(0)
    sides, re = inputs.batched_run_sizes(args.runs)
    u_rms = 0.1 / np.sqrt(3.0)
    taus = [[0.5 + 3.0 * u_rms * s / r, 1.0, 1.0] for s, r in zip(sides, re)]
    b = Batch([(int(s), int(s)) for s in sides], taus, storage="bf16")
    if args.batch_launch is None:
        threads, rows = b.autotune(10)
    else:  # a fixed mode (profiling: the autotuner's choice can differ under a profiler)
        b.set_tiles(64, 16)
        b.set_launch(0, 2, args.batch_launch)
        threads, rows = 64, 16
    for r, s in enumerate(sides):
        rho, u = inputs.decaying_turbulence_2d(int(s), seed=r, ma=0.1)
        b.init_run(r, rho, u)
    b.use_graph(True)
    _, _, split, depth, staged = b.launch()
    nodes = int(sum(int(s) ** 2 for s in sides))
    b.step(args.warmup + (args.warmup & 1))
    torch.cuda.synchronize()
    K = args.steps + (args.steps & 1)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        e0.record(b.stream)
        b.step(K)
        e1.record(b.stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    diverged = int(np.sum(b.status() != 0))
    peak, peak_kind = measured_peak_hbm()
    achieved = 36.0 * nodes * K / (ms * 1e-3) / 1e9

    # end to end through the public API on a fresh batch in the same launch mode: every
    # run initialised from pinned host fields, K x (one step + the per-run status read
    # back), then the per-run FP64 totals to host
    b.close()
    del b
    host = []
    for r, s in enumerate(sides):
        rho, u = inputs.decaying_turbulence_2d(int(s), seed=r, ma=0.1)
        host.append((torch.tensor(rho, dtype=torch.float64).pin_memory(),
                     torch.tensor(u, dtype=torch.float64).pin_memory()))
    b2 = Batch([(int(s), int(s)) for s in sides], taus, storage="bf16")
    b2.set_tiles(threads, rows)
    b2.set_launch(split, depth, staged)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b2.init_runs(host)  # lbm_batch_init_runs: one kernel reads every run's pinned fields
    for _ in range(K):
        b2.step(1)
        b2.status()
    b2.reduce()
    torch.cuda.synchronize()
    e_dt = time.perf_counter() - t0
    h2d = sum(rh.numel() * 8 + uh.numel() * 8 for rh, uh in host)
    b2.close()
    line = {"metric": METRIC, "value": nodes * K / (ms * 1e-3) / 1e6, "unit": UNIT, "n_gpus": 1, "steps": K,
            "warmup": args.warmup, "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": "%d independent D2Q9 CM-MRT decaying-turbulence runs, sides U{64..512}, "
                                   "Re log-uniform 1e3..1e5, BF16 offsets, one launch per step" % args.runs,
                       "nodes_per_step": nodes, "cuda_graph": True,
                       "launch": {"staged_shape": staged, "tiles": [threads, rows], "split": split, "depth": depth},
                       "l2": "inputs larger than L2 (%.2f GB of populations), no flush" % (18.0 * nodes / 1e9)},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": (profiled_traffic(BATCH_PROFILE, BATCH_SOURCES)
                                     if staged == 1 and args.runs == 512 else None),
                         "peak_kind": peak_kind,
                         "kernel": ("stg::staged_kernel<bf16> (shared-memory bands, shape %d)" % staged if staged
                                    else "batch_sweep_kernel<bf16>"),
                         "algorithmic_bytes_per_launch": 36.0 * nodes},
            "e2e": {"value": nodes * K / e_dt / 1e6, "unit": UNIT, "h2d_bytes_per_step": h2d / K,
                    "d2h_bytes_per_step": 4 * args.runs + 40 * args.runs / K,
                    "definition": "every run initialised from pinned host rho,u + K x (step + per-run status "
                                  "read back) + per-run FP64 totals to host"},
            "diverged_runs": diverged, "gpu_launches": K, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


THERMAL_N, THERMAL_THETA0, THERMAL_PR = 1024, 1.2, 0.71
# FP32 arithmetic of one 37-velocity thermal lattice update: 2 x 515 FFMA + 172 FADD +
# 36 FMUL, the one-node kernel's executed counts (ncu, FP32 storage, both parities);
# 16-bit offsets add 37 + 37 FMUL for the w_i scaling.
H37_FLOPS_PER_LUP = 1238.0
H37_SCALE_FLOPS = 74.0
# FP32 ALU peak from unit counts: 128 FP32 FMA lanes per SM x 2 flop x SMs x SM clock.
FP32_LANES_PER_SM = 128


def fp32_alu_peak_tflops(sm_mhz):
    sms = torch_sm_count()
    return sms * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12


def torch_sm_count():
    import torch
    return torch.cuda.get_device_properties(0).multi_processor_count


# FMA-throughput probe (lbm_alu_probe): iterations per launch so that one launch
# takes a few milliseconds at the expected rate
ALU_PROBE_ITERS = {"f32": 65536, "f32x2": 32768, "f64": 1024}


def measure_alu_peak(kind, launches=10, warmup=3):
    """Measured FMA throughput of this GPU in TFLOP/s for kind "f32" (scalar
    fma.rn.f32), "f32x2" (packed) or "f64": the median of `launches` timed probe
    launches (CUDA events on the probe's stream), 8 blocks of 256 threads per SM,
    8 independent FMA chains per thread."""
    import torch
    from paper_1808_04406_gb300 import lbm as L
    code = {"f32": L.LBM_PROBE_F32, "f32x2": L.LBM_PROBE_F32X2, "f64": L.LBM_PROBE_F64}[kind]
    sink = torch.zeros(16, device="cuda")
    st = torch.cuda.Stream()
    blocks = torch_sm_count() * 8
    times = []
    flops = 0.0
    for r in range(warmup + launches):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        flops = L.lbm_alu_probe(code, ALU_PROBE_ITERS[kind], blocks, 256, sink.data_ptr(), st.cuda_stream)
        b.record(st)
        torch.cuda.synchronize()
        if r >= warmup:
            times.append(a.elapsed_time(b))
    return flops / statistics.median(times) / 1e9


def run_alu_peak(args):
    """The FMA-throughput probes alone: measured FP32 (scalar and packed) and FP64
    peaks, the denominators of the ALU rooflines, with the clocks of the run."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    measure_alu_peak("f32", 2, 1)  # load and warm
    with ClockSampler(0) as clk, NvmlSampler(0) as nv:
        h0 = time.perf_counter()
        peaks = {k: measure_alu_peak(k) for k in ("f32", "f32x2", "f64")}
        nv.mark("probes", h0, time.perf_counter())
    sms = torch_sm_count()
    clocks = merge_clocks(clk.summary(), nv.summary())
    mhz = clocks.get("sm_mhz") or 2070.0
    nominal = {"f32": sms * FP32_LANES_PER_SM * 2 * mhz * 1e-6, "f64": sms * FP64_LANES_PER_SM * 2 * mhz * 1e-6}
    line = {"metric": "FMA throughput (measured ALU peaks)", "value": peaks["f32x2"], "unit": "TFLOP/s", "n_gpus": 1,
            "steps": 10, "warmup": 3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "lbm_alu_probe: 8 blocks x 256 threads per SM, 8 independent FMA chains per "
                                   "thread on registers, median of 10 launches", "iters": ALU_PROBE_ITERS},
            "result": {"f32_tflops": peaks["f32"], "f32x2_tflops": peaks["f32x2"], "f64_tflops": peaks["f64"],
                       "nominal_at_sampled_clock": {"f32_tflops": nominal["f32"], "f64_tflops": nominal["f64"]}},
            "gpu_launches": 3 * 13, "clocks": clocks}
    print(json.dumps(line), flush=True)


def run_thermal(args):
    """37-velocity thermal CM-MRT (Hermite N = M = 4), 1024^2 periodic, FP16
    offsets from the reference equilibrium, FP32 collision: a temperature wave
    plus a shear wave at mode 10 (theta0 1.2, amplitude 1e-3); tau_2 = 1/2 +
    0.1/theta0, tau_3 = 1/2 + (tau_2 - 1/2)/Pr, tau_4 = tau_2.  One launch per
    step (two-node FP32x2 kernel)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1808_04406_gb300 import inputs
    from paper_1808_04406_gb300 import lbm as L
    torch.cuda.set_device(0)
    n = THERMAL_N
    t2 = 0.5 + 0.1 / THERMAL_THETA0
    taus = [t2, 0.5 + (t2 - 0.5) / THERMAL_PR, t2]
    rho, u, th = inputs.thermal_wave((n, n), amplitude=1e-3, theta0=THERMAL_THETA0, mode=10,
                                     shear_amplitude=1e-3)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        flags = (L.LBM_THERMAL | (L.LBM_STOCHASTIC_ROUND if args.sround else 0)
                 | (L.LBM_FAST_TRANSFORMS if args.fast_transforms else 0))
        sim = L.Simulation("D2Q37", (n, n), taus, storage=args.storage or "f16", flags=flags,
                           theta_ref=THERMAL_THETA0, stream=stream)
        sim.init_fields(rho, u, th)
    sim.step(args.warmup)
    torch.cuda.synchronize()
    K = args.steps
    # launches of ~40 us: `value` comes from K back-to-back steps with no event
    # between them; the per-launch durations of the roofline from a second pass
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    with ClockSampler(0) as clk:
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        sim.step(K)
        t1.record(stream)
        torch.cuda.synchronize()
        for a, b in evs:
            a.record(stream)
            sim.step(1)
            b.record(stream)
        torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    launch = statistics.mean(a.elapsed_time(b) for a, b in evs) * 1e-3
    st = sim.status()
    esize = {"f16": 2, "bf16": 2, "f32": 4, "f64": 8}[args.storage or "f16"]
    bpl = 2 * 37 * esize
    # end to end: fields from pinned host, K x (step returning the FP64 totals of its input state), fields back
    rho_h = torch.tensor(rho).pin_memory()
    u_h = torch.tensor(u).pin_memory()
    th_h = torch.tensor(th).pin_memory()
    out_r = torch.empty(n * n, dtype=torch.float64).pin_memory()
    out_u = torch.empty(2, n * n, dtype=torch.float64).pin_memory()
    out_t = torch.empty(n * n, dtype=torch.float64).pin_memory()
    e_dt, e_blk, e_drift = e2e_legs(
        sim, K,
        lambda: L.lbm_init_fields(sim.handle, rho_h.data_ptr(), u_h.data_ptr(), th_h.data_ptr(), L.LBM_DTYPE_F64, 0),
        lambda: L.lbm_moments(sim.handle, out_r.data_ptr(), out_u.data_ptr(), out_t.data_ptr(), L.LBM_DTYPE_F64, 0))
    peak, peak_kind = measured_peak_hbm()
    achieved = bpl * n * n / launch / 1e9
    hbm = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
           "traffic": None, "peak_kind": peak_kind, "algorithmic_bytes_per_launch": bpl * n * n}
    clocks = clk.summary()
    sm_mhz = clocks.get("sm_max_mhz") or 2070.0
    flops = H37_FLOPS_PER_LUP + (H37_SCALE_FLOPS if esize == 2 else 0.0)
    # the sweep issues packed FP32x2 FMAs: its peak is the packed probe's (measured in this run)
    alu_peak = measure_alu_peak("f32x2")
    alu_achieved = flops * n * n / launch / 1e12
    alu = {"bound": "alu", "achieved": alu_achieved, "peak": alu_peak, "unit": "TFLOP/s", "frac": alu_achieved / alu_peak,
           "traffic": None, "peak_kind": "measured in this run: packed FP32x2 FMA probe (lbm_alu_probe), median "
                                         "of 10 launches",
           "nominal_peak": fp32_alu_peak_tflops(sm_mhz),
           "algorithmic_flops_per_launch": flops * n * n}
    # 16-bit populations of 1024^2 stay in L2: the FP32 arithmetic binds; FP32 populations stream from HBM
    roof = dict(alu if esize == 2 else hbm)
    exact = esize == 4 and not args.fast_transforms
    roof["kernel"] = ("h37_sweep_kernel (one node per thread, correctly rounded FP32 transforms)" if exact
                      else "h37_pair_kernel (two nodes per thread, packed FP32x2)")
    roof["hbm" if esize == 2 else "alu"] = hbm if esize == 2 else alu
    line = {"metric": METRIC, "value": n * n * K / (ms * 1e-3) / 1e6, "unit": UNIT, "n_gpus": 1, "steps": K,
            "warmup": args.warmup, "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.storage or "f16", "data": "synthetic",
            "config": {"workload": "37-velocity thermal CM-MRT (Hermite N = M = 4, K = 6), %d^2 periodic, "
                                   "temperature + shear waves at mode 10, theta0 %g, Pr %g, %s offsets, FP32 "
                                   "collision%s%s" % (n, THERMAL_THETA0, THERMAL_PR, args.storage or "f16",
                                                      ", stochastic rounding of the stores" if args.sround else "",
                                                      ", correctly rounded Hermite transforms" if exact else ""),
                       "lattice": "D2Q37", "grid": [n, n], "tau_per_order": taus, "bytes_per_lup": bpl,
                       "l2": "populations %.0f MB: %s" % (37 * n * n * esize / 1e6,
                                                         "larger than L2, no flush" if 37 * n * n * esize > 129e6
                                                         else "fit in L2; each sweep still reads and writes "
                                                              "all of them once")},
            "roofline": roof,
            "e2e": {"value": n * n * K / e_dt / 1e6, "unit": UNIT, "h2d_bytes_per_step": 4 * n * n * 8 / K,
                    "d2h_bytes_per_step": 4 * n * n * 8 / K + 40, "blocking_value": n * n * K / e_blk / 1e6,
                    "mass_drift": e_drift, "definition": E2E_DEFINITION},
            "gpu_launches": 2 * K, "clocks": clocks, "status": st}
    print(json.dumps(line), flush=True)


TG2D_N, TG2D_U0, TG2D_TAUS = 4096, 0.05, [0.6, 1.0, 1.0]
# FP64 arithmetic of one D2Q9 lattice update in the one-node sweep: 53 DFMA (2 flop),
# 43 DADD and 11 DMUL, the executed counts per node (ncu, 4096^2, both parities).
D2Q9_F64_FLOPS_PER_LUP = 160.0
D2Q9_F64_INST_PER_LUP = 107.0
SWEEP_PROFILE = os.path.join(ROOT, "profiles", "tp_sweep_d2q9_f64_tg4096.md")
SWEEP_SOURCES = ("tp_sweep.cu", "sweep_body.cuh", "pair_io.cuh", "tp_common.cuh", "f32x2.cuh", "lbm_internal.cuh")
# FP64 ALU peak from unit counts: the nominal 1.25 TFLOP/s FP64 rate of the 152-SM
# part at its 2070 MHz maximum clock is 2 FMA lanes per SM x 2 flop x SMs x clock.
FP64_LANES_PER_SM = 2


def run_tg2d(args):
    """D2Q9 CM-MRT in FP64 storage and arithmetic: the 2D Taylor-Green vortex
    (u0 0.05, rho0 1, tau_2 0.6, higher orders tau 1) on a 4096^2 periodic grid,
    so that the 1.2 GB of populations stream from HBM.  One launch per step (the
    one-node sweep; FP64 takes no packed FP32x2 path)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1808_04406_gb300 import inputs
    from paper_1808_04406_gb300 import lbm as L
    torch.cuda.set_device(0)
    n = TG2D_N
    rho, u = inputs.taylor_green_2d(n, n, u0=TG2D_U0)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        sim = L.Simulation("D2Q9", (n, n), TG2D_TAUS, storage="f64", stream=stream)
        sim.init_fields(rho, u)
    sim.step(args.warmup)
    torch.cuda.synchronize()
    K = args.steps
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    with ClockSampler(0) as clk:
        for a, b in evs:
            a.record(stream)
            sim.step(1)
            b.record(stream)
        torch.cuda.synchronize()
    times = [a.elapsed_time(b) for a, b in evs]
    ms = evs[0][0].elapsed_time(evs[-1][1])
    launch = statistics.mean(times) * 1e-3
    st = sim.status()
    bpl = 2 * 9 * 8
    # end to end: fields from pinned host, K x (step returning the FP64 totals of its input state), fields back
    rho_h = torch.tensor(rho).pin_memory()
    u_h = torch.tensor(u).pin_memory()
    out_r = torch.empty(n * n, dtype=torch.float64).pin_memory()
    out_u = torch.empty(2, n * n, dtype=torch.float64).pin_memory()
    e_dt, e_blk, e_drift = e2e_legs(
        sim, K, lambda: L.lbm_init_fields(sim.handle, rho_h.data_ptr(), u_h.data_ptr(), None, L.LBM_DTYPE_F64, 0),
        lambda: L.lbm_moments(sim.handle, out_r.data_ptr(), out_u.data_ptr(), None, L.LBM_DTYPE_F64, 0))
    peak, peak_kind = measured_peak_hbm()
    achieved = bpl * n * n / launch / 1e9
    traffic = profiled_traffic(SWEEP_PROFILE, SWEEP_SOURCES)
    hbm = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
           "traffic": traffic, "peak_kind": peak_kind, "algorithmic_bytes_per_launch": bpl * n * n}
    clocks = clk.summary()
    sm_mhz = clocks.get("sm_max_mhz") or 2070.0
    sms = torch_sm_count()
    nominal = sms * FP64_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
    alu_peak = measure_alu_peak("f64")
    alu_achieved = D2Q9_F64_FLOPS_PER_LUP * n * n / launch / 1e12
    # FP64 instructions issued per second against the measured DFMA instruction rate
    issue = D2Q9_F64_INST_PER_LUP * n * n / launch / (alu_peak * 1e12 / 2)
    alu = {"bound": "alu", "achieved": alu_achieved, "peak": alu_peak, "unit": "TFLOP/s",
           "frac": alu_achieved / alu_peak, "traffic": traffic, "fp64_issue_frac": issue,
           "peak_kind": "measured in this run: FP64 FMA probe (lbm_alu_probe), median of 10 launches",
           "nominal_peak": nominal,
           "algorithmic_flops_per_launch": D2Q9_F64_FLOPS_PER_LUP * n * n}
    # the FP64 arithmetic binds long before the bandwidth on this part; both are reported
    roof = dict(alu)
    roof["kernel"] = "tp_sweep_kernel<2, double> (one node per thread)"
    roof["hbm"] = hbm
    line = {"metric": METRIC, "value": n * n * K / (ms * 1e-3) / 1e6, "unit": UNIT, "n_gpus": 1, "steps": K,
            "warmup": args.warmup, "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "D2Q9 CM-MRT FP64, %d^2 periodic Taylor-Green vortex, u0 %g, rho0 1" % (
                           n, TG2D_U0),
                       "lattice": "D2Q9", "grid": [n, n], "tau_per_order": TG2D_TAUS, "bytes_per_lup": bpl,
                       "l2": "populations %.2f GB, larger than L2, no flush" % (9 * 8 * n * n / 1e9)},
            "roofline": roof,
            "e2e": {"value": n * n * K / e_dt / 1e6, "unit": UNIT, "h2d_bytes_per_step": 3 * n * n * 8 / K,
                    "d2h_bytes_per_step": 3 * n * n * 8 / K + 40, "blocking_value": n * n * K / e_blk / 1e6,
                    "mass_drift": e_drift, "definition": E2E_DEFINITION},
            "gpu_launches": K, "clocks": clocks, "status": st}
    if not args.no_cpu_baseline:
        import oracle
        cn, csteps = 1024, 300
        crho, cu = inputs.taylor_green_2d(cn, cn, u0=TG2D_U0)
        f = oracle.tp_init(2, crho, cu)
        om = oracle.omega_from_tau(2, TG2D_TAUS)
        t0 = time.perf_counter()
        oracle.tp_step(2, (cn, cn), om, f, csteps)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": cn * cn * csteps / dt / 1e6, "unit": UNIT, "cores": oracle.num_threads(),
                                "kind": "oracle",
                                "sample": "D2Q9 Taylor-Green %d^2, %d steps, FP64 oracle, %.1f s" % (cn, csteps, dt)}
    print(json.dumps(line), flush=True)


PAPER_MAX_MA = 0.2688  # thermal CM-MRT, Pr 1, Re 1e7, 128^2 double shear layer to t/t_c = 2


def run_stability(args):
    """Stability boundaries of the double shear layer (Sec. III.C): the largest Ma
    that survives to t/t_c = 2 on a 128^2 grid, by k-ary search (7 candidates per
    round, 4 rounds: bracket width 1/8^4 of the initial interval), for the
    37-velocity thermal and isothermal CM-MRT and raw-moment MRT at Pr 0.1, 1, 10
    (concurrent simulations) and D2Q9 CM-MRT and BGK (one batch per round).  A
    bracket [0.02, 0.0204] means no candidate survived."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1808_04406_gb300 import stability as S
    from paper_1808_04406_gb300 import lbm as L
    torch.cuda.set_device(0)
    n = 128
    res = [1e4, 1e5, 1e6, 1e7]
    table = {}
    t0 = time.time()
    with ClockSampler(0) as clk:
        for name, thermal, flags in (("thermal CM-MRT", True, 0), ("isothermal CM-MRT", False, 0),
                                     ("isothermal raw-moment MRT", False, L.LBM_RAW_MRT)):
            for pr in (0.1, 1.0, 10.0):
                rows = {}
                for re in res:
                    lo, hi = S.kary_search(S.h37_runner(n, re, pr, thermal, storage=args.storage or "f32",
                                                        flags=flags), 0.02, 1.2, k=7, rounds=4)
                    rows["%g" % re] = [lo, hi]
                table["D2Q37 %s, Pr %g" % (name, pr)] = rows
        for name, higher in (("D2Q9 CM-MRT (orders 3, 4 at tau 1)", None), ("D2Q9 CM-MRT (tau_3 1, tau_4 tau_2)", "t4"),
                             ("D2Q9 BGK", "bgk")):
            out = S.kary_search_many(S.d2q9_batch_runner(n, res, storage=args.storage or "f32", higher=higher),
                                     len(res), 0.02, 1.6, k=7, rounds=4)
            table[name] = {"%g" % re: list(b) for re, b in zip(res, out)}
    wall = time.time() - t0
    value = table["D2Q37 thermal CM-MRT, Pr 1"]["1e+07"][0]
    line = {"metric": METRIC, "value": value, "unit": "max Ma (double shear layer survives to t/t_c = 2, 128^2)",
            "n_gpus": 1, "steps": None, "warmup": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": value / PAPER_MAX_MA, "dtype": args.storage or "f32", "data": "synthetic",
            "config": {"workload": "double shear layer (rho 80, delta 0.05) on 128^2, thermal CM-MRT, Pr 1, "
                                   "Re 1e7 (value); tables for Re 1e4..1e7 and five models; tau_4 = tau_2",
                       "paper_value": PAPER_MAX_MA},
            "result": {"brackets": table, "wall_s": wall}, "gpu_launches": None, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def run_convergence(args):
    """Fig. 2: relative errors of nu and kappa on the eight minimal rules for
    L = 20 .. 320 (FP64, on-device decay fits).  `value` = the smallest observed
    order of accuracy between L = 160 and 320 over all rules and both
    coefficients (2 for a second-order scheme)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1808_04406_gb300 import convergence as C
    torch.cuda.set_device(0)
    t0 = time.time()
    with ClockSampler(0) as clk:
        res = C.study()
    wall = time.time() - t0
    orders = [r[k + "_order"][-1] for r in res.values() for k in ("viscous", "thermal")]
    line = {"metric": METRIC, "value": min(orders), "unit": "observed order of accuracy (L 160 -> 320)",
            "n_gpus": 1, "steps": None, "warmup": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "grid convergence of nu and kappa, shear and isobaric temperature waves of "
                                   "mode 1 on L x L, L = 20..320, the four 17-velocity (N = 3) and four "
                                   "37-velocity (N = 4) minimal rules, nu 0.1, kappa 0.2, theta0 1",
                       "sizes": list(C.SIZES)},
            "result": {"errors": res, "wall_s": wall}, "gpu_launches": None, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def run_closure(args):
    """Learned versus plain at equal kinetic-energy-spectrum error (not a steps
    loop): train the closure on box-filtered 512^3 runs of one seed, then run the
    other seed at 128^3 plain, 128^3 learned and 256^3 plain and compare each
    spectrum with the 512^3 run's over every shell the 128^3 grid resolves."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1808_04406_gb300 import closure as C
    torch.cuda.set_device(0)
    with ClockSampler(0) as clk:
        out = C.experiment(n_fine=4 * LEARNED_N, m=4, k0=LEARNED_K0, u_rms=LEARNED_URMS, re_lambda=LEARNED_RE,
                           ranges=((0.0, 2.0), LEARNED_RANGE), log=lambda *a: None)
    stable = [r for r in out["learned"] if r.get("spectrum_error") is not None]
    best = min(stable, key=lambda r: r["spectrum_error"]) if stable else None
    for r in out["learned"]:
        r.pop("E", None)
    for k in ("plain_coarse", "plain_medium"):
        out[k].pop("E", None)
    out.pop("E_ref", None)
    line = {"metric": METRIC, "value": best.get("time_ratio_at_equal_error") if best else None,
            "unit": "plain GPU time / learned GPU time at equal KE-spectrum error", "n_gpus": 1, "steps": None,
            "warmup": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+bf16",
            "data": "synthetic",
            "config": {"workload": "learned closure, D3Q27 decaying isotropic turbulence: train on 4^3 box-filtered "
                                   "512^3 FP32 runs (seed 1), evaluate seed 0 at 128^3 (plain, learned) and 256^3 "
                                   "(plain) against the 512^3 run; k0 4, u_rms 0.04, Re_lambda 100"},
            "result": out, "gpu_launches": None, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_SIDE)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-secondary", action="store_true",
                    help="tgv256 FP32 default: skip the other configurations measured in child processes")
    ap.add_argument("--workload", default="tgv256",
                    choices=["tgv256", "batch512", "learned128", "closure", "thermal1024", "stability",
                             "convergence", "tg4096", "alu_peak"])
    ap.add_argument("--storage", default=None,
                    help="tgv256: f32 (default), f16, bf16; thermal1024: f16 (default), bf16, f32")
    ap.add_argument("--sround", action="store_true", help="thermal1024 only: stochastic rounding of FP16/BF16")
    ap.add_argument("--fast-transforms", action="store_true",
                    help="thermal1024 with FP32 storage: plain FP32 Hermite transforms and the two-node sweep "
                         "instead of the correctly rounded transforms")
    ap.add_argument("--decomp", default="replicas", choices=["replicas", "slab"],
                    help="tgv256 with --gpus N > 1: N independent replicas (default) or one grid of n x n x nN "
                         "planes split into slabs with a halo exchange per odd step")
    ap.add_argument("--runs", type=int, default=512)
    ap.add_argument("--batch-launch", type=int, default=None,
                    help="batch512 only: fixed launch mode instead of the autotuner (0: tile sweep, "
                         "k >= 1: shared-memory band sweep of shape k)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "batch512":
        if rank == 0:
            run_batch(args)
        return
    if args.workload == "closure":
        if rank == 0:
            run_closure(args)
        return
    if args.workload == "thermal1024":
        if rank == 0:
            run_thermal(args)
        return
    if args.workload == "stability":
        if rank == 0:
            run_stability(args)
        return
    if args.workload == "tg4096":
        if rank == 0:
            run_tg2d(args)
        return
    if args.workload == "convergence":
        if rank == 0:
            run_convergence(args)
        return
    if args.workload == "alu_peak":
        if rank == 0:
            run_alu_peak(args)
        return
    dist = None
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        tdist.init_process_group("nccl")
        dist = tdist
    try:
        run_gpu(args, rank, world, dist)
    finally:
        if dist is not None:
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
