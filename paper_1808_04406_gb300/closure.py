"""Orchestration of the learned relaxation-rate closure (D3Q27, FP32 storage).

Host-side glue only: every computation runs in the library's kernels (box
filter, dataset, BF16 tensor-core training step, Adam, fused inference in the
sweep).  PyTorch provides device buffers and the stream.

Pipeline: run a fine simulation, box-filter its populations every ``m`` fine
steps (one coarse step in acoustic scaling), turn consecutive filtered states
into (features, targets), standardise the features, train the 20-64-64-6
network, and hand it to a coarse simulation with ``Simulation.set_closure``.
"""
import numpy as np

from . import lbm as L

N_IN = 20


class Dataset:
    """Device tensors X [n, 20] (standardised features) and abc [n, 18]."""

    def __init__(self, X, abc, norm):
        self.X, self.abc, self.norm = X, abc, norm

    @property
    def n(self):
        return int(self.X.shape[0])


def collect_pairs(fine, m, tau2_coarse, n_pairs, gap, neq_scale=1.0):
    """Training samples from a running fine simulation: at n_pairs times `gap`
    fine steps apart, box-filter the state, advance m fine steps (one coarse step
    in acoustic scaling), filter again, scale both coarse states' non-equilibrium
    by neq_scale (m tau_c / tau_f makes them coarse-model states), and turn them
    into (features, class sums) on the device.  Returns un-standardised X [n, 20]
    and abc [n, 18] (device FP32)."""
    import torch
    dev = fine.device
    nc = tuple(d // m for d in fine.dims)
    Nc = int(np.prod(nc))
    ident = torch.zeros(2 * N_IN, dtype=torch.float32, device=dev)
    ident[N_IN:] = 1.0
    X = torch.empty(n_pairs * Nc, N_IN, dtype=torch.float32, device=dev)
    abc = torch.empty(n_pairs * Nc, 18, dtype=torch.float32, device=dev)
    a = torch.empty(27, Nc, dtype=torch.float32, device=dev)
    b = torch.empty_like(a)
    st = fine.stream.cuda_stream
    for k in range(n_pairs):
        if k:
            fine.step(gap - m)
        L.lbm_closure_filter(fine.handle, m, a.data_ptr())
        fine.step(m)
        L.lbm_closure_filter(fine.handle, m, b.data_ptr())
        if neq_scale != 1.0:
            L.lbm_closure_rescale(nc, a.data_ptr(), neq_scale, st)
            L.lbm_closure_rescale(nc, b.data_ptr(), neq_scale, st)
        L.lbm_closure_dataset(nc, a.data_ptr(), b.data_ptr(), tau2_coarse, ident.data_ptr(),
                              X[k * Nc:(k + 1) * Nc].data_ptr(), abc[k * Nc:(k + 1) * Nc].data_ptr(), st)
    torch.cuda.synchronize(dev)
    return X, abc


def standardise(X, norm=None, sample=1 << 20, seed=0):
    """Feature mean and 1/std (estimated on a random subsample) unless given;
    tau_2 - 1/2 (one constant per run) is left as it is.  Returns (X_std, norm)."""
    import torch
    dev = X.device
    if norm is None:
        g = torch.Generator(device="cpu").manual_seed(seed)
        idx = torch.randint(0, X.shape[0], (min(sample, X.shape[0]),), generator=g).to(dev)
        xs = X[idx].double()
        mean = xs.mean(0)
        std = xs.std(0)
        mean[19] = 0.0
        std[19] = 1.0
        norm = torch.cat([mean, 1.0 / torch.where(std > 0, std, torch.ones_like(std))]).float()
    norm = torch.as_tensor(norm, dtype=torch.float32, device=dev)
    return ((X - norm[:N_IN]) * norm[N_IN:]).contiguous(), norm


def class_weights(abc):
    """Per-class loss weights 1 / mean(A): every class contributes on one scale."""
    A = abc[:, 0::3].double().mean(0).cpu().numpy()
    return (1.0 / np.where(A > 0, A, 1.0)).astype(np.float32)


class Trainer:
    """Adam state on the device; train() may be called repeatedly (learning-rate
    schedule by segments)."""

    def __init__(self, params, batch=65536):
        import torch
        self.params = params
        self.m = torch.zeros_like(params)
        self.v = torch.zeros_like(params)
        self.t = 0
        self.batch = batch
        self.wb = L.lbm_mlp_work_bytes(batch)
        self.work = torch.empty(self.wb, dtype=torch.uint8, device=params.device)

    def train(self, X, abc, cw, iters, lr, seed=0, omega_lo=0.0, omega_hi=2.0):
        import torch
        dev = X.device
        losses = torch.zeros(max(1, iters), dtype=torch.float32, device=dev)
        L.lbm_mlp_train(X.data_ptr(), abc.data_ptr(), X.shape[0], cw, self.params.data_ptr(), self.m.data_ptr(),
                        self.v.data_ptr(), iters, self.batch, lr, seed, self.t, losses.data_ptr(),
                        self.work.data_ptr(), self.wb, torch.cuda.current_stream(dev).cuda_stream, omega_lo, omega_hi)
        self.t += iters
        torch.cuda.synchronize(dev)
        return losses.cpu().numpy()[:iters]


def train(ds, params, iters, batch=8192, lr=2e-3, seed=0, cw=None):
    """Adam on the device for a Dataset; returns the per-iteration mini-batch losses."""
    cw = class_weights(ds.abc) if cw is None else cw
    return Trainer(params, batch).train(ds.X, ds.abc, cw, iters, lr, seed)


def loss_and_grad(X, abc, params, cw, omega_lo=0.0, omega_hi=2.0):
    import torch
    dev = X.device
    wb = L.lbm_mlp_work_bytes(X.shape[0])
    work = torch.empty(wb, dtype=torch.uint8, device=dev)
    grad = torch.empty_like(params)
    loss = L.lbm_mlp_loss_grad(X.data_ptr(), abc.data_ptr(), X.shape[0], cw, params.data_ptr(), grad.data_ptr(),
                               work.data_ptr(), wb, torch.cuda.current_stream(dev).cuda_stream, omega_lo, omega_hi)
    return loss, grad


def constant_rate_loss(abc, cw, omega):
    """The a-priori loss of fixed class rates omega[6] (the plain model) on the same samples."""
    import torch
    g = 1.0 - torch.as_tensor(np.asarray(omega, dtype=np.float64), device=abc.device)
    A, B, C = (abc[:, c::3].double() for c in range(3))
    per = g * g * A - 2 * g * B + C
    return float((per * torch.as_tensor(np.asarray(cw, dtype=np.float64), device=abc.device)).sum(1).mean())


def init_params(seed, device):
    """He-style random weights, zero biases (seeded), as one FP32 device vector
    W1[20][64], b1[64], W2[64][64], b2[64], W3[64][6], b3[6]."""
    import torch
    rng = np.random.default_rng(seed)
    parts = [rng.normal(0, np.sqrt(2.0 / N_IN), N_IN * 64), np.zeros(64), rng.normal(0, np.sqrt(2.0 / 64), 64 * 64),
             np.zeros(64), rng.normal(0, np.sqrt(1.0 / 64), 64 * 6), np.zeros(6)]
    return torch.as_tensor(np.concatenate(parts), dtype=torch.float32, device=device)


def rate_classes_of_orders(omega_per_order):
    """Class rates (3:(2,1,0), 3:(1,1,1), 4:(2,2,0), 4:(2,1,1), 5, 6) of a plain model
    with omega[n] per order n."""
    o = omega_per_order
    return [o[3], o[3], o[4], o[4], o[5], o[6]]


# ---- a-posteriori evaluation: kinetic-energy spectra -----------------------------

def velocity(sim):
    """Velocity field of a cubic simulation (host FP64, [3, n, n, n], index order [z, y, x])."""
    _, u = sim.moments(dtype="f32")
    n = sim.dims[0]
    return u.astype(np.float64).reshape(3, n, n, n)


def filtered_velocity(sim, m):
    """Velocity of the box-filtered populations on the (n/m)^3 grid (host FP64,
    [3, nc, nc, nc] with index order [z, y, x])."""
    import torch
    nc = [d // m for d in sim.dims]
    buf = torch.empty(27, int(np.prod(nc)), dtype=torch.float32, device=sim.device)
    L.lbm_closure_filter(sim.handle, m, buf.data_ptr())
    torch.cuda.synchronize(sim.device)
    off = buf.double().cpu().numpy()
    i = np.arange(27)
    e = np.stack([(i % 3) - 1, (i // 3) % 3 - 1, (i // 9) % 3 - 1]).astype(np.float64)  # [3, 27]
    rho = 1.0 + off.sum(0)  # sum_i w_i = 1, sum_i w_i e_i = 0
    u = (e @ off) / rho
    return u.reshape(3, nc[2], nc[1], nc[0])


def ke_spectrum(u):
    """Shell-summed kinetic-energy spectrum E(k), k = 0 .. n/2 (integer shells of
    |k| rounded), of a periodic velocity field u[3, n, n, n]."""
    import scipy.fft as sf
    n = u.shape[-1]
    k = np.fft.fftfreq(n, 1.0 / n)
    kr = np.fft.rfftfreq(n, 1.0 / n)
    KZ, KY, KX = np.meshgrid(k, k, kr, indexing="ij")
    shell = np.rint(np.sqrt(KX ** 2 + KY ** 2 + KZ ** 2)).astype(np.int64)
    wgt = np.where(KX == 0, 1.0, 2.0)  # rfft halves the spectrum
    wgt[..., -1] = np.where(n % 2 == 0, 1.0, 2.0)
    E = np.zeros(n // 2 + 1)
    for d in range(3):
        uh = sf.rfftn(u[d], workers=-1) / u[d].size
        p = 0.5 * wgt * (uh.real ** 2 + uh.imag ** 2)
        E += np.bincount(shell.reshape(-1), p.reshape(-1), minlength=shell.max() + 1)[:n // 2 + 1]
    return E


def spectrum_error(E, E_ref, kmax):
    """RMS of ln E - ln E_ref over shells 1 .. kmax."""
    k = np.arange(1, kmax + 1)
    return float(np.sqrt(np.mean((np.log(E[k]) - np.log(E_ref[k])) ** 2)))


def taylor_scale_viscosity(n, k0, u_rms, re_lambda):
    """nu (lattice units) giving Re_lambda = u' lambda / nu for the k^4 exp(-2 (k/k0)^2)
    spectrum, whose Taylor microscale is lambda = 2 / k0 box units (the box is 2 pi)."""
    lam = (2.0 / k0) * n / (2.0 * np.pi)
    return u_rms * lam / re_lambda


def timed_steps(sim, n):
    """GPU time (ms, CUDA events on the simulation's stream) of n steps."""
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(sim.stream)
    sim.step(n)
    e1.record(sim.stream)
    e1.synchronize()
    return e0.elapsed_time(e1)


# ---- the learned-versus-plain experiment ----------------------------------------

def experiment(n_fine=512, m=4, k0=4.0, u_rms=0.04, re_lambda=100.0, t_eval=2048, n_pairs=16, gap=128,
               schedule=((1500, 2e-3), (1000, 6e-4), (500, 2e-4)), batch=65536, seed_train=1, seed_eval=0,
               ranges=((0.0, 2.0),), higher_taus=None, rescale=True, log=print):
    """Train the closure on box-filtered fine runs (seed_train) and compare, at
    fine time t_eval and on seed_eval, the kinetic-energy spectra of the learned
    coarse runs (one per rate range), of the plain coarse run and of the plain
    run at twice the coarse resolution with that of the fine run, over every
    shell the coarse grid resolves.  Acoustic scaling: a grid n uses
    nu_n = nu_fine n / n_fine and t_eval n / n_fine steps; every run starts from
    the same band-limited field.  Returns a dict of errors, GPU times and losses."""
    import time
    import torch
    from . import inputs
    from .lbm import Simulation
    dev = torch.device("cuda")
    nc = n_fine // m
    nu_f = taylor_scale_viscosity(n_fine, k0, u_rms, re_lambda)
    hi_t = list(higher_taus) if higher_taus is not None else None

    def taus(n):
        t2 = 0.5 + 3.0 * nu_f * n / n_fine
        return [t2] + (hi_t if hi_t is not None else [1.0, t2, 1.0, t2])

    def fresh(n, seed):
        rho, u = inputs.isotropic_turbulence_3d(n, seed, k0=k0, u_rms=u_rms)
        sim = Simulation("D3Q27", (n, n, n), taus(n))
        sim.init_fields(rho, u)
        return sim

    def free(sim):
        sim.close()
        torch.cuda.empty_cache()

    tc, tf = taus(nc)[0], taus(n_fine)[0]
    s_neq = m * tc / tf if rescale else 1.0
    plain_cls = rate_classes_of_orders([0.0, 0.0] + [1.0 / x for x in taus(nc)])
    out = {"n_fine": n_fine, "n_coarse": nc, "m": m, "k0": k0, "u_rms": u_rms, "re_lambda": re_lambda,
           "nu_fine": nu_f, "tau2_fine": tf, "tau2_coarse": tc, "higher_taus": taus(nc)[1:],
           "neq_scale": s_neq, "t_eval_fine_steps": t_eval}
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # 1. training data from a fine run
    t0 = time.time()
    fine = fresh(n_fine, seed_train)
    log("fine %d^3 seed %d ready (%.1f s host)" % (n_fine, seed_train, time.time() - t0))
    ev0.record(fine.stream)
    Xr, abc = collect_pairs(fine, m, tc, n_pairs, gap, s_neq)
    ev1.record(fine.stream)
    ev1.synchronize()
    out["data_gpu_ms"] = ev0.elapsed_time(ev1)
    out["n_samples"] = int(Xr.shape[0])
    free(fine)
    X, norm = standardise(Xr)
    del Xr
    cw = class_weights(abc)
    A = abc[:, 0::3].double().sum(0)
    B = abc[:, 1::3].double().sum(0)
    out["apriori_best_constant_rates"] = (1.0 - B / A).cpu().numpy().tolist()
    # 2. held-out samples and the reference spectrum from the fine run of seed_eval
    fine = fresh(n_fine, seed_eval)
    n_test = 4
    tgap = t_eval // n_test
    ev0.record(fine.stream)
    Xt, abct = collect_pairs(fine, m, tc, n_test, tgap, s_neq)
    fine.step(t_eval - ((n_test - 1) * tgap + m))
    ev1.record(fine.stream)
    ev1.synchronize()
    out["fine_gpu_ms"] = ev0.elapsed_time(ev1)
    E_ref = ke_spectrum(velocity(fine))
    out["fine_status"] = fine.status()
    free(fine)
    Xt, _ = standardise(Xt, norm)
    out["apriori_loss_plain_test"] = constant_rate_loss(abct, cw, plain_cls)
    kmax = nc // 2 - 1
    out["spectrum_kmax"] = kmax
    out["E_ref"] = E_ref[:nc // 2 + 1].tolist()

    def evaluate(name, n, params=None, lo=0.0, hi=2.0):
        warm = Simulation("D3Q27", (n, n, 8), taus(n))  # the same kernels, warmed on a rest state
        warm.init_fields(np.ones(n * n * 8), np.zeros((3, n * n * 8)))
        if params is not None:
            warm.set_closure(params, norm, lo, hi)
        warm.step(4)
        free(warm)
        steps = t_eval * n // n_fine
        sim = fresh(n, seed_eval)
        if params is not None:
            sim.set_closure(params, norm, lo, hi)
        ms = timed_steps(sim, steps)
        st = sim.status()
        r = {"n": n, "steps": steps, "gpu_ms": ms, "status": st}
        if st == 0:
            E = ke_spectrum(velocity(sim))
            r["spectrum_error"] = spectrum_error(E, E_ref, kmax)
            r["spectrum_error_k_le_%d" % (nc // 4)] = spectrum_error(E, E_ref, nc // 4)
            r["E"] = E[:nc // 2 + 1].tolist()
        else:
            r["spectrum_error"] = None
        free(sim)
        log("%s %d^3: %.1f ms, status %d, error %s" % (name, n, ms, st, r["spectrum_error"]))
        out[name] = r
        return r

    pc = evaluate("plain_coarse", nc)
    pm = evaluate("plain_medium", 2 * nc) if 2 * nc < n_fine else None
    # 3. one network per rate range: train, a-priori test loss, a-posteriori run
    out["learned"] = []
    for lo, hi in ranges:
        params = init_params(seed_train, dev)
        tr = Trainer(params, batch)
        ev0.record()
        losses = np.concatenate([tr.train(X, abc, cw, it, lr, seed_train, lo, hi) for it, lr in schedule])
        ev1.record()
        ev1.synchronize()
        rec = {"omega_lo": lo, "omega_hi": hi, "train_gpu_ms": ev0.elapsed_time(ev1), "train_iters": int(losses.size),
               "train_loss_first": float(losses[:50].mean()), "train_loss_last": float(losses[-50:].mean()),
               "apriori_loss_test": loss_and_grad(Xt, abct, params, cw, lo, hi)[0]}
        rec["apriori_gain"] = out["apriori_loss_plain_test"] / rec["apriori_loss_test"]
        r = evaluate("learned_%g_%g" % (lo, hi), nc, params, lo, hi)
        rec.update({k: v for k, v in r.items() if k != "E"})
        rec["E"] = r.get("E")
        out.pop("learned_%g_%g" % (lo, hi))
        if pm and pc["spectrum_error"] and pm["spectrum_error"] and rec["spectrum_error"]:
            x = np.log([pm["spectrum_error"], pc["spectrum_error"]])
            y = np.log([pm["gpu_ms"], pc["gpu_ms"]])
            xl = np.log(rec["spectrum_error"])
            slope = (y[1] - y[0]) / (x[1] - x[0]) if x[1] != x[0] else 0.0
            t_eq = float(np.exp(y[0] + slope * (xl - x[0])))
            rec["plain_gpu_ms_at_equal_error"] = t_eq
            rec["time_ratio_at_equal_error"] = t_eq / rec["gpu_ms"]
            rec["equal_error_interpolated"] = bool(min(x) <= xl <= max(x))
        out["learned"].append(rec)
        log("range [%g, %g]: loss %.4g -> %.4g, a-priori gain %.3f" % (lo, hi, rec["train_loss_first"],
                                                                       rec["train_loss_last"], rec["apriori_gain"]))
    return out
