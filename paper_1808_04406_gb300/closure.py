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


def filtered_states(fine, m, steps_between, count):
    """Filter the fine simulation now and after every `steps_between` fine steps:
    returns a list of `count` coarse offset tensors [27, Nc] (device, FP32)."""
    torch = fine.torch
    nc = [d // m for d in fine.dims]
    out = []
    for k in range(count):
        if k:
            fine.step(steps_between)
        buf = torch.empty(27, int(np.prod(nc)), dtype=torch.float32, device=fine.device)
        L.lbm_closure_filter(fine.handle, m, buf.data_ptr())
        out.append(buf)
    torch.cuda.synchronize(fine.device)
    return out, tuple(nc)


def build_dataset(states, dims_c, tau2, norm=None, sample=65536, seed=0):
    """(features, targets) from consecutive coarse states; the standardisation
    (mean, 1/std per feature) is estimated on a random subsample unless given."""
    import torch
    dev = states[0].device
    Nc = int(np.prod(dims_c))
    ident = torch.zeros(2 * N_IN, dtype=torch.float32, device=dev)
    ident[N_IN:] = 1.0
    Xs, As = [], []
    for a, b in zip(states[:-1], states[1:]):
        X = torch.empty(Nc, N_IN, dtype=torch.float32, device=dev)
        abc = torch.empty(Nc, 18, dtype=torch.float32, device=dev)
        L.lbm_closure_dataset(dims_c, a.data_ptr(), b.data_ptr(), tau2, ident.data_ptr(), X.data_ptr(), abc.data_ptr(),
                              torch.cuda.current_stream(dev).cuda_stream)
        Xs.append(X)
        As.append(abc)
    X = torch.cat(Xs)
    abc = torch.cat(As)
    if norm is None:
        rng = np.random.default_rng(seed)
        idx = rng.integers(0, X.shape[0], min(sample, X.shape[0]))
        xs = X[torch.as_tensor(idx, device=dev)].double().cpu().numpy()
        mean = xs.mean(0)
        std = xs.std(0)
        mean[19] = 0.0  # tau_2 - 1/2 is one constant per run: keep it as it is
        std[19] = 1.0
        norm = np.concatenate([mean, 1.0 / np.where(std > 0, std, 1.0)]).astype(np.float32)
    nt = torch.as_tensor(norm, device=dev)
    X = (X - nt[:N_IN]) * nt[N_IN:]
    return Dataset(X.contiguous(), abc.contiguous(), nt)


def class_weights(ds):
    """Per-class loss weights 1 / mean(A): every class contributes on one scale."""
    A = ds.abc[:, 0::3].double().mean(0).cpu().numpy()
    return (1.0 / np.where(A > 0, A, 1.0)).astype(np.float32)


def train(ds, params, iters, batch=8192, lr=2e-3, seed=0, cw=None):
    """Adam on the device; returns the per-iteration mini-batch losses (numpy)."""
    import torch
    dev = ds.X.device
    cw = class_weights(ds) if cw is None else cw
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    losses = torch.zeros(max(1, iters), dtype=torch.float32, device=dev)
    wb = L.lbm_mlp_work_bytes(batch)
    work = torch.empty(wb, dtype=torch.uint8, device=dev)
    L.lbm_mlp_train(ds.X.data_ptr(), ds.abc.data_ptr(), ds.n, cw, params.data_ptr(), m.data_ptr(), v.data_ptr(),
                    iters, batch, lr, seed, 0, losses.data_ptr(), work.data_ptr(), wb,
                    torch.cuda.current_stream(dev).cuda_stream)
    torch.cuda.synchronize(dev)
    return losses.cpu().numpy()[:iters]


def loss_and_grad(ds, params, cw):
    import torch
    dev = ds.X.device
    wb = L.lbm_mlp_work_bytes(ds.n)
    work = torch.empty(wb, dtype=torch.uint8, device=dev)
    grad = torch.empty_like(params)
    loss = L.lbm_mlp_loss_grad(ds.X.data_ptr(), ds.abc.data_ptr(), ds.n, cw, params.data_ptr(), grad.data_ptr(),
                               work.data_ptr(), wb, torch.cuda.current_stream(dev).cuda_stream)
    return loss, grad
