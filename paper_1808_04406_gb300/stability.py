"""Maximum stable Mach number of the double shear layer (the stability
boundaries of the paper's Sec. III.C).

For a fixed Re (and Pr), a run "survives" when it reaches t / t_c = 2 with no
node flagged unphysical (the sweep's status word: rho <= 0, theta <= 0, a
non-finite value or a runaway speed), t_c = L / u0 in lattice steps.  The
largest surviving Ma is found by a k-ary search: every round evaluates k Mach
numbers spread over the current bracket at once, on the GPU, and keeps the
sub-interval between the last survivor and the first failure.

Runners (all computation in the library's kernels):
  * 37-velocity lattice: k independent simulations on their own CUDA streams,
    stepped in chunks and dropped as soon as they diverge or reach their time;
  * D2Q9: one batched launch per step over every candidate (and every Re).
Units follow the paper: Hermite units with c_s = 1 on the 37-velocity lattice,
Re = u0 c L / nu and Ma = u0 (lattice speed u0 / c); on D2Q9, Ma = u / c_s with
c_s^2 = 1/3 in lattice units and Re = u L / nu.
"""
import math

import numpy as np

from . import inputs


def kary_search(survive, lo, hi, k=7, rounds=4):
    """survive(list of Ma) -> list of bool.  Survival is taken as monotone in Ma:
    the first failure (in increasing Ma) closes the bracket.  Returns (lo, hi)
    with lo the largest Ma seen to survive (or the initial lo) and hi the
    smallest seen to fail (or the initial hi)."""
    for _ in range(rounds):
        cand = [lo + (hi - lo) * (i + 1) / (k + 1) for i in range(k)]
        ok = list(survive(cand))
        first_fail = next((i for i, s in enumerate(ok) if not s), None)
        if first_fail is None:
            lo = cand[-1]
        else:
            hi = cand[first_fail]
            if first_fail > 0:
                lo = cand[first_fail - 1]
    return lo, hi


def h37_params(L, ma, re, pr, thermal, theta0=1.0, tau4=None):
    """(taus, steps, lattice velocity) for one 37-velocity DSL run."""
    from .gen_d2q37 import lattice_scale
    c = lattice_scale()
    nu = ma * c * L / re  # Hermite units
    kap = nu / pr
    t2 = 0.5 + nu / theta0
    t3 = 0.5 + kap / theta0
    taus = [t2, t3, t2 if tau4 is None else tau4]
    u_lat = ma / c
    steps = int(math.ceil(2.0 * L / u_lat))
    return taus, steps, u_lat


def h37_runner(L, re, pr, thermal, storage="f32", chunk=256, device=None, flags=0, tau4=None):
    """survive(list of Ma) for the 37-velocity lattice: concurrent simulations."""
    import torch
    from . import lbm as Lb

    def survive(mas):
        sims = []
        for ma in mas:
            taus, steps, u_lat = h37_params(L, ma, re, pr, thermal, tau4=tau4)
            rho, u = inputs.double_shear_layer(L, u_lat)
            st = torch.cuda.Stream(device=device)
            f = flags | (Lb.LBM_THERMAL if thermal else 0)
            sim = Lb.Simulation("D2Q37", (L, L), taus, storage=storage, flags=f, theta_ref=1.0, stream=st,
                                device=device)
            sim.init_fields(rho, u, np.ones(L * L))
            sims.append([sim, steps, None])
        active = list(range(len(sims)))
        while active:
            for i in active:
                sim, steps, _ = sims[i]
                sim.step(min(chunk, steps - sim.step_count))
            still = []
            for i in active:
                sim, steps, _ = sims[i]
                if sim.status() != 0:
                    sims[i][2] = False
                elif sim.step_count >= steps:
                    sims[i][2] = True
                else:
                    still.append(i)
            active = still
        out = [s[2] for s in sims]
        for s in sims:
            s[0].close()
        return out

    return survive


def d2q9_params(L, ma, re, higher=None):
    u_lat = ma / math.sqrt(3.0)
    nu = u_lat * L / re
    t2 = 0.5 + 3.0 * nu
    taus = [t2] + (list(higher) if higher is not None else [1.0, 1.0])
    return taus, int(math.ceil(2.0 * L / u_lat)), u_lat


def d2q9_batch_runner(L, res, storage="f32", chunk=256, higher=None):
    """survive for several Re at once on D2Q9: returns f(list of Ma per Re) ->
    list of list of bool, every (Re, Ma) pair one run of a single batch.
    higher: relaxation times of orders 3 and 4 (default 1), "bgk" (both tau_2) or
    "t4" (tau_3 = 1, tau_4 = tau_2)."""
    from . import lbm as Lb

    def survive_all(mas_per_re):
        dims, taus, steps, fields = [], [], [], []
        for re, mas in zip(res, mas_per_re):
            for ma in mas:
                t, s, u_lat = d2q9_params(L, ma, re)
                if higher == "bgk":
                    t = [t[0], t[0], t[0]]
                elif higher == "t4":
                    t = [t[0], 1.0, t[0]]
                elif higher is not None:
                    t = [t[0]] + list(higher)
                dims.append((L, L))
                taus.append(t)
                steps.append(s)
                fields.append(inputs.double_shear_layer(L, u_lat))
        b = Lb.Batch(dims, taus, storage=storage)
        for r, (rho, u) in enumerate(fields):
            b.init_run(r, rho, u)
        need = np.array(steps)
        alive_at = np.zeros(len(dims), dtype=bool)
        done = np.zeros(len(dims), dtype=bool)
        t = 0
        while not done.all():
            todo = int(min(chunk, need[~done].max() - t))
            b.step(todo)
            t += todo
            st = b.status()
            newly = (~done) & ((st != 0) | (t >= need))
            alive_at[newly] = (st[newly] == 0)
            done |= newly
        b.close()
        out, k = [], 0
        for mas in mas_per_re:
            out.append([bool(alive_at[k + i]) for i in range(len(mas))])
            k += len(mas)
        return out

    return survive_all


def kary_search_many(survive_all, n, lo, hi, k=7, rounds=4):
    """kary_search for n independent problems evaluated together:
    survive_all(list of n candidate lists) -> list of n bool lists."""
    los, his = [lo] * n, [hi] * n
    for _ in range(rounds):
        cands = [[los[j] + (his[j] - los[j]) * (i + 1) / (k + 1) for i in range(k)] for j in range(n)]
        oks = survive_all(cands)
        for j in range(n):
            ff = next((i for i, s in enumerate(oks[j]) if not s), None)
            if ff is None:
                los[j] = cands[j][-1]
            else:
                his[j] = cands[j][ff]
                if ff > 0:
                    los[j] = cands[j][ff - 1]
    return list(zip(los, his))
