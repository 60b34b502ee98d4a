"""Grid convergence of the CM-MRT transport coefficients on the minimal
quadrature rules (Sec. III.A, Fig. 2).

For each rule and lattice size L, a shear wave and an isobaric temperature wave
of mode 1 (k = 2 pi / L) decay on an L x L periodic grid.  The decay rate per
step is D k^2 / c^2 for a diffusivity D in Hermite units (xi = c e), so
D = rate c^2 / k^2.  The shear rate is the on-device FP64 fit of u_y's mode;
the thermal rate is fitted to the mode of dtheta / theta0 - drho / rho0, which
carries no part of the sound modes the initial state also excites.  The
relative errors against nu = theta0 (tau_2 - 1/2) and kappa = theta0 (tau_3 - 1/2)
(Chapman-Enskog, Sec. II.C) are the quantities of Fig. 2.  Parameters:
nu = 0.1, kappa = 0.2 (Pr = 0.5) as in Fig. 1, rho0 = 1, amplitude 1e-3,
tau_4 = tau_2, and theta0 = 1: with the expansion truncated at N = M = 3 the
17-velocity rules conduct heat at kappa / theta0^2 (measured -30.5 % at
theta0 = 1.2, second-order convergent at theta0 = 1), so they model heat
conduction about the reference temperature only.
"""
import numpy as np

from . import gen_rules, inputs

RULES = ("E7-A", "E7-B", "E7-C", "E7-D", "E9-A", "E9-B", "E9-C", "E9-D")
SIZES = (20, 40, 80, 160, 320)


def relative_error(name, L, kind, nu=0.1, kappa=0.2, theta0=1.0, amp=1e-3, storage="f64", n_rec=40):
    """Measured / analytic - 1 for the viscosity ("viscous") or the thermal
    diffusivity ("thermal") on an L x L grid."""
    from . import lbm
    e, w, c, order = gen_rules.rule(name)
    taus = [0.5 + nu / theta0, 0.5 + kappa / theta0, 0.5 + nu / theta0]
    dims = (L, L)
    if kind == "thermal":
        rho, u, th = inputs.thermal_wave(dims, amplitude=amp, theta0=theta0, mode=1)
        field, D = 3, kappa
    else:
        rho, u = inputs.shear_wave(dims, amplitude=amp, mode=1, k_axis=0, u_axis=1)
        th = np.full(rho.size, theta0)
        field, D = 2, nu
    k = 2 * np.pi / L
    steps = int(0.7 / (D * k * k / c ** 2))
    stride = max(1, steps // (n_rec - 1))

    def history(fld):
        sim = lbm.HermiteSimulation((e, w, c, order), dims, taus, storage=storage, flags=lbm.LBM_THERMAL,
                                    theta_ref=theta0)
        sim.init_fields(rho, u, th)
        fit, amps = sim.mode_history(fld, (1, 0), n_rec, stride)
        sim.close()
        return fit, amps

    if kind == "thermal":
        # the entropy-like combination dtheta / theta0 - drho / rho0 vanishes on the
        # adiabatic sound modes (gamma = (D + 2) / D = 2), so its decay is the thermal
        # mode's alone; the two amplitude histories come from identical runs
        _, a_th = history(3)
        _, a_rho = history(0)
        s = a_th / theta0 - a_rho
        rate = -np.polyfit(np.arange(n_rec) * stride, np.log(np.abs(s)), 1)[0]
    else:
        fit, _ = history(field)
        rate = fit[0]
    return rate * c ** 2 / (k * k) / D - 1.0


def study(rules=RULES, sizes=SIZES, **kw):
    """{rule: {"viscous": [err per size], "thermal": [...]}} and the observed
    orders log2(err(L) / err(2L)) between consecutive sizes."""
    out = {}
    for name in rules:
        r = {}
        for kind in ("viscous", "thermal"):
            errs = [relative_error(name, L, kind, **kw) for L in sizes]
            r[kind] = errs
            r[kind + "_order"] = [float(np.log2(abs(a) / abs(b))) for a, b in zip(errs[:-1], errs[1:])]
        out[name] = r
    return out
