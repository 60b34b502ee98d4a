"""FP64 oracle of the learned relaxation-rate closure (TEST INFRASTRUCTURE ONLY).

The paper leaves every relaxation rate above the second order free (Sec. II.C,
after Eq. omega: each central moment relaxes at its own rate, and only omega_2
and omega_3 enter the Navier-Stokes-Fourier transport coefficients).  The
closure chooses the D3Q27 rates of orders 3..6 per node from the local
non-equilibrium state, fitted so that a coarse grid follows a box-filtered fine
run.  This module restates, plainly and in FP64:

* the box filter of fine populations onto a grid ``m`` times coarser (acoustic
  scaling: one coarse step is m fine steps, lattice velocities unchanged);
* the rescaling of a filtered state's non-equilibrium part,
  f -> f^eq(rho, u) + s (f - f^eq(rho, u)): the first-order non-equilibrium
  f^(1) = -tau dt D f^(0) of the Chapman-Enskog expansion is tau times one
  lattice step of the gradients, so a fine state filtered onto a grid m times
  coarser carries tau_f / (m tau_c) of what the coarse model holds for the same
  flow; s = m tau_c / tau_f makes it a coarse-model state (s = 1: unchanged);
* the a-priori targets: with f_c(t) and f_c(t + 1) the (rescaled) filtered
  states one coarse step apart, the "ideal" post-collision state is the arriving
  populations pulled back along their velocity, f*_i(x) = f_c,i(x + e_i, t + 1);
  its non-equilibrium central moments are taken about its own velocity and
  with its own equilibrium (a collision conserves rho and u, Eq. omega
  relaxes in the node's own frame);
* the features: the 19 non-equilibrium central moments of orders 2..4 of
  f_c(t) (Eq. omega's f^(1) moments), each divided by rho c_s^n, and tau_2 - 1/2,
  then standardised with a given mean / inverse deviation;
* the six rate classes of orders 3..6 (permutation classes of alpha):
  3:(2,1,0), 3:(1,1,1), 4:(2,2,0), 4:(2,1,1), 5:(2,2,1), 6:(2,2,2);
* per sample and class the sums A = sum k1^2, B = sum k1 k1*, C = sum k1*^2 of the
  scaled non-equilibrium moments k1 (pre-collision) and k1* (ideal
  post-collision), so that sum_alpha ((1 - omega) k1 - k1*)^2 = (1-omega)^2 A
  - 2 (1-omega) B + C;
* the network 20 -> 64 -> 64 -> 6 (ReLU, ReLU, omega = lo + (hi - lo) sigmoid(z);
  lo = 0, hi = 2 spans every rate Eq. omega allows) and the
  loss L = mean_s sum_c cw_c [(1-omega_c)^2 A - 2 (1-omega_c) B + C], with its
  gradient by hand-written backpropagation.

Parameter vector (flat): W1[20][64], b1[64], W2[64][64], b2[64], W3[64][6], b3[6]
(W[k][n]: input k, output n).
"""
import numpy as np

CS2 = 1.0 / 3.0
N_IN, N_H, N_OUT = 20, 64, 6
SHAPES = [("W1", (N_IN, N_H)), ("b1", (N_H,)), ("W2", (N_H, N_H)), ("b2", (N_H,)), ("W3", (N_H, N_OUT)),
          ("b3", (N_OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def alphas3():
    """All 27 multi-indices in the order a = a_x + 3 a_y + 9 a_z."""
    return [((a) % 3, (a // 3) % 3, (a // 9) % 3) for a in range(27)]


def feature_alphas():
    """The 19 multi-indices of orders 2..4, in increasing a."""
    return [al for al in alphas3() if 2 <= sum(al) <= 4]


def class_of(al):
    """Rate class 0..5 of a multi-index of order 3..6 (None for orders <= 2)."""
    s = sorted(al, reverse=True)
    n = sum(al)
    table = {(2, 1, 0): 0, (1, 1, 1): 1, (2, 2, 0): 2, (2, 1, 1): 3, (2, 2, 1): 4, (2, 2, 2): 5}
    return table.get(tuple(s)) if n >= 3 else None


def velocities3():
    return np.array([((i % 3) - 1, ((i // 3) % 3) - 1, ((i // 9) % 3) - 1) for i in range(27)])


def box_filter(f, dims, m):
    """Average m^3 blocks of fine populations f[27, N] (N = nx ny nz, x fastest)."""
    nx, ny, nz = dims
    g = f.reshape(27, nz // m, m, ny // m, m, nx // m, m)
    return g.mean(axis=(2, 4, 6)).reshape(27, -1)


def pull_back(f_next, dims):
    """f*_i(x) = f_next,i(x + e_i): the populations that left x, one step later."""
    nx, ny, nz = dims
    e = velocities3()
    out = np.empty_like(f_next)
    for i in range(27):
        plane = f_next[i].reshape(nz, ny, nx)
        out[i] = np.roll(plane, shift=(-e[i, 2], -e[i, 1], -e[i, 0]), axis=(0, 1, 2)).reshape(-1)
    return out


def _central(f, u):
    """kappa[27, N]: central moments sum_i f_i prod_d (e_id - u_d)^alpha_d."""
    e = velocities3().astype(float)
    out = np.zeros((27, f.shape[1]))
    for a, al in enumerate(alphas3()):
        p = np.ones((27, f.shape[1]))
        for d in range(3):
            if al[d]:
                p = p * (e[:, d:d + 1] - u[d][None, :]) ** al[d]
        out[a] = np.sum(f * p, axis=0)
    return out


def _keq(rho):
    m = [1.0, 0.0, CS2]
    return np.array([rho * m[al[0]] * m[al[1]] * m[al[2]] for al in alphas3()])


def rescale_neq(f, s):
    """f^eq(rho, u) + s (f - f^eq(rho, u)) per node, f^eq by its definition
    C(u)^{-1} kappa^eq (absolute populations [27, N])."""
    from . import tp_init
    e = velocities3().astype(float)
    rho = f.sum(0)
    u = (e.T @ f) / rho
    feq = tp_init(3, rho, u)
    return feq + s * (f - feq)


def _scaled_neq(f):
    """Non-equilibrium central moments about the state's own velocity, divided by
    rho c_s^n: [27, N]."""
    e = velocities3().astype(float)
    rho = f.sum(0)
    u = (e.T @ f) / rho
    k1 = _central(f, u) - _keq(rho)
    scale = np.array([np.sqrt(CS2) ** sum(a) for a in alphas3()])[:, None] * rho[None, :]
    return k1 / scale


def features_and_targets(f_t, f_t1, dims, tau2, norm):
    """X[N, 20] (standardised with norm = (mean[20], inv_std[20])) and ABC[N, 18]
    (A, B, C for class 0, then class 1, ...) from coarse states one step apart."""
    k1 = _scaled_neq(f_t)
    k1s = _scaled_neq(pull_back(f_t1, dims))
    al = alphas3()
    fa = [a for a in range(27) if 2 <= sum(al[a]) <= 4]
    X = np.zeros((f_t.shape[1], N_IN))
    X[:, :19] = k1[fa].T
    X[:, 19] = tau2 - 0.5
    mean, inv_std = norm
    X = (X - mean[None, :]) * inv_std[None, :]
    ABC = np.zeros((f_t.shape[1], 3 * N_OUT))
    for a in range(27):
        c = class_of(al[a])
        if c is None:
            continue
        ABC[:, 3 * c] += k1[a] ** 2
        ABC[:, 3 * c + 1] += k1[a] * k1s[a]
        ABC[:, 3 * c + 2] += k1s[a] ** 2
    return X, ABC


def unpack(params):
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = np.asarray(params[o:o + n], dtype=np.float64).reshape(shp)
        o += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).reshape(-1) for name, _ in SHAPES])


def init_params(seed):
    """He-style random weights, zero biases (seeded)."""
    rng = np.random.default_rng(seed)
    d = {"W1": rng.normal(0, np.sqrt(2.0 / N_IN), (N_IN, N_H)), "b1": np.zeros(N_H),
         "W2": rng.normal(0, np.sqrt(2.0 / N_H), (N_H, N_H)), "b2": np.zeros(N_H),
         "W3": rng.normal(0, np.sqrt(1.0 / N_H), (N_H, N_OUT)), "b3": np.zeros(N_OUT)}
    return pack(d)


def forward(params, X, lo=0.0, hi=2.0):
    p = unpack(params)
    z1 = X @ p["W1"] + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"] + p["b2"]
    h2 = np.maximum(z2, 0.0)
    z3 = h2 @ p["W3"] + p["b3"]
    sig = 1.0 / (1.0 + np.exp(-z3))
    return {"z1": z1, "h1": h1, "z2": z2, "h2": h2, "z3": z3, "sig": sig, "omega": lo + (hi - lo) * sig}


def loss(params, X, ABC, cw, lo=0.0, hi=2.0):
    om = forward(params, X, lo, hi)["omega"]
    A, B, C = ABC[:, 0::3], ABC[:, 1::3], ABC[:, 2::3]
    g = 1.0 - om
    return float(np.mean(np.sum(cw[None, :] * (g * g * A - 2 * g * B + C), axis=1)))


def grad(params, X, ABC, cw, lo=0.0, hi=2.0):
    """dL/dparams by backpropagation (FP64)."""
    p = unpack(params)
    fw = forward(params, X, lo, hi)
    n = X.shape[0]
    A, B = ABC[:, 0::3], ABC[:, 1::3]
    g = 1.0 - fw["omega"]
    dom = cw[None, :] * (-2.0 * g * A + 2.0 * B) / n
    dz3 = dom * (hi - lo) * fw["sig"] * (1.0 - fw["sig"])
    gW3 = fw["h2"].T @ dz3
    gb3 = dz3.sum(0)
    dh2 = dz3 @ p["W3"].T
    dz2 = dh2 * (fw["z2"] > 0)
    gW2 = fw["h1"].T @ dz2
    gb2 = dz2.sum(0)
    dh1 = dz2 @ p["W2"].T
    dz1 = dh1 * (fw["z1"] > 0)
    gW1 = X.T @ dz1
    gb1 = dz1.sum(0)
    return pack({"W1": gW1, "b1": gb1, "W2": gW2, "b2": gb2, "W3": gW3, "b3": gb3})


def class_rates(params, X, lo=0.0, hi=2.0):
    """Per-node omega for the 27 moments: classes map onto orders 3..6; orders <= 2
    get 0 here (their rates come from the relaxation times)."""
    om = forward(params, X, lo, hi)["omega"]
    out = np.zeros((X.shape[0], 27))
    for a, al in enumerate(alphas3()):
        c = class_of(al)
        if c is not None:
            out[:, a] = om[:, c]
    return out


def orders3():
    return np.array([sum(al) for al in alphas3()])


def learned_step(f, dims, tau2, params, norm, lo=0.0, hi=2.0):
    """One collide-and-stream step of D3Q27 CM-MRT (Eq. omega, one rate per
    central moment) with order 2 at 1/tau2 and orders 3..6 at the network's
    class rates for each node; periodic streaming f_i(x + e_i) <- f*_i(x).
    f: absolute populations [27, N]."""
    from . import tp_collide_node_rates
    X, _ = features_and_targets(f, f, dims, tau2, norm)
    rates = class_rates(params, X, lo, hi)
    rates[:, orders3() == 2] = 1.0 / tau2
    post = np.empty_like(f)
    for k in range(f.shape[1]):
        post[:, k] = tp_collide_node_rates(3, rates[k], f[:, k])
    nx, ny, nz = dims
    e = velocities3()
    out = np.empty_like(f)
    for i in range(27):
        plane = post[i].reshape(nz, ny, nx)
        out[i] = np.roll(plane, shift=(e[i, 2], e[i, 1], e[i, 0]), axis=(0, 1, 2)).reshape(-1)
    return out


def constant_params(omega_per_class, lo=0.0, hi=2.0):
    """A network whose output is omega_c everywhere: zero weights,
    b3 = logit((omega_c - lo) / (hi - lo))."""
    d = unpack(np.zeros(N_PARAMS))
    q = (np.asarray(omega_per_class, dtype=np.float64) - lo) / (hi - lo)
    d["b3"] = np.log(q / (1.0 - q))
    return pack(d)
