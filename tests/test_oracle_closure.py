"""Pins of the learned-closure oracle: backpropagation against finite
differences, the class-sum form of the loss against the per-moment sum, the box
filter and pull-back against their definitions, and the a-priori targets against
Eq. omega (a coarse state evolved by one CM-MRT step with known rates yields
exactly those rates as the loss minimiser)."""
import numpy as np
import pytest

import oracle
from oracle import closure as C
from paper_1808_04406_gb300 import inputs


@pytest.fixture(scope="module")
def orc():
    oracle.lib()
    return oracle


def _dataset(rng, n=40):
    X = rng.normal(size=(n, C.N_IN))
    A = rng.uniform(0.1, 1.0, (n, C.N_OUT))
    B = A * rng.uniform(-0.5, 0.9, (n, C.N_OUT))
    Cc = B * B / A + rng.uniform(0, 0.1, (n, C.N_OUT))
    ABC = np.zeros((n, 18))
    ABC[:, 0::3], ABC[:, 1::3], ABC[:, 2::3] = A, B, Cc
    return X, ABC


def test_parameter_count_and_classes():
    assert C.N_PARAMS == 20 * 64 + 64 + 64 * 64 + 64 + 64 * 6 + 6
    counts = np.bincount([C.class_of(a) for a in C.alphas3() if C.class_of(a) is not None])
    assert list(counts) == [6, 1, 3, 3, 3, 1]
    assert len(C.feature_alphas()) == 19


# Flat offsets of the network's parameter blocks, counted by hand from the
# layout the library's closure calls also take: W1[20 x 64] row-major (input
# i, hidden unit j at i * 64 + j), b1[64], W2[64 x 64] (unit j of layer 1 to
# unit k of layer 2 at j * 64 + k), b2[64], W3[64 x 6], b3[6].
OFF_W1, OFF_B1, OFF_W2, OFF_B2, OFF_W3, OFF_B3 = 0, 1280, 1344, 5440, 5504, 5888


def _hand_network():
    """A sparse network whose every intermediate value is worked out by hand
    below: asymmetric weights (a transposed matrix reads other entries), a unit
    of each hidden layer that ReLU must zero, and output logits at ln 3, -ln 7,
    0 and -ln 3 (sigmoids 3/4, 1/8, 1/2, 1/4)."""
    p = np.zeros(5894)
    w1 = {(0, 0): 1.0, (1, 0): 1.0, (0, 1): 2.0, (1, 1): -3.0, (1, 2): 1.0}
    for (i, j), v in w1.items():
        p[OFF_W1 + i * 64 + j] = v
    p[OFF_B1 + 1], p[OFF_B1 + 2] = 1.0, -0.5
    w2 = {(0, 0): 2.0, (1, 0): 100.0, (2, 1): -1.0, (2, 3): 2.0}
    for (j, k), v in w2.items():
        p[OFF_W2 + j * 64 + k] = v
    p[OFF_B2 + 3] = -1.0
    w3 = {(0, 0): 0.25, (3, 1): -0.5, (1, 3): 50.0, (0, 4): 1.0, (3, 4): -3.0}
    for (k, c), v in w3.items():
        p[OFF_W3 + k * 6 + c] = v
    p[OFF_B3 + 0] = np.log(3.0) - 1.5
    p[OFF_B3 + 1] = 1.0 - np.log(7.0)
    p[OFF_B3 + 5] = -np.log(3.0)
    return p


def test_forward_and_unpack_on_a_hand_computed_network():
    """Sample 1 (x0 = 1, x1 = 2, other inputs 0):
      layer 1: z = (1 + 2, 2 - 6 + 1, 2 - 0.5) = (3, -3, 1.5) -> h1 = (3, 0, 1.5);
      layer 2: z2_0 = 2 * 3 + 100 * 0 = 6, z2_1 = -1.5, z2_3 = 2 * 1.5 - 1 = 2 -> h2 = (6, 0, 0, 2);
      output: z3 = (6/4 + ln 3 - 1.5, -1 + 1 - ln 7, 0, 50 * 0, 6 - 6, -ln 3)
                 = (ln 3, -ln 7, 0, 0, 0, -ln 3), sigmoid (3/4, 1/8, 1/2, 1/2, 1/2, 1/4).
    Sample 2 (x0 = -1, x1 = 3): h1 = (2, 0, 2.5) (z1_1 = -2 - 9 + 1 = -10),
      h2 = (4, 0, 0, 4), z3 = (1 + ln 3 - 1.5, -2 + 1 - ln 7, 0, 0, 4 - 12, -ln 3)."""
    p = _hand_network()
    d = C.unpack(p)
    assert d["W1"][1, 2] == 1.0 and d["W1"][2, 1] == 0.0 and d["W2"][1, 0] == 100.0
    assert d["W3"][1, 3] == 50.0 and d["b2"][3] == -1.0 and d["b3"][5] == -np.log(3.0)
    np.testing.assert_array_equal(C.pack(d), p)
    X = np.zeros((2, 20))
    X[0, :2] = (1.0, 2.0)
    X[1, :2] = (-1.0, 3.0)
    fw = C.forward(p, X)
    h1 = np.zeros((2, 64))
    h1[0, :3] = (3.0, 0.0, 1.5)
    h1[1, :3] = (2.0, 0.0, 2.5)
    np.testing.assert_allclose(fw["h1"], h1, atol=1e-15)
    h2 = np.zeros((2, 64))
    h2[0, :4] = (6.0, 0.0, 0.0, 2.0)
    h2[1, :4] = (4.0, 0.0, 0.0, 4.0)
    np.testing.assert_allclose(fw["h2"], h2, atol=1e-15)
    l3, l7 = np.log(3.0), np.log(7.0)
    z3 = np.array([[l3, -l7, 0.0, 0.0, 0.0, -l3], [l3 - 0.5, -1.0 - l7, 0.0, 0.0, -8.0, -l3]])
    np.testing.assert_allclose(fw["z3"], z3, atol=1e-14)
    np.testing.assert_allclose(fw["omega"][0], 2.0 * np.array([0.75, 0.125, 0.5, 0.5, 0.5, 0.25]), atol=1e-15)
    # the rate range maps the same sigmoids onto [lo, hi]
    np.testing.assert_allclose(C.forward(p, X[:1], 1.0, 1.98)["omega"][0],
                               1.0 + 0.98 * np.array([0.75, 0.125, 0.5, 0.5, 0.5, 0.25]), atol=1e-15)


@pytest.mark.parametrize("lo,hi", [(0.0, 2.0), (0.7, 1.9)])
def test_backpropagation_matches_central_differences(lo, hi):
    rng = np.random.default_rng(0)
    X, ABC = _dataset(rng)
    cw = rng.uniform(0.5, 2.0, C.N_OUT)
    p = C.init_params(3)
    g = C.grad(p, X, ABC, cw, lo, hi)
    idx = rng.choice(C.N_PARAMS, 60, replace=False)
    h = 1e-6
    for k in idx:
        e = np.zeros_like(p)
        e[k] = h
        fd = (C.loss(p + e, X, ABC, cw, lo, hi) - C.loss(p - e, X, ABC, cw, lo, hi)) / (2 * h)
        assert g[k] == pytest.approx(fd, rel=1e-5, abs=1e-9)


def test_rate_range_maps_the_sigmoid_onto_lo_hi():
    X = np.random.default_rng(1).normal(size=(50, C.N_IN))
    p = C.init_params(4)
    om = C.forward(p, X, 0.7, 1.9)["omega"]
    sig = C.forward(p, X)["sig"]
    np.testing.assert_allclose(om, 0.7 + 1.2 * sig, rtol=1e-15)
    assert (om >= 0.7).all() and (om <= 1.9).all() and om.std() > 0.05
    np.testing.assert_allclose(C.forward(C.constant_params([0.8, 1.0, 1.2, 1.4, 1.6, 1.8], 0.7, 1.9), X, 0.7,
                                         1.9)["omega"], np.tile([0.8, 1.0, 1.2, 1.4, 1.6, 1.8], (50, 1)), rtol=1e-14)


def test_rescaled_state_is_a_collision_with_rate_one_minus_s(orc):
    """f^eq + s (f - f^eq) relaxes every central moment of order >= 2 with
    omega = 1 - s (Eq. omega); rho and u stay, the scaled non-equilibrium moments
    grow by s."""
    dims = (4, 3, 2)
    rho, u = inputs.random_noise(dims, seed=9, du=0.05)
    f = orc.tp_init(3, rho, u)
    orc.tp_step(3, dims, orc.omega_from_tau(3, [0.6, 0.9, 0.7, 1.1, 0.8]), f, 2)
    s = 3.7
    g = C.rescale_neq(f, s)
    om = np.array([0.0, 0.0] + [1.0 - s] * 5)
    for k in range(f.shape[1]):
        np.testing.assert_allclose(g[:, k], orc.tp_collide_node(3, om, f[:, k]), rtol=0, atol=1e-14)
    np.testing.assert_allclose(C._scaled_neq(g), s * C._scaled_neq(f), rtol=1e-9, atol=1e-14)
    np.testing.assert_allclose(C.rescale_neq(f, 1.0), f, rtol=0, atol=1e-15)


def test_class_sum_loss_equals_the_per_moment_sum(orc):
    """sum_alpha ((1 - omega_c) k1 - k1*)^2 written as (1-w)^2 A - 2 (1-w) B + C."""
    dims = (8, 8, 8)
    rho, u = inputs.random_smooth(dims, seed=1, du=0.05)
    f = orc.tp_init(3, rho, u)
    orc.tp_step(3, dims, orc.omega_from_tau(3, [0.6, 0.9, 0.7, 1.1, 0.8]), f, 2)
    f1 = f.copy()
    orc.tp_step(3, dims, orc.omega_from_tau(3, [0.55, 1.2, 0.9, 0.7, 1.0]), f1, 1)
    norm = (np.zeros(20), np.ones(20))
    X, ABC = C.features_and_targets(f, f1, dims, 0.6, norm)
    om = np.random.default_rng(2).uniform(0.5, 1.8, (X.shape[0], 6))
    e = C.velocities3().astype(float)
    r = f.sum(0)
    uu = (e.T @ f) / r
    k1 = C._central(f, uu) - C._keq(r)
    fs = C.pull_back(f1, dims)
    rs = fs.sum(0)  # the post-collision state in its own frame
    us = (e.T @ fs) / rs
    k1s = C._central(fs, us) - C._keq(rs)
    direct = np.zeros(X.shape[0])
    for a, al in enumerate(C.alphas3()):
        c = C.class_of(al)
        if c is None:
            continue
        s = np.sqrt(1 / 3) ** sum(al)
        direct += ((1 - om[:, c]) * k1[a] / (r * s) - k1s[a] / (rs * s)) ** 2
    A, B, Cc = ABC[:, 0::3], ABC[:, 1::3], ABC[:, 2::3]
    viaabc = np.sum((1 - om) ** 2 * A - 2 * (1 - om) * B + Cc, axis=1)
    np.testing.assert_allclose(viaabc, direct, rtol=1e-10, atol=1e-20)


def test_box_filter_and_pull_back(orc):
    dims = (8, 4, 4)
    rho, u = inputs.random_noise(dims, seed=3)
    f = orc.tp_init(3, rho, u)
    fc = C.box_filter(f, dims, 2)
    np.testing.assert_allclose(fc.sum(1), f.sum(1) / 8, rtol=1e-13)
    uni = orc.tp_init(3, np.full(128, 1.01), np.tile([[0.02], [-0.01], [0.03]], 128))
    np.testing.assert_allclose(C.box_filter(uni, dims, 2), uni[:, :16], rtol=1e-14)
    # zero rates make a step pure streaming; pulling back undoes it
    g = orc.tp_step(3, dims, np.zeros(7), f.copy(), 1)
    np.testing.assert_allclose(C.pull_back(g, dims), f, rtol=1e-13)


def test_targets_recover_the_rates_of_a_known_cm_mrt_step(orc):
    """If the 'filtered' evolution is itself one CM-MRT step with rates omega_n
    (m = 1), then for every class B / A = 1 - omega_order exactly: Eq. omega."""
    dims = (6, 6, 6)
    rho, u = inputs.random_smooth(dims, seed=4, du=0.05)
    f = orc.tp_init(3, rho, u)
    orc.tp_step(3, dims, orc.omega_from_tau(3, [0.6, 0.9, 0.7, 1.1, 0.8]), f, 2)
    taus = [0.57, 1.3, 0.8, 1.6, 0.9]
    f1 = orc.tp_step(3, dims, orc.omega_from_tau(3, taus), f.copy(), 1)
    _, ABC = C.features_and_targets(f, f1, dims, taus[0], (np.zeros(20), np.ones(20)))
    om = orc.omega_from_tau(3, taus)
    order_of_class = [3, 3, 4, 4, 5, 6]
    for c in range(6):
        np.testing.assert_allclose(ABC[:, 3 * c + 1] / ABC[:, 3 * c], 1 - om[order_of_class[c]], rtol=1e-8)


def test_per_moment_rates_collide_reduces_to_the_order_rates(orc):
    rng = np.random.default_rng(5)
    om = orc.omega_from_tau(3, [0.6, 0.9, 1.2, 0.8, 1.1])
    per = np.array([om[sum(a)] for a in C.alphas3()])
    f = orc.tp_product_equilibrium_node(3, 1.02, [0.03, -0.02, 0.01]) + rng.normal(0, 1e-3, 27)
    np.testing.assert_allclose(orc.tp_collide_node_rates(3, per, f), orc.tp_collide_node(3, om, f), atol=1e-15)


def test_learned_step_with_a_constant_network_is_the_cm_mrt_step(orc):
    """A network that outputs omega_c = 1/tau_order everywhere turns the learned
    step into the plain CM-MRT collide-and-stream step of Eq. omega."""
    dims = (5, 4, 3)
    rho, u = inputs.random_noise(dims, seed=6, du=0.04)
    f = orc.tp_init(3, rho, u)
    orc.tp_step(3, dims, orc.omega_from_tau(3, [0.6, 0.9, 0.7, 1.1, 0.8]), f, 2)
    taus = [0.57, 1.3, 0.8, 1.6, 0.9]
    om = orc.omega_from_tau(3, taus)
    P = C.constant_params([om[3], om[3], om[4], om[4], om[5], om[6]])
    got = C.learned_step(f, dims, taus[0], P, (np.zeros(20), np.ones(20)))
    want = orc.tp_step(3, dims, om, f.copy(), 1)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-14)


def test_learned_step_conserves_mass_and_momentum(orc):
    """Orders 0 and 1 are never relaxed (Eq. omega), whatever rates the network picks."""
    dims = (4, 3, 3)
    rho, u = inputs.random_noise(dims, seed=7, du=0.04)
    f = orc.tp_init(3, rho, u)
    orc.tp_step(3, dims, orc.omega_from_tau(3, [0.6, 0.9, 0.7, 1.1, 0.8]), f, 1)
    P = C.init_params(8)
    X, _ = C.features_and_targets(f, f, dims, 0.6, (np.zeros(20), np.ones(20)))
    om = C.forward(P, X)["omega"]
    assert om.std(0).min() > 1e-3  # the rates do vary from node to node
    g = C.learned_step(f, dims, 0.6, P, (np.zeros(20), np.ones(20)))
    e = C.velocities3()
    np.testing.assert_allclose(g.sum(), f.sum(), rtol=1e-14)
    np.testing.assert_allclose(e.T @ g.sum(1), e.T @ f.sum(1), atol=1e-12)


def test_features_vanish_at_equilibrium_and_ignore_the_density_scale(orc):
    """The 19 features are non-equilibrium central moments divided by rho c_s^n.
    At the C oracle's equilibrium of any (rho, u) they vanish: the Python central
    moments and closed-form equilibrium moments agree with the C equilibrium.
    Scaling every population by a constant leaves u and the features unchanged,
    which pins the division by rho."""
    rng = np.random.default_rng(3)
    n = 50
    rho = rng.uniform(0.8, 1.2, n)
    u = rng.uniform(-0.1, 0.1, (3, n))
    feq = orc.tp_init(3, rho, u)
    k_eq = C._scaled_neq(feq)
    assert np.abs(k_eq).max() < 1e-13  # rounding, amplified by 1 / c_s^n up to 27
    f = feq + 1e-3 * rng.normal(size=feq.shape) * feq
    k = C._scaled_neq(f)
    assert np.abs(k).max() > 1e-5  # a non-equilibrium state has non-zero features
    np.testing.assert_allclose(C._scaled_neq(2.5 * f), k, rtol=1e-10, atol=1e-15)
    # orders 0 and 1 of the non-equilibrium part vanish by construction of u
    al = C.alphas3()
    low = [a for a in range(27) if sum(al[a]) <= 1]
    assert np.abs(k[low]).max() < 1e-13
