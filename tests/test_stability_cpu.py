"""Host logic of the maximum-Mach search of the double shear layer (Sec. III.C):
the k-ary bracket search against known thresholds, and the initial field."""
import numpy as np
import pytest

from paper_1808_04406_gb300 import inputs, stability as S


@pytest.mark.parametrize("thr", [0.0731, 0.2688, 0.7, 0.999])
def test_bracket_contains_the_threshold(thr):
    calls = []

    def survive(mas):
        calls.append(len(mas))
        return [m < thr for m in mas]

    lo, hi = S.kary_search(survive, 0.05, 1.0, k=7, rounds=4)
    assert lo < hi
    assert (lo <= thr <= hi) or (thr < 0.05 and hi <= 0.05 + 0.95 / 8)
    assert hi - lo <= 0.95 / 8 ** 4 + 1e-12
    assert calls == [7, 7, 7, 7]


def test_first_failure_closes_the_bracket():
    """A survivor above a failure (non-monotone noise) does not reopen the bracket."""
    lo, hi = S.kary_search(lambda m: [x < 0.3 or 0.6 < x < 0.7 for x in m], 0.0, 1.0, k=3, rounds=1)
    assert (lo, hi) == (0.25, 0.5)


def test_many_problems_are_searched_together():
    thr = [0.2, 0.45, 0.9]
    out = S.kary_search_many(lambda c: [[x < t for x in cc] for cc, t in zip(c, thr)], 3, 0.05, 1.0)
    for (lo, hi), t in zip(out, thr):
        assert lo <= t <= hi and hi - lo < 1e-3


def test_double_shear_layer_field():
    n, u0 = 64, 0.1
    rho, u = inputs.double_shear_layer(n, u0)
    ux = u[0].reshape(n, n)
    uy = u[1].reshape(n, n)
    assert np.all(rho == 1.0)
    assert np.allclose(ux, ux[:, :1])  # u_x depends on y only
    assert np.allclose(uy, uy[:1, :])  # u_y depends on x only: divergence-free
    assert ux[n // 4, 0] == 0.0 and np.isclose(ux[3 * n // 4, 0], 0.0)
    assert np.isclose(np.abs(ux).max(), u0 * np.tanh(80 * 0.25))
    assert np.isclose(np.abs(uy).max(), 0.05 * u0)


def test_units_of_the_search():
    """Re = u0 c L / nu and t_c = L / (u0 / c) steps on the 37-velocity lattice."""
    from paper_1808_04406_gb300.gen_d2q37 import lattice_scale
    c = lattice_scale()
    taus, steps, u_lat = S.h37_params(128, 0.25, 1e4, 2.0, True)
    assert np.isclose(u_lat, 0.25 / c)
    assert np.isclose((taus[0] - 0.5) * 1e4, 0.25 * c * 128)
    assert np.isclose(taus[1] - 0.5, (taus[0] - 0.5) / 2.0)
    assert steps == int(np.ceil(2 * 128 * c / 0.25))
    t9, s9, u9 = S.d2q9_params(128, 0.1, 1e4)
    assert np.isclose(u9, 0.1 / np.sqrt(3)) and np.isclose((t9[0] - 0.5) / 3 * 1e4, u9 * 128)
