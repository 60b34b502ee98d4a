"""Pins of the oracle's analysis helpers (Sec. III.A measures transport
coefficients from one Fourier component of a field and its decay rate).

The amplitude is checked against numpy's FFT on non-square 2D and 3D grids with
modes along each axis, so that a transposed axis, a wrong sign of the phase or
a wrong stride fails.  The fit is checked on exact exponentials and on an
exponential times a constant complex phase (only |A| enters)."""
import numpy as np
import pytest

from oracle import analysis


@pytest.mark.parametrize("dims,mode", [
    ((12, 7), (1, 0)), ((12, 7), (0, 2)), ((12, 7), (3, -1)),
    ((6, 5, 4), (1, 0, 0)), ((6, 5, 4), (0, 1, 0)), ((6, 5, 4), (0, 0, 3)), ((6, 5, 4), (2, -1, 1)),
])
def test_mode_amplitude_is_the_fft_component(dims, mode):
    rng = np.random.default_rng(0)
    n = int(np.prod(dims))
    q = rng.normal(size=n)
    # fields are flattened with x fastest: as an array indexed [z, y, x] (or [y, x])
    arr = q.reshape(tuple(reversed(dims)))
    F = np.fft.fftn(arr)
    idx = tuple(m % d for m, d in zip(reversed(mode), reversed(dims)))
    got = analysis.mode_amplitude(q, dims, mode)
    assert abs(got - F[idx]) <= 1e-12 * max(1.0, abs(F[idx]))


def test_mode_amplitude_of_a_plane_wave():
    """cos(2 pi m.x / L) has amplitude N / 2 at +m and at -m, and 0 elsewhere."""
    dims = (16, 10)
    x, y = np.meshgrid(np.arange(dims[0]), np.arange(dims[1]), indexing="xy")  # [y, x]
    q = np.cos(2 * np.pi * (2 * x / dims[0] + 1 * y / dims[1])).reshape(-1)
    N = dims[0] * dims[1]
    assert abs(analysis.mode_amplitude(q, dims, (2, 1)) - N / 2) < 1e-10
    assert abs(analysis.mode_amplitude(q, dims, (-2, -1)) - N / 2) < 1e-10
    assert abs(analysis.mode_amplitude(q, dims, (2, -1))) < 1e-10
    assert abs(analysis.mode_amplitude(q, dims, (1, 2))) < 1e-10


def test_decay_fit_recovers_exact_rates():
    t = np.arange(0, 500, 10.0)
    for gamma in (1e-5, 2.7554e-4, 3e-2):
        a = 0.37 * np.exp(-gamma * t)
        assert analysis.fit_decay_rate(t, a) == pytest.approx(gamma, rel=1e-10, abs=1e-15)
        # only |A| enters: a constant complex phase and a sign change nothing
        assert analysis.fit_decay_rate(t, -1j * np.exp(0.3j) * a) == pytest.approx(gamma, rel=1e-10, abs=1e-15)
    # a growing mode gives a negative rate
    assert analysis.fit_decay_rate(t, np.exp(1e-3 * t)) == pytest.approx(-1e-3, rel=1e-10)
