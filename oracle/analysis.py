"""FP64 analysis of oracle runs: single-wavenumber amplitudes and decay fits.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. III.A measures transport coefficients from the time history of one Fourier
component of a field: the viscous mode from u_perp, the thermal mode from the
pressure p = rho theta.  The amplitude is the discrete Fourier sum
A(t) = sum_x q(x, t) exp(-i k.x); its modulus decays as exp(-Gamma t), and the
dispersion relations (Eq. dr) give Gamma = nu k^2 for the viscous mode.
"""
import numpy as np


def mode_amplitude(q, dims, mode):
    """A = sum_x q(x) exp(-2 pi i sum_d m_d x_d / L_d) for a field q[node]."""
    dims = tuple(dims)
    D = len(dims)
    grids = np.meshgrid(*[np.arange(n) for n in dims], indexing="ij")
    phase = np.zeros(grids[0].shape)
    for d in range(D):
        phase = phase + 2 * np.pi * mode[d] * grids[d] / dims[d]
    # grids are [x, y, z]; fields are flattened with x fastest
    phase = phase.transpose(tuple(range(D))[::-1]).reshape(-1)
    return np.sum(np.asarray(q, dtype=np.float64) * np.exp(-1j * phase))


def fit_decay_rate(t, amp):
    """Least-squares slope of ln|A(t)| against t: returns Gamma with |A| ~ exp(-Gamma t)."""
    t = np.asarray(t, dtype=np.float64)
    y = np.log(np.abs(np.asarray(amp)))
    tm, ym = t.mean(), y.mean()
    slope = np.sum((t - tm) * (y - ym)) / np.sum((t - tm) ** 2)
    return -slope
