"""Seeded synthetic initial fields (density, velocity, temperature).

This module only builds input fields; it contains none of the collision
arithmetic.  Both the CUDA library (through the Python binding) and the CPU
oracle in the tests are fed from here, so that they start from the very same
numbers.  All fields are float64 numpy arrays in lattice units with the layout
``rho[node]``, ``u[d, node]``, ``node = x + nx*(y + ny*z)``.

Workloads:
  * Taylor-Green vortex in 2D (decaying, analytic decay exp(-2 nu k^2 t)) and 3D
    (the Re = 1600 transition benchmark's initial field);
  * shear and longitudinal waves on a uniform background flow, the linear-mode
    tests of Sec. III.A (Eq. modes), used to measure nu and Galilean invariance;
  * random smooth perturbations for parity tests;
  * decaying-turbulence fields with a prescribed energy spectrum for the
    batched runs (E(k) ~ k^-3 in 2D) and the closure (k^4 exp(-2 (k/k0)^2), 3D).
"""
import numpy as np

CS2_TP = 1.0 / 3.0  # sound speed squared of D2Q9 / D3Q27 in lattice units


def _grid(dims):
    dims = tuple(int(d) for d in dims)
    axes = [np.arange(n, dtype=np.float64) for n in dims]
    mesh = np.meshgrid(*axes, indexing="ij")  # mesh[d][x, y, z]
    # flatten with x fastest: transpose so the last index is x
    return dims, [m.transpose(tuple(range(len(dims)))[::-1]).reshape(-1) for m in mesh]


def taylor_green_2d(nx: int, ny: int, u0: float = 0.05, rho0: float = 1.0, cs2: float = CS2_TP):
    """u_x = -u0 cos(kx x) sin(ky y), u_y = u0 (kx/ky) sin(kx x) cos(ky y), with the
    matching pressure p = p0 - rho0 u0^2/4 (cos 2kx x + (kx/ky)^2 cos 2ky y), rho = p/cs2."""
    _, (x, y) = _grid((nx, ny))
    kx, ky = 2 * np.pi / nx, 2 * np.pi / ny
    ux = -u0 * np.cos(kx * x) * np.sin(ky * y)
    uy = u0 * (kx / ky) * np.sin(kx * x) * np.cos(ky * y)
    dp = -rho0 * u0 * u0 / 4.0 * (np.cos(2 * kx * x) + (kx / ky) ** 2 * np.cos(2 * ky * y))
    rho = rho0 + dp / cs2
    return rho, np.stack([ux, uy])


def taylor_green_3d(n: int, U0: float, rho0: float = 1.0, cs2: float = CS2_TP, dims=None):
    """u = U0 sin x cos y cos z, v = -U0 cos x sin y cos z, w = 0 on [0, 2pi)^3 at the
    node positions; p = p0 + rho0 U0^2/16 (cos 2x + cos 2y)(cos 2z + 2), rho = p / cs2."""
    dims = dims or (n, n, n)
    _, (x, y, z) = _grid(dims)
    X = 2 * np.pi * x / dims[0]
    Y = 2 * np.pi * y / dims[1]
    Z = 2 * np.pi * z / dims[2]
    ux = U0 * np.sin(X) * np.cos(Y) * np.cos(Z)
    uy = -U0 * np.cos(X) * np.sin(Y) * np.cos(Z)
    uz = np.zeros_like(ux)
    dp = rho0 * U0 * U0 / 16.0 * (np.cos(2 * X) + np.cos(2 * Y)) * (np.cos(2 * Z) + 2.0)
    return rho0 + dp / cs2, np.stack([ux, uy, uz])


def taylor_green_3d_planes(n: int, U0: float, nz: int, planes, rho0: float = 1.0, cs2: float = CS2_TP):
    """The Taylor-Green vortex of taylor_green_3d on an (n, n, nz) grid (period
    2 pi along each axis), evaluated at the given global z planes only, in their
    order: the fields of one slab of a decomposed grid (ghost planes included)."""
    planes = np.asarray(planes, dtype=np.float64)
    _, (x, y) = _grid((n, n))
    X = (2 * np.pi * x / n)[None, :]
    Y = (2 * np.pi * y / n)[None, :]
    Z = (2 * np.pi * planes / nz)[:, None]
    ux = U0 * np.sin(X) * np.cos(Y) * np.cos(Z)
    uy = -U0 * np.cos(X) * np.sin(Y) * np.cos(Z)
    dp = rho0 * U0 * U0 / 16.0 * (np.cos(2 * X) + np.cos(2 * Y)) * (np.cos(2 * Z) + 2.0)
    return (rho0 + dp / cs2).reshape(-1), np.stack([ux.reshape(-1), uy.reshape(-1), np.zeros(ux.size)])


def shear_wave(dims, amplitude: float = 1e-3, u0: float = 0.0, mode: int = 1, k_axis: int = 0,
               u_axis: int = 1, rho0: float = 1.0):
    """Viscous (shear) mode of Sec. III.A: u_perp = u0 + A sin(2 pi m x_k / L_k) along
    u_axis, uniform density; the base flow u0 is perpendicular to k as in the
    Galilean-invariance test."""
    D = len(dims)
    _, coords = _grid(dims)
    L = dims[k_axis]
    u = np.zeros((D, coords[0].size))
    u[u_axis] = u0 + amplitude * np.sin(2 * np.pi * mode * coords[k_axis] / L)
    return np.full(coords[0].size, rho0), u


def random_smooth(dims, seed: int, du: float = 0.02, drho: float = 0.01, modes: int = 3):
    """Sum of a few random low Fourier modes in every field: smooth, periodic,
    with |u| <= ~du and |rho - 1| <= ~drho."""
    rng = np.random.default_rng(seed)
    D = len(dims)
    _, coords = _grid(dims)
    N = coords[0].size

    def field(amp):
        acc = np.zeros(N)
        for _ in range(modes):
            k = [rng.integers(0, 3) for _ in range(D)]
            ph = rng.uniform(0, 2 * np.pi)
            arg = sum(2 * np.pi * k[d] * coords[d] / dims[d] for d in range(D)) + ph
            acc += rng.uniform(-1, 1) * np.cos(arg)
        return amp * acc / modes

    rho = 1.0 + field(drho)
    u = np.stack([field(du) for _ in range(D)])
    return rho, u


def random_noise(dims, seed: int, du: float = 0.02, drho: float = 0.01):
    """Independent uniform noise at every node (rough, exercises every stencil path)."""
    rng = np.random.default_rng(seed)
    N = int(np.prod(dims))
    D = len(dims)
    return 1.0 + rng.uniform(-drho, drho, N), rng.uniform(-du, du, (D, N))


def _solenoidal_2d(n: int, rng, spectrum, u_rms: float):
    """Random-phase solenoidal 2D velocity from a stream function with energy
    spectrum E(k) = spectrum(|k|) (k in box wavenumbers), scaled to u_rms."""
    kx = np.fft.fftfreq(n, 1.0 / n)
    KX, KY = np.meshgrid(kx, kx, indexing="xy")  # [y, x]
    K = np.sqrt(KX ** 2 + KY ** 2)
    E = np.zeros_like(K)
    nz = K > 0
    E[nz] = spectrum(K[nz])
    # |u_hat|^2 ~ E(k) / (2 pi k) in 2D; psi_hat = u_hat / k
    amp = np.zeros_like(K)
    amp[nz] = np.sqrt(E[nz] / (2 * np.pi * K[nz])) / K[nz]
    psi_hat = amp * np.exp(2j * np.pi * rng.uniform(size=K.shape))
    psi = np.real(np.fft.ifft2(psi_hat))
    psi_hat = np.fft.fft2(psi)
    ux = np.real(np.fft.ifft2(1j * KY * psi_hat)) * (2 * np.pi / n)
    uy = np.real(np.fft.ifft2(-1j * KX * psi_hat)) * (2 * np.pi / n)
    rms = np.sqrt(np.mean(ux ** 2 + uy ** 2))
    s = u_rms / rms if rms > 0 else 0.0
    return np.stack([ux.reshape(-1) * s, uy.reshape(-1) * s])


def decaying_turbulence_2d(n: int, seed: int, ma: float = 0.1, cs2: float = CS2_TP):
    """Square run of side n: solenoidal random-phase velocity with E(k) ~ k^-3 for
    1 <= |k| <= n/8, RMS speed ma * c_s; uniform density."""
    rng = np.random.default_rng(seed)
    kmax = n / 8.0
    spec = lambda k: np.where((k >= 1) & (k <= kmax), k ** -3.0, 0.0)
    u = _solenoidal_2d(n, rng, spec, ma * np.sqrt(cs2))
    return np.ones(n * n), u


def batched_run_sizes(n_runs: int = 512, lo: int = 64, hi: int = 512, seed: int = 0):
    """Side lengths s ~ U{lo..hi} (seeded), and Reynolds numbers log-uniform in
    [1e3, 1e5] for each of n_runs independent square runs."""
    rng = np.random.default_rng(seed)
    sides = rng.integers(lo, hi + 1, size=n_runs)
    re = 10.0 ** rng.uniform(3.0, 5.0, size=n_runs)
    return sides, re


def isotropic_turbulence_3d(n: int, seed: int, k0: float = 4.0, u_rms: float = 0.04, kmax: int = None):
    """Random-phase solenoidal 3D velocity with E(k) ~ k^4 exp(-2 (k/k0)^2) (k in box
    wavenumbers), scaled to the given RMS component speed.

    The field is band-limited: its Fourier coefficients live on the cube
    |k_d| <= kmax (default 5 k0, where E has fallen by ~1e-18 from its peak) and
    are drawn from the seed alone, so every grid size n > 2 kmax samples the very
    same continuous field (the coarse field is the fine one spectrally
    truncated).  Evaluated by separable DFT matrix products, one axis at a time."""
    K = int(kmax if kmax is not None else np.ceil(5 * k0))
    if n <= 2 * K:
        raise ValueError("grid too small for the band limit")
    rng = np.random.default_rng(seed)
    k = np.arange(-K, K + 1, dtype=np.float64)
    KZ, KY, KX = np.meshgrid(k, k, k, indexing="ij")  # [kz, ky, kx]
    K2 = KX ** 2 + KY ** 2 + KZ ** 2
    Kn = np.sqrt(K2)
    nz = K2 > 0
    E = np.where(nz, Kn ** 4 * np.exp(-2.0 * (Kn / k0) ** 2), 0.0)
    amp = np.zeros_like(Kn)
    amp[nz] = np.sqrt(E[nz] / (4 * np.pi * K2[nz]))
    comps = [amp * np.exp(2j * np.pi * rng.uniform(size=Kn.shape)) for _ in range(3)]
    kd = [KX, KY, KZ]
    div = sum(kd[d] * comps[d] for d in range(3))
    safe = np.where(nz, K2, 1.0)
    comps = [np.where(nz, comps[d] - kd[d] * div / safe, 0.0) for d in range(3)]  # Leray projection
    x = np.arange(n, dtype=np.float64)
    F = np.exp(2j * np.pi * np.outer(x, k) / n)  # [x, k]
    L = 2 * K + 1
    out = []
    for c in comps:
        a = (F @ c.reshape(L, L * L)).reshape(n, L, L)  # [z, ky, kx]
        b = np.einsum("yk,zkx->zyx", F, a)  # [z, y, kx]
        b = b.reshape(n * n, L)
        u = b.real @ F.real.T - b.imag @ F.imag.T  # real part of the x sum: [z*y, x]
        out.append(u.reshape(-1))
    u = np.stack(out)
    rms = np.sqrt(np.mean(u ** 2))
    return np.ones(n ** 3), u * (u_rms / rms)


def thermal_wave(dims, amplitude=1e-3, theta0=1.2, mode=1, k_axis=0, shear_amplitude=0.0, u0=0.0,
                 u_axis=1, rho0=1.0):
    """Linear modes of Sec. III.A (Eq. modes) on a base state (rho0, u0, theta0):
    an isobaric temperature wave theta = theta0 + A sin(2 pi m x_k / L_k) with
    rho theta = rho0 theta0, optionally superposed with a shear wave
    u_perp = u0 + A_s sin(...) along u_axis (lattice units).  Returns rho, u, theta."""
    D = len(dims)
    _, coords = _grid(dims)
    s = np.sin(2 * np.pi * mode * coords[k_axis] / dims[k_axis])
    theta = theta0 + amplitude * s
    rho = rho0 * theta0 / theta
    u = np.zeros((D, coords[0].size))
    u[u_axis] = u0 + shear_amplitude * s
    return rho, u, theta


def double_shear_layer(n: int, u0: float, shape: float = 80.0, delta: float = 0.05):
    """Double shear layer on the periodic unit square sampled at x = i/n, y = j/n:
    u_x = u0 tanh(shape (y - 1/4)) for y <= 1/2 and u0 tanh(shape (3/4 - y)) above,
    u_y = delta u0 sin(2 pi (x + 1/4)); uniform density.  u0 in lattice units."""
    _, coords = _grid((n, n))
    x = coords[0] / n
    y = coords[1] / n
    ux = np.where(y <= 0.5, u0 * np.tanh(shape * (y - 0.25)), u0 * np.tanh(shape * (0.75 - y)))
    uy = delta * u0 * np.sin(2 * np.pi * (x + 0.25))
    return np.ones(n * n), np.stack([ux, uy])
