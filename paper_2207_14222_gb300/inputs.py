"""Seeded synthetic workloads: physical fields only.

This module produces the *raw* physical description of a problem -- the
wavenumber field k^2(r) of a Helmholtz medium, the absorption rate eta(r) of a
diffusion medium, and the source S(r) -- from a seed.  It holds none of the
method's arithmetic: no canonical scaling, no spectral operator, no iteration.
Both the CUDA solver (through its own canonicalisation) and the FP64 oracle
(through its own) start from these arrays.

Physical conventions (the paper's Helmholtz problem, Sec. 3.1):
    laplacian(psi) + k^2(r) psi = -S(r)
pixel = lambda/4, so with dx = 1 the vacuum wavenumber is k0 = 2*pi/4.

Diffusion (steady state of the paper's diffusion equation, Sec. 3.2, scalar
constant D):
    -D laplacian(u) + eta(r) u = S(r)

Array layout: C order, the last axis fastest ([nz][ny][nx] in 3-D).
"""

import numpy as np

K0_QUARTER_WAVE = 2.0 * np.pi / 4.0   # pixel = lambda/4, dx = 1


def smooth_field(shape, sigma_px, rng):
    """White Gaussian noise convolved (periodically) with a Gaussian of
    standard deviation ``sigma_px`` pixels, then normalised to zero mean and
    unit variance."""
    noise = rng.standard_normal(shape)
    spec = np.fft.rfftn(noise)
    k2 = np.zeros(spec.shape)
    for ax, n in enumerate(shape):
        if ax == len(shape) - 1:
            f = np.fft.rfftfreq(n)
        else:
            f = np.fft.fftfreq(n)
        sh = [1] * len(shape)
        sh[ax] = f.size
        k2 = k2 + ((2.0 * np.pi * f) ** 2).reshape(sh)
    spec *= np.exp(-0.5 * sigma_px ** 2 * k2)
    g = np.fft.irfftn(spec, s=shape, axes=tuple(range(len(shape))))
    g -= g.mean()
    sd = g.std()
    return g / sd if sd > 0 else g


def boundary_depth(shape, width):
    """Normalised depth d/W in [0, 1] into an absorbing layer of ``width``
    pixels on every face (0 in the interior).  Per axis the depth is measured
    from the inner edge of the layer; axes combine by their maximum."""
    d = np.zeros(shape)
    if width <= 0:
        return d
    for ax, n in enumerate(shape):
        i = np.arange(n, dtype=np.float64)
        da = np.maximum(np.maximum(width - i, i - (n - 1 - width)), 0.0) / width
        da = np.minimum(da, 1.0)
        sh = [1] * len(shape)
        sh[ax] = n
        d = np.maximum(d, da.reshape(sh))
    return d


def _centre_point_source(shape, dx):
    S = np.zeros(shape, dtype=np.complex128)
    S[tuple(n // 2 for n in shape)] = 1.0 / dx ** len(shape)
    return S


def helmholtz_medium(shape, n_index, abl_width, k0=K0_QUARTER_WAVE,
                     kappa_max=1.0):
    """k^2(r) of a medium with refractive index ``n_index`` in the interior,
    tapered to vacuum inside an absorbing layer where
    k^2 = k0^2 (n^2 + i kappa_max (d/W)^2)."""
    d = boundary_depth(shape, abl_width)
    taper = (1.0 - d) ** 2
    n_eff = 1.0 + (n_index - 1.0) * taper
    return k0 ** 2 * (n_eff ** 2 + 1j * kappa_max * d ** 2)


def helmholtz_2d(n=128, seed=0, sigma_px=4.0, amplitude=0.3, abl_width=16):
    """2-D Helmholtz medium: n = 1 + amplitude*g with g a smoothed random field
    peak-normalised to [-1, 1]; absorbing layer; unit point source at the
    centre pixel."""
    rng = np.random.default_rng(seed)
    shape = (n, n)
    g = smooth_field(shape, sigma_px, rng)
    g = g / np.max(np.abs(g))
    n_index = 1.0 + amplitude * g
    k2 = helmholtz_medium(shape, n_index, abl_width)
    return dict(kind="helmholtz", k2=k2, S=_centre_point_source(shape, 1.0),
                dx=1.0, k0=K0_QUARTER_WAVE, seed=seed)


def helmholtz_3d(n=256, seed=0, n_spheres=8):
    """3-D Helmholtz medium: n in [1, 1.5] from a smoothed random field
    (sigma = 6 px at n = 256, lengths scale with n/256), plus spheres of
    n = 1.45 in the interior, absorbing layer of n/8 px per face, and a
    Gaussian beam source (waist 16 px at n = 256, flat phase) on the plane
    z = W + 2."""
    scale = n / 256.0
    rng = np.random.default_rng(seed)
    shape = (n, n, n)
    W = int(round(32 * scale))
    g = smooth_field(shape, 6.0 * scale, rng)
    g = (g - g.min()) / (g.max() - g.min())
    n_index = 1.0 + 0.5 * g
    zz, yy, xx = np.meshgrid(*(np.arange(n, dtype=np.float64),) * 3,
                             indexing="ij")
    for _ in range(n_spheres):
        rad = rng.uniform(8.0, 24.0) * scale
        c = rng.uniform(W + rad, n - 1 - W - rad, size=3)
        inside = (zz - c[0]) ** 2 + (yy - c[1]) ** 2 + (xx - c[2]) ** 2 <= rad ** 2
        n_index[inside] = 1.45
    del zz, yy, xx
    k2 = helmholtz_medium(shape, n_index, W)
    w0 = 16.0 * scale
    S = np.zeros(shape, dtype=np.complex128)
    y1 = np.arange(n, dtype=np.float64) - n / 2
    rho2 = y1[:, None] ** 2 + y1[None, :] ** 2
    S[W + 2] = np.exp(-rho2 / w0 ** 2)
    return dict(kind="helmholtz", k2=k2, S=S, dx=1.0, k0=K0_QUARTER_WAVE,
                seed=seed)


def diffusion_3d(n=256, seed=0, median_eta=0.01, sigma_log=0.5, D=1.0):
    """3-D steady diffusion medium: log-normal absorption rate
    eta = median * exp(sigma_log * g), g a unit-variance smoothed random field
    (sigma = 6 px at n = 256); constant D; unit point source at the centre;
    periodic, no absorbing layer."""
    scale = n / 256.0
    rng = np.random.default_rng(seed)
    shape = (n, n, n)
    g = smooth_field(shape, 6.0 * scale, rng)
    eta = median_eta * np.exp(sigma_log * g)
    return dict(kind="diffusion", eta=eta, D=D,
                S=_centre_point_source(shape, 1.0), dx=1.0, seed=seed)


def random_helmholtz(shape, seed, sigma_px=2.0, amplitude=0.3, abl_width=None,
                     source="point"):
    """Small random Helmholtz medium of any shape (parity and edge cases)."""
    rng = np.random.default_rng(seed)
    if abl_width is None:
        abl_width = max(1, min(shape) // 8)
    g = smooth_field(shape, sigma_px, rng)
    m = np.max(np.abs(g))
    g = g / m if m > 0 else g
    k2 = helmholtz_medium(shape, 1.0 + amplitude * g, abl_width)
    if source == "point":
        S = _centre_point_source(shape, 1.0)
    else:
        S = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))
    return dict(kind="helmholtz", k2=k2, S=S, dx=1.0, k0=K0_QUARTER_WAVE,
                seed=seed)


def random_diffusion(shape, seed, sigma_px=2.0, median_eta=0.05, sigma_log=0.5,
                     D=1.0):
    """Small random diffusion medium of any shape."""
    rng = np.random.default_rng(seed)
    g = smooth_field(shape, sigma_px, rng)
    eta = median_eta * np.exp(sigma_log * g)
    return dict(kind="diffusion", eta=eta, D=D,
                S=_centre_point_source(shape, 1.0), dx=1.0, seed=seed)


def white_helmholtz(shape, seed, contrast=0.3, absorption=0.3, k0=K0_QUARTER_WAVE):
    """Unsmoothed random medium of any shape, including axes of length 2:
    k^2 = k0^2 (n^2 + i kappa) with n - 1 and kappa uniform per pixel, and a
    random complex source."""
    rng = np.random.default_rng(seed)
    n_index = 1.0 + contrast * rng.uniform(size=shape)
    kappa = absorption * rng.uniform(size=shape)
    S = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    return dict(kind="helmholtz", k2=k0 ** 2 * (n_index ** 2 + 1j * kappa), S=S, dx=1.0,
                k0=k0, seed=seed)


def random_field(shape, seed, complex_=True):
    """Standard normal (complex) test vector."""
    rng = np.random.default_rng(seed)
    if complex_:
        return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    return rng.standard_normal(shape)


BATCH_SIDES = (64, 96, 128, 192, 256, 384, 512)


def batch_problem(i, seed0=1000):
    """Problem ``i`` of the mixed-size batch of 2-D problems: seed seed0 + i;
    side drawn uniformly from BATCH_SIDES; smoothing sigma uniform in
    [2, 8] px; even i: Helmholtz with n in [1, 1.5] (the smoothed field
    rescaled to that range), absorbing layer side/8 px, centre point source;
    odd i: steady diffusion with log-normal absorption (median 0.01/px,
    sigma_log 0.5, D = 1), centre point source."""
    rng = np.random.default_rng(seed0 + i)
    side = int(BATCH_SIDES[rng.integers(len(BATCH_SIDES))])
    sigma = float(rng.uniform(2.0, 8.0))
    shape = (side, side)
    g = smooth_field(shape, sigma, rng)
    S = _centre_point_source(shape, 1.0)
    if i % 2 == 0:
        g = (g - g.min()) / (g.max() - g.min())
        k2 = helmholtz_medium(shape, 1.0 + 0.5 * g, side // 8)
        return dict(kind="helmholtz", k2=k2, S=S, dx=1.0, k0=K0_QUARTER_WAVE,
                    seed=seed0 + i, sigma_px=sigma)
    eta = 0.01 * np.exp(0.5 * g)
    return dict(kind="diffusion", eta=eta, D=1.0, S=S, dx=1.0, seed=seed0 + i,
                sigma_px=sigma)


def gain_helmholtz(shape, seed, contrast=0.2, gain=0.15, k0=K0_QUARTER_WAVE, sigma_px=2.0):
    """Helmholtz medium with gain and loss: k^2 = k0^2 (n^2 + i kappa), n - 1
    in [0, contrast] and kappa in [-gain, gain] from smoothed random fields
    (kappa < 0: gain), so the values k^2 lie on both sides of the real axis
    and the problem's numerical range is not confined to a half plane;
    random complex source."""
    rng = np.random.default_rng(seed)
    g1 = smooth_field(shape, sigma_px, rng)
    g2 = smooth_field(shape, sigma_px, rng)
    n_index = 1.0 + contrast * (g1 - g1.min()) / max(g1.max() - g1.min(), 1e-30)
    kappa = gain * (2.0 * (g2 - g2.min()) / max(g2.max() - g2.min(), 1e-30) - 1.0)
    S = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    return dict(kind="helmholtz", k2=k0 ** 2 * (n_index ** 2 + 1j * kappa), S=S, dx=1.0,
                k0=k0, seed=seed)


def variable_diffusion(shape, seed, median_eta=0.05, sigma_log=0.5, d_range=(1.0, 2.0),
                       sigma_px=2.0):
    """Steady diffusion with a spatially varying scalar diffusion coefficient:
    log-normal absorption eta, D uniform in d_range from a smoothed field,
    unit point source at the centre."""
    rng = np.random.default_rng(seed)
    g = smooth_field(shape, sigma_px, rng)
    eta = median_eta * np.exp(sigma_log * g)
    h = smooth_field(shape, sigma_px, rng)
    t = (h - h.min()) / max(h.max() - h.min(), 1e-30)
    D = d_range[0] + (d_range[1] - d_range[0]) * t
    return dict(kind="diffusion", eta=eta, D=D, S=_centre_point_source(shape, 1.0), dx=1.0,
                seed=seed)
