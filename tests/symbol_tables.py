"""Tabulated symbols for the table-symbol tests: the Fourier symbol of a
finite-difference operator on a periodic grid,

    L = a (-Laplacian by 3-point stencils) + b + sum_ax drift_ax D_ax,

D_ax the central difference along axis ax.  Its symbol, with
p_ax = 2 pi m / (n_ax dx) in FFT order, is

    Lhat(p) = a sum_ax (2 - 2 cos(p_ax dx)) / dx^2 + b + i sum_ax drift_ax sin(p_ax dx) / dx.

The drift term is anti-Hermitian, so Re Lhat is that of the diffusion part
and accretivity (Sec. 2) is unchanged; it also makes the table odd in p, so
a mirrored or transposed index changes the result."""

import numpy as np


def stencil_symbol(shape, dx, a, b, drift=(0.0, 0.0, 0.0), dtype=np.complex64):
    """Table of the grid's shape (k-space, FFT order); complex64 is what the
    library takes."""
    lap = np.zeros(shape)
    adv = np.zeros(shape)
    for ax, n in enumerate(shape):
        p = 2.0 * np.pi * np.fft.fftfreq(n, d=dx)
        sh = [1] * len(shape)
        sh[ax] = n
        lap = lap + ((2.0 - 2.0 * np.cos(p * dx)) / dx ** 2).reshape(sh)
        adv = adv + (drift[ax] * np.sin(p * dx) / dx).reshape(sh)
    return (complex(a) * lap + complex(b) + 1j * adv).astype(dtype)


def stencil_apply(x, dx, a, b, drift=(0.0, 0.0, 0.0)):
    """The same operator applied in real space with periodic stencils."""
    x = np.asarray(x, np.complex128)
    out = complex(b) * x
    for ax in range(x.ndim):
        up = np.roll(x, -1, axis=ax)     # x[i + 1]
        dn = np.roll(x, 1, axis=ax)      # x[i - 1]
        out = out + complex(a) * (2.0 * x - up - dn) / dx ** 2
        out = out + drift[ax] * (up - dn) / (2.0 * dx)
    return out
