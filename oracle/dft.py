"""Oracle: the discrete Fourier transform by its definition.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import anything under ``oracle/``.  The
oracle shares no code with the CUDA path.

The paper applies (L+I)^-1 through "the Fourier transform over all spatial
dimensions" (Sec. 3.1, Eq. laplacian_inverse) without fixing sign or
normalisation.  Reading used throughout: forward transform unnormalised with
the negative exponent, X[m] = sum_j x[j] exp(-2 pi i j m / n), inverse with 1/n.
"""

import numpy as np


def dft_matrix(n, inverse=False):
    """The n x n DFT matrix, written from its definition.  The phase index
    j*m is reduced modulo n in integer arithmetic before the exponential so
    large products do not lose phase accuracy."""
    j = np.arange(n)
    jm = np.mod(np.outer(j, j), n)
    sgn = 1.0 if inverse else -1.0
    F = np.exp(sgn * 2j * np.pi * jm / n)
    if inverse:
        F = F / n
    return F


def naive_dftn(x, inverse=False):
    """Separable DFT over every axis of ``x``: one dense DFT-matrix product per
    axis, O(n) work per point per axis."""
    out = np.asarray(x, dtype=np.complex128)
    for ax in range(out.ndim):
        F = dft_matrix(out.shape[ax], inverse)
        out = np.moveaxis(np.tensordot(F, np.moveaxis(out, ax, 0), axes=(1, 0)),
                          0, ax)
    return out


def loop_dft_1d(x, inverse=False):
    """Pure-Python double loop over the definition (tiny sizes only)."""
    n = len(x)
    sgn = 1.0 if inverse else -1.0
    out = []
    for m in range(n):
        s = 0j
        for j in range(n):
            s += complex(x[j]) * np.exp(sgn * 2j * np.pi * ((j * m) % n) / n)
        out.append(s / n if inverse else s)
    return np.array(out)


def dense_dft_operator(shape, inverse=False):
    """The DFT over all axes as one dense matrix acting on C-order vectors
    (Kronecker product of the per-axis matrices, last axis fastest)."""
    M = np.ones((1, 1), dtype=np.complex128)
    for n in shape:
        M = np.kron(M, dft_matrix(n, inverse))
    return M
