"""Oracle: the operators as dense matrices (tiny grids only).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import anything under ``oracle/``.

Builds L, V, A = L + V, B = I - V and the preconditioned operators of the
paper as explicit matrices on C-order vectors, with the Fourier transform
taken from its definition (``oracle.dft``), so that the spectral path of
``oracle.usp_oracle`` can be checked against plain linear algebra.
"""

import numpy as np

from .dft import dense_dft_operator
from .usp_oracle import lhat as _lhat


def dense_L(shape, dx, a, b):
    """L = F^-1 diag(L^(p)) F as a dense matrix."""
    F = dense_dft_operator(shape)
    Fi = dense_dft_operator(shape, inverse=True)
    Lh = _lhat(shape, dx, a, b).ravel()
    return Fi @ (Lh[:, None] * F)


def dense_system(shape, dx, a, b, V):
    """Dense (A, L, B) for A = L + diag(V), B = I - diag(V)."""
    L = dense_L(shape, dx, a, b)
    Vd = np.diag(np.asarray(V, np.complex128).ravel())
    I = np.eye(L.shape[0])
    return L + Vd, L, I - Vd


def preconditioned(A, B, alpha):
    """Gamma^-1 A = alpha B (A + B)^-1 A  (Thm 1 with L + I = A + B)."""
    return alpha * B @ np.linalg.solve(A + B, A)


def iteration_matrix(A, B, alpha):
    """M = I - Gamma^-1 A."""
    return np.eye(A.shape[0]) - preconditioned(A, B, alpha)


def real_part_bound(X):
    """Re[X] = inf Re <x, X x>/<x, x> = smallest eigenvalue of (X + X*)/2
    (definition in Eq. accretivity-condition)."""
    H = 0.5 * (X + X.conj().T)
    return float(np.linalg.eigvalsh(H)[0])


def alpha_max(A, B):
    """alpha_max = 2 Re[A^-1 + B^-1]  (Thm 2)."""
    return 2.0 * real_part_bound(np.linalg.inv(A) + np.linalg.inv(B))


def op_norm(X):
    return float(np.linalg.norm(X, 2))
