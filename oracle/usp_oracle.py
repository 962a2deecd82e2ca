"""Oracle: the preconditioned fixed-point iteration in FP64 (complex128).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import anything under ``oracle/``.  The
oracle shares no code with the CUDA path; it is plain NumPy, slow and direct.

What it computes (paper Sec. 2 and 2.1):
  * A = L + V with L translation invariant (a Fourier multiplier L^(p)) and V
    a pointwise potential, scaled so that ||V|| < 1.
  * B = I - V.  Forward-eliminated preconditioned operator (Sec. 2.1):
        Gamma^-1 A = alpha B [I - (L+I)^-1 B].
  * (L+I)^-1 = F^-1 diag(1 / (L^(p) + 1)) F  (Eq. laplacian_inverse), with
    L^(p) = a |p|^2 + b sampled at p = 2 pi m / (n dx), m the FFT-order
    frequency index (readings: the continuous symbol is sampled, not a
    finite-difference symbol; the forward transform is unnormalised with the
    negative exponent).
  * Algorithm 1: x <- 0; repeat  Delta <- B[(L+I)^-1 (B x + y) - x];
    x <- x + alpha Delta;  until ||Delta|| / ||Gamma^-1 y|| < eps.
    Reading of the denominator: the alpha-free ||B (L+I)^-1 y|| (Delta at
    x = 0).  The test follows the update; the iteration count is the number
    of Delta evaluations.  Norms are the plain discrete l2 norm, summed in
    FP64.

The FFT is a library primitive (scipy.fft) standing in for the transform's
definition; ``oracle.dft`` holds the definition itself and the tests pin one
against the other.  scipy.fft runs on as many host threads as the caller
allows (``scipy.fft.set_workers``); the arithmetic does not depend on it.
Inputs are taken to complex128 before every transform (scipy.fft would
otherwise keep single precision for complex64 data).
"""

import numpy as np
import scipy.fft as sfft


# ----------------------------------------------------------------- symbol ---

def momentum_sq(shape, dx):
    """|p|^2 on the FFT-ordered frequency grid, p_ax = 2 pi m / (n_ax dx)."""
    p2 = np.zeros(shape)
    for ax, n in enumerate(shape):
        p = 2.0 * np.pi * np.fft.fftfreq(n, d=dx)
        sh = [1] * len(shape)
        sh[ax] = n
        p2 = p2 + (p ** 2).reshape(sh)
    return p2


def lhat(shape, dx, a, b):
    """Fourier symbol L^(p) = a |p|^2 + b of the translation-invariant part."""
    return complex(a) * momentum_sq(shape, dx) + complex(b)


# ----------------------------------------------------------- the operators --

def apply_L_plus_I_inverse(t, Lhat):
    """(L+I)^-1 t = F^-1 [ F t / (L^ + 1) ]  (Eq. laplacian_inverse)."""
    return sfft.ifftn(sfft.fftn(np.asarray(t, np.complex128)) / (Lhat + 1.0))


def apply_L(x, Lhat):
    """L x = F^-1 [ L^ F x ]."""
    return sfft.ifftn(Lhat * sfft.fftn(np.asarray(x, np.complex128)))


def apply_A(x, V, Lhat):
    """A x = L x + V x (the forward operator; never used by the iteration)."""
    return apply_L(x, Lhat) + V * x


def residual_delta(x, y, V, Lhat):
    """Delta = B [ (L+I)^-1 (B x + y) - x ],  B = I - V  (Algorithm 1)."""
    B = 1.0 - V
    u = apply_L_plus_I_inverse(B * x + y, Lhat)
    return B * (u - x)


def reference_norm(y, V, Lhat):
    """||Gamma^-1 y|| without the alpha factor: ||B (L+I)^-1 y||."""
    return float(np.linalg.norm((1.0 - V) * apply_L_plus_I_inverse(y, Lhat)))


def alpha_star(V):
    """Worst-case optimal step alpha = Re[B^-1] (appendix, convergence-rate
    theorem).  For the multiplication operator B = 1 - V(r) the numerical
    range of B^-1 is the convex hull of 1/(1 - V(r)), so
    Re[B^-1] = min_r Re 1/(1 - V(r))."""
    return float(np.min(np.real(1.0 / (1.0 - np.asarray(V, np.complex128)))))


# ------------------------------------------------------------ Algorithm 1 ---

def iterate(V, y, Lhat, alpha, n_iter, x0=None, ref_norm=None):
    """Exactly ``n_iter`` steps of Algorithm 1.  Returns (x, history) with
    history[i] = ||Delta_{i+1}|| / ref_norm."""
    V = np.asarray(V, np.complex128)
    y = np.asarray(y, np.complex128)
    x = np.zeros_like(y) if x0 is None else np.array(x0, np.complex128)
    if ref_norm is None:
        ref_norm = reference_norm(y, V, Lhat)
    hist = []
    for _ in range(n_iter):
        d = residual_delta(x, y, V, Lhat)
        x = x + alpha * d
        hist.append(float(np.linalg.norm(d)) / ref_norm)
    return x, np.array(hist)


def solve(V, y, Lhat, alpha, tol, maxit, x0=None, ref_norm=None):
    """Algorithm 1 until ||Delta|| / ||Gamma^-1 y|| < tol or ``maxit`` steps.
    Returns (x, history, converged)."""
    V = np.asarray(V, np.complex128)
    y = np.asarray(y, np.complex128)
    x = np.zeros_like(y) if x0 is None else np.array(x0, np.complex128)
    if ref_norm is None:
        ref_norm = reference_norm(y, V, Lhat)
    hist = []
    converged = False
    for _ in range(maxit):
        d = residual_delta(x, y, V, Lhat)
        x = x + alpha * d
        r = float(np.linalg.norm(d)) / ref_norm
        hist.append(r)
        if r < tol:
            converged = True
            break
    return x, np.array(hist), converged


def relative_residual(x, y, V, Lhat):
    """Unpreconditioned relative residual ||A x - y|| / ||y|| (the measure
    of the paper's tables, Sec. 4.1)."""
    return float(np.linalg.norm(apply_A(x, V, Lhat) - y) / np.linalg.norm(y))
