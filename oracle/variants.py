"""Oracle: the paper's block variants of the canonical form, FP64.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import anything under ``oracle/``.  Plain
NumPy; shares no code with the CUDA path.

Both variants keep Algorithm 1 and the forward-eliminated form (Sec. 2.1)
unchanged,  Delta = B[(L+I)^-1 (B x + y) - x],  B = I - V,  but the unknown
has K components per grid point, V is a K x K matrix per point and L a K x K
matrix of Fourier multipliers.  Fields are arrays (K,) + grid shape.

Antisymmetrised form (Sec. 2.2, Eq. antisymmetrised), for a raw problem
A0 psi = y0 whose numerical range is not confined to a half plane: with
A0 = L0 + V0 and a real scale c,
    A = [[0, -A0^*], [A0, 0]] / c,   L = [[0, -L0^*], [L0, 0]] / c,
    x = [psi; psi'],  y = [-y0'; y0] / c,
so A is skew-Hermitian and therefore accretive; psi' solves the adjoint
problem A0^* psi' = y0' (zero when y0' = 0).  For the Helmholtz operator
A0 = laplacian + k^2 (y0 = -S): L0 = laplacian + kbar2 with kbar2 the centre
of the smallest circle enclosing the values k^2 and c = rho / 0.95 (rho its
radius), so that max |V0| / c = 0.95.  Per frequency
    (L+I)^-1 = [[1, conj(l)], [-l, 1]] / (1 + |l|^2),  l = (-|p|^2 + kbar2)/c,
and per point V = [[0, -conj(v)], [v, 0]] with v = (k^2 - kbar2)/c.

Flux form of steady diffusion (Sec. 3.2, Eqs. diffusion-F-scalar,
diffusion-F-vector, diffusion-equation-matrix-form, with d/dt = 0 and a
scalar D(r) > 0): unknown (u, J) with J = -D grad u, K = 1 + d,
    L = C^-1/2 [[etabar, div], [grad, Dinvbar I]] C^-1/2,
    V = C^-1/2 diag(eta - etabar, (1/D - Dinvbar) I) C^-1/2,
    x = C^1/2 [u; J],   y = C^-1/2 [S; 0].
etabar, Dinvbar: midpoints of the ranges of eta and 1/D (their smallest
circles on the real line).  C = diag(c_u, c_J I) equilibrates the two blocks
of V: c_u = r_eta / 0.95, c_J = r_D / 0.95 with r the half-ranges (a block
whose values are all equal takes the other block's scale), so that
||V|| = 0.95.  grad -> i p and div -> i p^T, p sampled in FFT order as in
the scalar form.  Per frequency, with a = etabar/c_u + 1, b = Dinvbar/c_J + 1,
s = (c_u c_J)^-1/2 and S = a + s^2 |p|^2 / b (Schur complement),
    (L+I)^-1 [T_u; T_J] = [ (T_u - i s p.T_J / b) / S ;
                            T_J / b - s^2 p (p.T_J) / (b^2 S) - i s p T_u / (b S) ].
"""

import numpy as np

from . import canon


def momenta(shape, dx):
    """p_ax = 2 pi m / (n dx), m the FFT-order index, broadcastable."""
    out = []
    for ax, n in enumerate(shape):
        p = 2.0 * np.pi * np.fft.fftfreq(n, d=dx)
        sh = [1] * len(shape)
        sh[ax] = n
        out.append(p.reshape(sh))
    return out


def _fft(x):
    """Unnormalised forward transform of every component (exponent -i)."""
    return np.fft.fftn(x, axes=tuple(range(1, x.ndim)))


def _ifft(x):
    return np.fft.ifftn(x, axes=tuple(range(1, x.ndim)))


# -------------------------------------------------------- antisymmetric ---

def antisymmetric_helmholtz(k2, S, dx, norm_v=0.95, S_adj=None):
    """Canonical antisymmetrised system of laplacian psi + k^2 psi = -S (and
    of the adjoint problem with source -S_adj, if given)."""
    k2 = np.asarray(k2, np.complex128)
    kbar2, rho = canon.min_enclosing_circle(k2)
    if rho <= 0:
        raise ValueError("homogeneous medium: V0 = 0, no scale")
    c = rho / norm_v
    y0 = -np.asarray(S, np.complex128)
    y0a = np.zeros_like(y0) if S_adj is None else -np.asarray(S_adj, np.complex128)
    return dict(kind="antisymmetric", v=(k2 - kbar2) / c, a=-1.0 / c, b=kbar2 / c, c=c,
                kbar2=kbar2, dx=dx, y=np.stack([-y0a / c, y0 / c]))


class Antisymmetric:
    """Operators of an antisymmetrised canonical system (dict from
    ``antisymmetric_helmholtz``)."""

    K = 2

    def __init__(self, cf):
        self.v = cf["v"]
        shape = self.v.shape
        p2 = sum(p * p for p in momenta(shape, cf["dx"]))
        self.l = cf["a"] * p2 + cf["b"]

    def B(self, x):
        v = self.v
        return np.stack([x[0] + np.conj(v) * x[1], -v * x[0] + x[1]])

    def V(self, x):
        return x - self.B(x)

    def L(self, x):
        T = _fft(x)
        return _ifft(np.stack([-np.conj(self.l) * T[1], self.l * T[0]]))

    def LpI_inv(self, t):
        T = _fft(t)
        det = 1.0 + np.abs(self.l) ** 2
        return _ifft(np.stack([(T[0] + np.conj(self.l) * T[1]) / det,
                               (-self.l * T[0] + T[1]) / det]))

    def alpha_star(self):
        """min over points of Re 1/lambda over the eigenvalues 1 -+ i|v| of
        the normal matrix B: 1 / (1 + |v|^2)."""
        return float(np.min(1.0 / (1.0 + np.abs(self.v) ** 2)))


# ----------------------------------------------------------------- flux ---

def _midpoint(vals):
    lo, hi = float(np.min(vals)), float(np.max(vals))
    return 0.5 * (lo + hi), 0.5 * (hi - lo)


def flux_diffusion(eta, D, S, dx, norm_v=0.95):
    """Canonical flux form of -div(D grad u) + eta u = S (eta >= 0, D > 0
    real arrays, S real)."""
    eta = np.asarray(eta, np.float64)
    D = np.broadcast_to(np.asarray(D, np.float64), eta.shape)
    if np.any(D <= 0) or np.any(eta < 0):
        raise ValueError("need D > 0 and eta >= 0")
    etabar, r_eta = _midpoint(eta)
    dbar, r_d = _midpoint(1.0 / D)
    if r_eta <= 0 and r_d <= 0:
        raise ValueError("homogeneous medium: V = 0, no scale")
    c_u = (r_eta if r_eta > 0 else r_d) / norm_v
    c_J = (r_d if r_d > 0 else r_eta) / norm_v
    d = eta.ndim
    y = np.zeros((1 + d,) + eta.shape, np.complex128)
    y[0] = np.asarray(S, np.float64) / np.sqrt(c_u)
    return dict(kind="flux", Vu=(eta - etabar) / c_u, VJ=(1.0 / D - dbar) / c_J,
                alpha=etabar / c_u + 1.0, beta=dbar / c_J + 1.0, s=1.0 / np.sqrt(c_u * c_J),
                c_u=c_u, c_J=c_J, etabar=etabar, dbar=dbar, dx=dx, y=y)


class Flux:
    """Operators of a canonical flux-form diffusion system (dict from
    ``flux_diffusion``)."""

    def __init__(self, cf):
        self.cf = cf
        self.Vu, self.VJ = cf["Vu"], cf["VJ"]
        self.p = momenta(self.Vu.shape, cf["dx"])
        self.K = 1 + self.Vu.ndim

    def V(self, x):
        return np.stack([self.Vu * x[0]] + [self.VJ * x[k] for k in range(1, self.K)])

    def B(self, x):
        return x - self.V(x)

    def L(self, x):
        cf = self.cf
        T = _fft(x)
        s = cf["s"]
        div = sum(1j * self.p[k] * T[1 + k] for k in range(self.K - 1))
        out = [(cf["alpha"] - 1.0) * T[0] + s * div]
        for k in range(self.K - 1):
            out.append(s * 1j * self.p[k] * T[0] + (cf["beta"] - 1.0) * T[1 + k])
        return _ifft(np.stack(out))

    def LpI_inv(self, t):
        cf = self.cf
        T = _fft(t)
        a, b, s = cf["alpha"], cf["beta"], cf["s"]
        p2 = sum(p * p for p in self.p)
        Sc = a + s * s * p2 / b
        pT = sum(self.p[k] * T[1 + k] for k in range(self.K - 1))
        out = [(T[0] - 1j * s * pT / b) / Sc]
        for k in range(self.K - 1):
            out.append(T[1 + k] / b - s * s * self.p[k] * pT / (b * b * Sc)
                       - 1j * s * self.p[k] * T[0] / (b * Sc))
        return _ifft(np.stack(out))

    def alpha_star(self):
        """B is real diagonal: min over entries of 1 / (1 - V)."""
        return float(min(np.min(1.0 / (1.0 - self.Vu)), np.min(1.0 / (1.0 - self.VJ))))

    def density(self, x):
        """u from the unknown x = C^1/2 [u; J]."""
        return x[0] / np.sqrt(self.cf["c_u"])


# ---------------------------------------------------- Algorithm 1 (blocks) --

def apply_A(op, x):
    return op.L(x) + op.V(x)


def residual_delta(op, x, y):
    """Delta = B[(L+I)^-1 (B x + y) - x] (Sec. 2.1)."""
    return op.B(op.LpI_inv(op.B(x) + y) - x)


def reference_norm(op, y):
    return float(np.linalg.norm(residual_delta(op, np.zeros_like(y), y)))


def iterate(op, y, alpha, n_iter, x0=None, ref_norm=None):
    """n_iter steps of Algorithm 1; returns (x, history ||Delta_i||/ref)."""
    x = np.zeros_like(y) if x0 is None else np.array(x0, np.complex128)
    ref = reference_norm(op, y) if ref_norm is None else ref_norm
    hist = []
    for _ in range(n_iter):
        d = residual_delta(op, x, y)
        x = x + alpha * d
        hist.append(np.linalg.norm(d) / ref)
    return x, np.array(hist)


def solve(op, y, alpha, tol, maxit):
    """Algorithm 1 until ||Delta|| / ref < tol; returns (x, history, ok)."""
    x = np.zeros_like(y)
    ref = reference_norm(op, y)
    hist = []
    for _ in range(maxit):
        d = residual_delta(op, x, y)
        x = x + alpha * d
        r = np.linalg.norm(d) / ref
        hist.append(r)
        if r < tol:
            return x, np.array(hist), True
    return x, np.array(hist), False
