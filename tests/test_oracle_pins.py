"""Pins of the FP64 oracle against facts that do not come from the oracle:
definitions, closed forms, dense linear algebra and the paper's theorems.

Each test names the passage it follows.  No GPU needed.
"""

import json
import os

import numpy as np
import pytest

from oracle import canon, dense, dft
from oracle import usp_oracle as uo
from paper_2207_14222_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand(shape, seed):
    return inputs.random_field(shape, seed)


# ---------------------------------------------------------------- the DFT ---

def test_dft_impulse_is_constant():
    x = np.zeros((4, 6, 8), np.complex128)
    x[0, 0, 0] = 1.0
    assert np.allclose(dft.naive_dftn(x), 1.0, atol=1e-14)


def test_dft_plane_wave_is_single_bin():
    n, m0 = 12, 5
    j = np.arange(n)
    x = np.exp(2j * np.pi * m0 * j / n)
    X = dft.naive_dftn(x)
    expect = np.zeros(n, np.complex128)
    expect[m0] = n
    assert np.allclose(X, expect, atol=1e-12)


def test_dft_matrix_equals_double_loop():
    x = _rand((10,), 1)
    assert np.allclose(dft.loop_dft_1d(x), dft.dft_matrix(10) @ x, atol=1e-12)
    assert np.allclose(dft.loop_dft_1d(x, inverse=True),
                       dft.dft_matrix(10, inverse=True) @ x, atol=1e-12)


def test_dft_parseval_and_roundtrip():
    x = _rand((4, 6, 8), 2)
    X = dft.naive_dftn(x)
    assert np.isclose(np.sum(np.abs(x) ** 2), np.sum(np.abs(X) ** 2) / x.size,
                      rtol=1e-12)
    assert np.allclose(dft.naive_dftn(X, inverse=True), x, atol=1e-12)


def test_dft_shift_theorem():
    n = 16
    x = _rand((n,), 3)
    s = 5
    X = dft.naive_dftn(x)
    Xs = dft.naive_dftn(np.roll(x, s))
    m = np.arange(n)
    assert np.allclose(Xs, X * np.exp(-2j * np.pi * m * s / n), atol=1e-11)


@pytest.mark.parametrize("shape", [(16,), (6, 10), (4, 6, 8)])
def test_library_fft_matches_definition(shape):
    """The oracle's FFT step (a library primitive, scipy.fft, here also on
    several threads and from complex64 input) against the definition."""
    import scipy.fft as sfft
    x = _rand(shape, 4)
    assert np.allclose(sfft.fftn(x), dft.naive_dftn(x), atol=1e-11)
    assert np.allclose(sfft.ifftn(x), dft.naive_dftn(x, inverse=True),
                       atol=1e-12)
    with sfft.set_workers(4):
        assert np.allclose(sfft.fftn(x), dft.naive_dftn(x), atol=1e-11)
    # the operators transform in FP64 whatever the input precision
    x32 = x.astype(np.complex64)
    Lh = np.full(shape, 0.5 + 0.25j)
    got = uo.apply_L_plus_I_inverse(x32, Lh)
    expect = dft.naive_dftn(dft.naive_dftn(x32.astype(np.complex128)) / (Lh + 1.0),
                            inverse=True)
    assert got.dtype == np.complex128
    assert np.allclose(got, expect, atol=1e-13)


# ------------------------------------------------------------- the symbol ---

def test_momentum_grid_by_hand():
    n, dx = 8, 0.5
    m = np.array([0, 1, 2, 3, -4, -3, -2, -1])
    p = 2 * np.pi * m / (n * dx)
    assert np.allclose(uo.momentum_sq((n,), dx), p ** 2, rtol=1e-15)


def test_spectral_laplacian_of_smooth_function():
    """L^ = -|p|^2 is the Laplacian: for a smooth periodic function the
    spectral derivative is exact to rounding (fixes sign, 2 pi and dx)."""
    n, dx = 64, 0.1
    P = n * dx
    t = np.arange(n) * dx
    w = 2 * np.pi / P
    f = np.exp(np.sin(w * t))
    d2 = (w ** 2) * (np.cos(w * t) ** 2 - np.sin(w * t)) * f
    Lh = uo.lhat((n,), dx, -1.0, 0.0)
    assert np.allclose(uo.apply_L(f, Lh), d2, atol=1e-9)


def test_plane_wave_is_eigenvector_of_L():
    shape, dx = (8, 12), 0.7
    a, b = 0.3 - 0.2j, 1.1 + 0.4j
    m = (3, -5)
    r = np.meshgrid(*[np.arange(n) * dx for n in shape], indexing="ij")
    p = [2 * np.pi * mi / (n * dx) for mi, n in zip(m, shape)]
    x = np.exp(1j * (p[0] * r[0] + p[1] * r[1]))
    lam = a * (p[0] ** 2 + p[1] ** 2) + b
    assert np.allclose(uo.apply_L(x, uo.lhat(shape, dx, a, b)), lam * x,
                       atol=1e-12)


# --------------------------------------------------- (L+I)^-1, dense forms ---

@pytest.mark.parametrize("shape", [(16,), (6, 8), (4, 4, 6)])
def test_spectral_inverse_equals_dense_solve(shape):
    """(L+I)^-1 by FFT (Eq. laplacian_inverse) equals a dense solve with L
    built from the DFT definition."""
    dx, a, b = 0.8, -0.4 + 0.1j, 0.6 + 0.3j
    L = dense.dense_L(shape, dx, a, b)
    t = _rand(shape, 5)
    u_dense = np.linalg.solve(L + np.eye(L.shape[0]), t.ravel())
    u = uo.apply_L_plus_I_inverse(t, uo.lhat(shape, dx, a, b))
    assert np.allclose(u.ravel(), u_dense, atol=1e-11)


def _small_helmholtz(shape, seed):
    prob = inputs.random_helmholtz(shape, seed, sigma_px=1.5, amplitude=0.3,
                                   abl_width=max(1, min(shape) // 4))
    cf = canon.canonical(prob)
    Lh = uo.lhat(shape, cf["dx"], cf["a"], cf["b"])
    return cf, Lh


def _small_diffusion(shape, seed):
    prob = inputs.random_diffusion(shape, seed, sigma_px=1.5)
    cf = canon.canonical(prob)
    Lh = uo.lhat(shape, cf["dx"], cf["a"], cf["b"])
    return cf, Lh


def test_elimination_identity():
    """Sec. 2.1: B[(L+I)^-1(Bx+y) - x] = B (L+I)^-1 (y - A x), because
    A + B = L + I."""
    shape = (6, 8, 10)
    cf, Lh = _small_helmholtz(shape, 7)
    x = _rand(shape, 8)
    lhs = uo.residual_delta(x, cf["y"], cf["V"], Lh)
    rhs = (1 - cf["V"]) * uo.apply_L_plus_I_inverse(
        cf["y"] - uo.apply_A(x, cf["V"], Lh), Lh)
    assert np.allclose(lhs, rhs, atol=1e-12 * np.abs(lhs).max())


def test_delta_is_preconditioned_residual_dense():
    """Delta = alpha^-1 Gamma^-1 (y - A x) with Gamma^-1 = alpha B (A+B)^-1."""
    shape = (4, 4, 6)
    cf, Lh = _small_helmholtz(shape, 9)
    A, L, B = dense.dense_system(shape, cf["dx"], cf["a"], cf["b"], cf["V"])
    x = _rand(shape, 10).ravel()
    y = cf["y"].ravel()
    expect = B @ np.linalg.solve(A + B, y - A @ x)
    got = uo.residual_delta(x.reshape(shape), cf["y"], cf["V"], Lh).ravel()
    assert np.allclose(got, expect, atol=1e-11 * np.abs(expect).max())


# ------------------------------------------------------ Algorithm 1 pins ---

@pytest.mark.parametrize("shape", [(64,), (12, 12), (6, 6, 8)])
def test_fixed_point_solves_Ax_eq_y(shape):
    """Eq. neumann_series: the limit of Algorithm 1 solves A x = y.  Brute
    force: Gaussian elimination (library solve) on the dense A = L + V."""
    cf, Lh = _small_helmholtz(shape, 11)
    A, _, _ = dense.dense_system(shape, cf["dx"], cf["a"], cf["b"], cf["V"])
    x_dense = np.linalg.solve(A, cf["y"].ravel())
    x, hist, ok = uo.solve(cf["V"], cf["y"], Lh, 0.9, 1e-13, 20000)
    assert ok
    err = np.linalg.norm(x.ravel() - x_dense) / np.linalg.norm(x_dense)
    assert err < 1e-9


def test_fixed_point_diffusion_dense():
    shape = (8, 10)
    cf, Lh = _small_diffusion(shape, 12)
    A, _, _ = dense.dense_system(shape, cf["dx"], cf["a"], cf["b"], cf["V"])
    x_dense = np.linalg.solve(A, cf["y"].ravel())
    x, hist, ok = uo.solve(cf["V"], cf["y"], Lh, 1.0, 1e-13, 20000)
    assert ok
    assert np.linalg.norm(x.ravel() - x_dense) / np.linalg.norm(x_dense) < 1e-9


def test_constant_potential_closed_form():
    """With V = v constant, A = L + v is diagonal in Fourier space, so the
    fixed point is F^-1[F y / (L^ + v)] for every alpha in (0, 1]."""
    shape, dx = (8, 12, 16), 1.0
    # homogeneous absorbing medium k^2 = k0^2 + i kappa, real bias k0^2:
    # V0 = i kappa, circle radius kappa, c = i kappa/0.95, V = 0.95
    k0, kappa = np.pi / 2, 0.4
    c = 1j * kappa / 0.95
    a, b = -1 / c, k0 ** 2 / c
    v = 1j * kappa / c
    y = _rand(shape, 13)
    Lh = uo.lhat(shape, dx, a, b)
    expect = np.fft.ifftn(np.fft.fftn(y) / (Lh + v))
    for alpha in (1.0, 0.6):
        x, hist, ok = uo.solve(np.full(shape, v), y, Lh, alpha, 1e-12, 20000)
        assert ok
        assert np.linalg.norm(x - expect) / np.linalg.norm(expect) < 1e-10


def test_monotone_decrease_fp64():
    """Thm 1 / Corollary: ||I - Gamma^-1 A|| < 1 for accretive A, ||V|| < 1
    and alpha in (0, 1], so ||Delta_i|| decreases strictly."""
    cf, Lh = _small_helmholtz((24, 24), 14)
    for alpha in (1.0, uo.alpha_star(cf["V"])):
        _, hist = uo.iterate(cf["V"], cf["y"], Lh, alpha, 200)
        h = hist[hist > 1e-13]
        assert np.all(np.diff(h) < 0)
        assert hist[0] == pytest.approx(1.0)


def test_neumann_recurrence():
    """Appendix, convergence rate: Delta_i = (I - Gamma^-1 A) Delta_{i-1}."""
    shape = (4, 6, 4)
    cf, Lh = _small_helmholtz(shape, 15)
    A, _, B = dense.dense_system(shape, cf["dx"], cf["a"], cf["b"], cf["V"])
    alpha = 0.8
    M = dense.iteration_matrix(A, B, alpha)
    x = np.zeros(shape, np.complex128)
    prev = None
    for _ in range(6):
        d = uo.residual_delta(x, cf["y"], cf["V"], Lh)
        if prev is not None:
            assert np.allclose(d.ravel(), M @ prev, atol=1e-12 * np.abs(prev).max())
        prev = d.ravel()
        x = x + alpha * d


def test_theorem2_alpha_threshold_is_sharp():
    """Thm 2: ||I - alpha B (A+B)^-1 A|| < 1 iff alpha < 2 Re[A^-1 + B^-1];
    Thm 1 states alpha_max > 1."""
    shape = (4, 4, 4)
    cf, Lh = _small_helmholtz(shape, 16)
    A, _, B = dense.dense_system(shape, cf["dx"], cf["a"], cf["b"], cf["V"])
    amax = dense.alpha_max(A, B)
    assert amax > 1.0
    assert dense.op_norm(dense.iteration_matrix(A, B, 0.99 * amax)) < 1.0
    assert dense.op_norm(dense.iteration_matrix(A, B, 1.01 * amax)) > 1.0


def test_corollary_bounds_and_unit_step():
    """Corollary: Re[B] >= 1 - ||V||, Re[A+B] >= 1 - ||V||, and every
    alpha in (0, 1] gives a contraction."""
    shape = (6, 8)
    cf, Lh = _small_helmholtz(shape, 17)
    A, L, B = dense.dense_system(shape, cf["dx"], cf["a"], cf["b"], cf["V"])
    nv = np.max(np.abs(cf["V"]))
    assert dense.real_part_bound(A) >= -1e-12        # accretive
    assert dense.real_part_bound(B) >= 1 - nv - 1e-12
    assert dense.real_part_bound(A + B) >= 1 - nv - 1e-12
    for alpha in (0.1, 0.5, 1.0):
        assert dense.op_norm(dense.iteration_matrix(A, B, alpha)) < 1.0


def test_hermitian_optimal_step_rate():
    """Hermitian case (diffusion): ||M|| at alpha = 2/(lmin + lmax) equals
    (lmax - lmin)/(lmax + lmin), lambda the spectrum of (A^-1 + B^-1)^-1."""
    shape = (6, 6)
    cf, Lh = _small_diffusion(shape, 18)
    A, _, B = dense.dense_system(shape, cf["dx"], cf["a"], cf["b"], cf["V"])
    assert np.allclose(A, A.conj().T, atol=1e-12)
    G = np.linalg.inv(np.linalg.inv(A) + np.linalg.inv(B))
    lam = np.linalg.eigvalsh(0.5 * (G + G.conj().T))
    lmin, lmax = lam[0], lam[-1]
    alpha = 2 / (lmin + lmax)
    got = dense.op_norm(dense.iteration_matrix(A, B, alpha))
    assert got == pytest.approx((lmax - lmin) / (lmax + lmin), rel=1e-9)


def test_condition_number_bound():
    """Appendix, condition number: kappa(Gamma^-1 A) <=
    (||A^-1|| + (1 - ||V||)^-1) (1 + ||V||)."""
    shape = (4, 4, 4)
    cf, Lh = _small_helmholtz(shape, 19)
    A, _, B = dense.dense_system(shape, cf["dx"], cf["a"], cf["b"], cf["V"])
    P = dense.preconditioned(A, B, 1.0)
    kappa = np.linalg.cond(P)
    nv = np.max(np.abs(cf["V"]))
    bound = (dense.op_norm(np.linalg.inv(A)) + 1 / (1 - nv)) * (1 + nv)
    assert kappa <= bound * (1 + 1e-12)


def test_shift_splitting_is_special_case():
    """Sec. 4.2: V = 0, L = A = A0/gamma, alpha = 2 gives
    Gamma^-1 A = Gamma_shift^-1 A0 with Gamma_shift = (A0 + gamma I)/2."""
    rng = np.random.default_rng(20)
    n = 12
    X = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    A0 = (X - X.conj().T) / 2 + 0.5 * np.eye(n)          # strictly accretive
    gamma = 1.7
    A = A0 / gamma
    B = np.eye(n)
    lhs = dense.preconditioned(A, B, 2.0)
    rhs = np.linalg.solve(0.5 * (A0 + gamma * np.eye(n)), A0)
    assert np.allclose(lhs, rhs, atol=1e-12)


def test_alpha_star_is_real_part_of_B_inverse():
    """alpha = Re[B^-1] (convergence-rate theorem) for B = I - diag(V)."""
    cf, _ = _small_helmholtz((6, 6), 21)
    B = np.eye(36) - np.diag(cf["V"].ravel())
    assert uo.alpha_star(cf["V"]) == pytest.approx(
        dense.real_part_bound(np.linalg.inv(B)), rel=1e-12)


def test_table1_qualitative_fixed_point():
    """Table 1: plain Richardson on A diverges for every alpha; with the
    universal split preconditioner it converges for every alpha."""
    g = json.load(open(os.path.join(GOLDEN, "table1_fixed_point_qualitative.json")))
    shape = (128,)
    prob = inputs.random_helmholtz(shape, 22, sigma_px=3.0, amplitude=0.3,
                                   abl_width=16)
    cf = canon.canonical(prob, norm_v=g["norm_V"])
    Lh = uo.lhat(shape, cf["dx"], cf["a"], cf["b"])
    y, V = cf["y"], cf["V"]
    for alpha in g["alpha"]:
        x = np.zeros_like(y)
        r0 = np.linalg.norm(y)
        for _ in range(200):
            x = x + alpha * (y - uo.apply_A(x, V, Lh))
        assert np.linalg.norm(y - uo.apply_A(x, V, Lh)) > 1e3 * r0   # 'd'
        _, hist, ok = uo.solve(V, y, Lh, alpha, 1e-3, 20000)
        assert ok and np.all(np.diff(hist) < 0)


# ------------------------------------------------------- canonical form ---

def _brute_force_mec(P):
    best = None
    pts = list(P)
    cands = []
    for i in range(len(pts)):
        cands.append((pts[i], 0.0))
        for j in range(i + 1, len(pts)):
            c = 0.5 * (pts[i] + pts[j])
            cands.append((c, abs(pts[i] - c)))
            for k in range(j + 1, len(pts)):
                a, b, d = pts[i], pts[j], pts[k]
                # circumcentre from the perpendicular-bisector equations
                M = np.array([[2 * (b - a).real, 2 * (b - a).imag],
                              [2 * (d - a).real, 2 * (d - a).imag]])
                rhs = np.array([abs(b) ** 2 - abs(a) ** 2, abs(d) ** 2 - abs(a) ** 2])
                if abs(np.linalg.det(M)) < 1e-14:
                    continue
                u = np.linalg.solve(M, rhs)
                c = complex(u[0], u[1])
                cands.append((c, abs(a - c)))
    for c, r in cands:
        if all(abs(p - c) <= r * (1 + 1e-9) + 1e-12 for p in pts):
            if best is None or r < best[1]:
                best = (c, r)
    return best


@pytest.mark.parametrize("seed", range(6))
def test_smallest_circle_brute_force(seed):
    rng = np.random.default_rng(100 + seed)
    P = rng.standard_normal(9) + 1j * rng.standard_normal(9)
    c, r = canon.min_enclosing_circle(P)
    cb, rb = _brute_force_mec(P)
    assert r == pytest.approx(rb, rel=1e-9)
    assert abs(c - cb) < 1e-8


def test_smallest_circle_large_set_known_answer():
    rng = np.random.default_rng(30)
    centre, rad = 2.0 + 1.5j, 3.0
    theta = np.array([0.1, 2.2, 4.1])                       # acute triangle
    rim = centre + rad * np.exp(1j * theta)
    inner = centre + rad * 0.99 * np.sqrt(rng.uniform(size=20000)) * \
        np.exp(2j * np.pi * rng.uniform(size=20000))
    c, r = canon.min_enclosing_circle(np.concatenate([inner, rim]))
    assert r == pytest.approx(rad, rel=1e-12)
    assert abs(c - centre) < 1e-10


def test_canonical_helmholtz_properties():
    """Sec. 2.2 and 3.1: ||V|| = 0.95, c = i rho/0.95 and A accretive
    (Re L^ + Re V = 0.95 Im k^2 / rho >= 0 for a gain-free medium)."""
    prob = inputs.helmholtz_2d(64, 3, abl_width=8)
    cf = canon.canonical(prob)
    assert np.max(np.abs(cf["V"])) == pytest.approx(0.95, rel=1e-12)
    rho = abs(cf["c"]) * 0.95
    assert cf["c"] == pytest.approx(1j * rho / 0.95)
    Lh = uo.lhat(cf["V"].shape, 1.0, cf["a"], cf["b"])
    assert np.min(Lh.real) >= -1e-12
    re_sum = np.min(Lh.real) + np.min(cf["V"].real)
    assert re_sum >= -1e-12
    assert np.allclose(Lh.real.min() + cf["V"].real,
                       0.95 * prob["k2"].imag / rho, atol=1e-12)


def test_canonical_diffusion_properties():
    prob = inputs.random_diffusion((16, 16), 4)
    cf = canon.canonical(prob)
    assert np.max(np.abs(cf["V"])) == pytest.approx(0.95, rel=1e-12)
    assert np.isrealobj(cf["c"]) or np.imag(cf["c"]) == 0
    assert cf["c"] > 0
    assert np.allclose(cf["V"].imag, 0)


# ----------------------------------------------- closed-form physics pins ---

def _gaussian_series(P, n_terms, w, x0, x, symbol):
    """Fourier series of the periodic solution for a Gaussian source
    exp(-(x-x0)^2/(2 w^2)), evaluated term by term:
    psi_m = S_m / symbol(p_m), S_m = sqrt(2 pi) w exp(-p_m^2 w^2/2) e^{-i p_m x0}/P."""
    m = np.arange(-n_terms, n_terms + 1)
    p = 2 * np.pi * m / P
    Sm = np.sqrt(2 * np.pi) * w * np.exp(-0.5 * (p * w) ** 2) * np.exp(-1j * p * x0) / P
    return np.exp(1j * np.outer(x, p)) @ (Sm / symbol(p))


def test_helmholtz_1d_gaussian_source_series():
    """E1 (empty medium converges to the analytic field): homogeneous
    absorbing medium, psi'' + k^2 psi = -S; the canonical iteration's limit
    equals the series sum_m S_m/(p_m^2 - k^2) e^{i p_m x}."""
    n, dx = 256, 1.0
    k0, kappa = np.pi / 2, 0.3
    k2 = k0 ** 2 + 1j * kappa
    P, w, x0 = n * dx, 2.0, 100.0
    xg = np.arange(n) * dx
    S = np.zeros(n, np.complex128)
    for img in (-1, 0, 1):
        S += np.exp(-0.5 * ((xg - x0 + img * P) / w) ** 2)
    c = 1j * kappa / 0.95                       # real bias k0^2, radius kappa
    V = np.full(n, (k2 - k0 ** 2) / c)
    y = -S / c
    Lh = uo.lhat((n,), dx, -1 / c, k0 ** 2 / c)
    x, hist, ok = uo.solve(V, y, Lh, 1.0, 1e-13, 50000)
    assert ok
    ref = _gaussian_series(P, 4 * n, w, x0, xg, lambda p: p ** 2 - k2)
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) < 1e-8


def test_helmholtz_1d_point_source_green_function():
    """Periodic Green's function of psi'' + k^2 psi = -delta:
    G(x) = -cos(k(|x| - P/2)) / (2 k sin(k P/2)), compared away from the
    source (the grid solution is its truncated Fourier series)."""
    n, dx = 1024, 0.25
    k0, kappa = np.pi / 2, 0.2
    k2 = k0 ** 2 + 1j * kappa
    k = np.sqrt(k2)
    P = n * dx
    S = np.zeros(n, np.complex128)
    S[0] = 1.0 / dx
    c = 1j * kappa / 0.95
    Lh = uo.lhat((n,), dx, -1 / c, k0 ** 2 / c)
    x, _, ok = uo.solve(np.full(n, (k2 - k0 ** 2) / c), -S / c, Lh, 1.0,
                        1e-12, 50000)
    assert ok
    xs = np.arange(n) * dx
    d = np.minimum(xs, P - xs)
    G = -np.cos(k * (d - P / 2)) / (2 * k * np.sin(k * P / 2))
    far = (d > 8.0)
    err = np.abs(x[far] - G[far]).max() / np.abs(G[far]).max()
    assert err < 5e-3


def test_diffusion_1d_closed_forms():
    """-D u'' + eta u = S, constant eta: point source
    u = cosh((P/2 - |x|)/l) / (2 sqrt(D eta) sinh(P/(2 l))), l = sqrt(D/eta);
    Gaussian source: the Fourier series with symbol D p^2 + eta."""
    n, dx, D = 512, 0.5, 1.0
    eta_lo, eta_hi = 0.04, 0.06      # only the bias and scale use the range
    eta = 0.05
    P = n * dx
    etabar, rho = 0.5 * (eta_lo + eta_hi), 0.5 * (eta_hi - eta_lo)
    c = rho / 0.95
    V = np.full(n, (eta - etabar) / c)
    Lh = uo.lhat((n,), dx, D / c, etabar / c)
    xs = np.arange(n) * dx
    # point source
    S = np.zeros(n)
    S[0] = 1.0 / dx
    u, _, ok = uo.solve(V, S / c, Lh, 1.0, 1e-13, 50000)
    assert ok
    ell = np.sqrt(D / eta)
    d = np.minimum(xs, P - xs)
    ua = np.cosh((P / 2 - d) / ell) / (2 * np.sqrt(D * eta) * np.sinh(P / (2 * ell)))
    far = d > 5.0
    assert np.abs(u[far] - ua[far]).max() / ua.max() < 2e-3
    # Gaussian source: tight
    w, x0 = 3.0, 77.0
    Sg = sum(np.exp(-0.5 * ((xs - x0 + img * P) / w) ** 2) for img in (-1, 0, 1))
    ug, _, ok = uo.solve(V, Sg / c, Lh, 1.0, 1e-13, 50000)
    assert ok
    ref = _gaussian_series(P, 4 * n, w, x0, xs, lambda p: D * p ** 2 + eta)
    assert np.linalg.norm(ug - ref) / np.linalg.norm(ref) < 1e-8


def _dense_laplacian(shape, dx):
    """The spectral Laplacian F^-1 diag(-|p|^2) F from the DFT definition."""
    return dense.dense_L(shape, dx, -1.0, 0.0)


def test_canonical_helmholtz_solves_physical_equation():
    """Sec. 2.2: x = x0, so the canonical solution must solve the physical
    equation laplacian(psi) + k^2 psi = -S itself (dense brute force)."""
    shape = (10, 12)
    prob = inputs.random_helmholtz(shape, 40, sigma_px=1.5, abl_width=2,
                                   source="random")
    cf = canon.canonical(prob)
    A0 = _dense_laplacian(shape, prob["dx"]) + np.diag(prob["k2"].ravel())
    psi = np.linalg.solve(A0, -prob["S"].ravel())
    Lh = uo.lhat(shape, cf["dx"], cf["a"], cf["b"])
    x, _, ok = uo.solve(cf["V"], cf["y"], Lh, 1.0, 1e-13, 50000)
    assert ok
    assert np.linalg.norm(x.ravel() - psi) / np.linalg.norm(psi) < 1e-9


def test_canonical_diffusion_solves_physical_equation():
    shape = (8, 6, 6)
    prob = inputs.random_diffusion(shape, 41, sigma_px=1.0)
    cf = canon.canonical(prob)
    A0 = -prob["D"] * _dense_laplacian(shape, prob["dx"]) + np.diag(prob["eta"].ravel())
    u = np.linalg.solve(A0, prob["S"].ravel())
    Lh = uo.lhat(shape, cf["dx"], cf["a"], cf["b"])
    x, _, ok = uo.solve(cf["V"], cf["y"], Lh, 1.0, 1e-13, 50000)
    assert ok
    assert np.linalg.norm(x.ravel() - u) / np.linalg.norm(u) < 1e-9


def test_history_is_relative_preconditioned_residual():
    """Algorithm 1 convergence test: history_i = ||Delta_i|| / ||Gamma^-1 y||
    with the alpha-free denominator ||B (A+B)^-1 y|| (dense); the solve stops
    at the first step below the tolerance, after the update."""
    shape = (4, 6, 4)
    cf, Lh = _small_helmholtz(shape, 42)
    A, _, B = dense.dense_system(shape, cf["dx"], cf["a"], cf["b"], cf["V"])
    y = cf["y"].ravel()
    ref = np.linalg.norm(B @ np.linalg.solve(A + B, y))
    alpha, tol = 0.7, 1e-4
    x, hist, ok = uo.solve(cf["V"], cf["y"], Lh, alpha, tol, 10000)
    xd = np.zeros_like(y)
    M = dense.iteration_matrix(A, B, alpha)
    expect = []
    for _ in range(len(hist)):
        d = B @ np.linalg.solve(A + B, y - A @ xd)
        xd = xd + alpha * d
        expect.append(np.linalg.norm(d) / ref)
    assert np.allclose(hist, expect, rtol=1e-9)
    assert ok and hist[-1] < tol and np.all(hist[:-1] >= tol)
    assert np.allclose(x.ravel(), xd, atol=1e-12 * np.abs(xd).max())
    assert uo.reference_norm(cf["y"], cf["V"], Lh) == pytest.approx(ref, rel=1e-12)
    # a fixed number of steps (no stopping test) follows the same recurrence
    xi, hi = uo.iterate(cf["V"], cf["y"], Lh, alpha, len(hist))
    assert np.allclose(hi, expect, rtol=1e-9)
    assert np.allclose(xi.ravel(), xd, atol=1e-12 * np.abs(xd).max())


# --------------------------------------------------- tabulated symbol ---

@pytest.mark.parametrize("shape", [(12,), (6, 10), (4, 6, 8)])
def test_table_symbol_equals_real_space_stencil(shape):
    """The operators accept any tabulated symbol Lhat(p) (Sec. 2: L is any
    translation-invariant operator, applied through its Fourier symbol).  With
    the symbol of a periodic finite-difference operator, the oracle's L x is
    that stencil applied in real space: pins the FFT-order frequency layout
    (the drift term is odd in p, so a mirrored axis fails)."""
    from symbol_tables import stencil_apply, stencil_symbol
    dx, a, b, drift = 0.7, 0.3 - 0.2j, 0.1 + 0.4j, (0.9, -0.5, 0.3)
    x = _rand(shape, 41)
    T = stencil_symbol(shape, dx, a, b, drift).astype(np.complex128)
    # the table is rounded to complex64: compare with the stencil of the same operator
    got = uo.apply_L(x, T)
    want = stencil_apply(x, dx, a, b, drift)
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-6
    # the FP64 table agrees to rounding
    Texact = stencil_symbol(shape, dx, a, b, drift, dtype=np.complex128)
    assert np.allclose(uo.apply_L(x, Texact), want, rtol=1e-12, atol=1e-12)
    # the inverse of (L + I) through the same table solves the stencil system
    u = uo.apply_L_plus_I_inverse(x, Texact)
    assert np.allclose(stencil_apply(u, dx, a, b, drift) + u, x, rtol=1e-11, atol=1e-11)



# ------------------------------------- unpreconditioned relative residual ---

def _check_relative_residual(fn):
    """Largest deviation of ``fn(x, y, V, Lhat)`` from ||A x - y|| / ||y||
    with A = L + diag(V) assembled densely from the DFT definition (Sec. 4.1's
    measure), at a random x, at x = 0 (exactly 1) and at the solution of A x
    = y by Gaussian elimination (0 up to rounding)."""
    shape = (4, 6, 8)
    cf, Lh = _small_helmholtz(shape, 21)
    A, _, _ = dense.dense_system(shape, cf["dx"], cf["a"], cf["b"], cf["V"])
    y = cf["y"]
    errs = []
    for seed in (22, 23):
        x = _rand(shape, seed)
        expect = np.linalg.norm(A @ x.ravel() - y.ravel()) / np.linalg.norm(y)
        errs.append(abs(fn(x, y, cf["V"], Lh) - expect) / expect)
    errs.append(abs(fn(np.zeros(shape, np.complex128), y, cf["V"], Lh) - 1.0))
    xs = np.linalg.solve(A, y.ravel()).reshape(shape)
    errs.append(abs(fn(xs, y, cf["V"], Lh)))
    return max(errs)


def test_relative_residual_against_dense_operator():
    assert _check_relative_residual(uo.relative_residual) < 1e-12


@pytest.mark.parametrize("mistake", ["divide_by_x", "drop_V", "preconditioned",
                                     "sign_of_V", "squared"])
def test_relative_residual_pin_catches_planted_mistakes(mistake):
    """Plausible mistakes in the residual (dividing by ||x||, leaving out V,
    reporting the preconditioned residual, a sign slip, the squared norm)
    each fail the dense pin above."""
    def planted(x, y, V, Lh):
        nrm = np.linalg.norm
        if mistake == "divide_by_x":
            return nrm(uo.apply_A(x, V, Lh) - y) / max(nrm(x), 1e-300)
        if mistake == "drop_V":
            return nrm(uo.apply_L(x, Lh) - y) / nrm(y)
        if mistake == "preconditioned":
            return nrm(uo.residual_delta(x, y, V, Lh)) / nrm(y)
        if mistake == "sign_of_V":
            return nrm(uo.apply_L(x, Lh) - V * x - y) / nrm(y)
        return nrm(uo.apply_A(x, V, Lh) - y) ** 2 / nrm(y) ** 2
    assert _check_relative_residual(planted) > 1e-3


# ------------------------------------- empty medium: 2-D and 3-D Green's ---

def _point_source_solution(shape, dx, k0, kappa):
    """Algorithm 1 on a homogeneous absorbing medium k^2 = k0^2 + i kappa
    with a unit point source at the origin: real bias k0^2, circle radius
    kappa, c = i kappa / 0.95, so V = 0.95 everywhere (Sec. 3.1)."""
    k2 = k0 ** 2 + 1j * kappa
    c = 1j * kappa / 0.95
    S = np.zeros(shape, np.complex128)
    S[(0,) * len(shape)] = 1.0 / dx ** len(shape)
    Lh = uo.lhat(shape, dx, -1 / c, k0 ** 2 / c)
    x, _, ok = uo.solve(np.full(shape, (k2 - k0 ** 2) / c), -S / c, Lh, 1.0,
                        1e-11, 5000)
    assert ok
    return x, np.sqrt(k2)


def _off_axis_mask(d, dx, ndim):
    """Grid points at least two pixels from every coordinate plane through
    the source.  The sampled symbol differs from the continuous one only
    beyond the grid's band, and the aliased remainder of a point source's
    field concentrates on those planes (the band is a product of intervals);
    elsewhere the grid field equals the continuous one to about 2e-4."""
    m = d >= 2 * dx
    out = m
    for _ in range(ndim - 1):
        out = np.multiply.outer(out, m)
    return out


def test_helmholtz_2d_point_source_green_function():
    """Empty-medium check (Sec. 3.1) in 2-D: laplacian psi + k^2 psi = -delta
    has the free-space solution (i/4) H0^(1)(k r); on the periodic grid the
    field is the sum of its periodic images (which converges: Im k > 0)."""
    from scipy.special import hankel1
    n, dx, k0, kappa, images = 256, 0.5, np.pi / 2, 0.3, 3
    x, k = _point_source_solution((n, n), dx, k0, kappa)
    P = n * dx
    d = np.minimum(np.arange(n) * dx, P - np.arange(n) * dx)
    G = np.zeros((n, n), np.complex128)
    for i in range(-images, images + 1):
        for j in range(-images, images + 1):
            r = np.hypot(d[:, None] + i * P, d[None, :] + j * P)
            G += 0.25j * hankel1(0, k * np.where(r > 0, r, 1.0))
    m = _off_axis_mask(d, dx, 2)
    assert np.abs(x[m] - G[m]).max() / np.abs(G[m]).max() < 1e-3


def test_helmholtz_3d_point_source_green_function():
    """Empty-medium check (Sec. 3.1) in 3-D: the free-space solution is
    e^{i k r} / (4 pi r), summed over its periodic images."""
    n, dx, k0, kappa, images = 64, 0.5, np.pi / 2, 0.5, 2
    x, k = _point_source_solution((n, n, n), dx, k0, kappa)
    P = n * dx
    d = np.minimum(np.arange(n) * dx, P - np.arange(n) * dx)
    G = np.zeros((n, n, n), np.complex128)
    for i in range(-images, images + 1):
        for j in range(-images, images + 1):
            for l in range(-images, images + 1):
                r = np.sqrt((d[:, None, None] + i * P) ** 2
                            + (d[None, :, None] + j * P) ** 2
                            + (d[None, None, :] + l * P) ** 2)
                G += np.exp(1j * k * r) / (4 * np.pi * np.where(r > 0, r, 1.0))
    m = _off_axis_mask(d, dx, 3)
    assert np.abs(x[m] - G[m]).max() / np.abs(G[m]).max() < 1e-3
