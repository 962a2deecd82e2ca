"""Pins of the block-variant oracle (oracle/variants.py): the antisymmetrised
form of a non-accretive Helmholtz problem and the flux form of steady
diffusion, checked against dense Gaussian elimination of the raw problems,
the closed-form inverse against the forward operator, skew-Hermitian /
accretive structure, the scalar diffusion form, and the slab solution with
the mixed boundary condition (analytic)."""

import numpy as np
import pytest

from oracle import canon, usp_oracle as uo, variants as ov


def _dense_from(apply, shape):
    """Dense matrix of a linear map on fields of `shape` (column by column)."""
    n = int(np.prod(shape))
    M = np.zeros((n, n), np.complex128)
    for j in range(n):
        e = np.zeros(n, np.complex128)
        e[j] = 1.0
        M[:, j] = apply(e.reshape(shape)).ravel()
    return M


def _grad_ops(shape, dx):
    """Spectral derivatives d/dx_ax as dense matrices (i p in FFT order)."""
    ps = ov.momenta(shape, dx)
    return [_dense_from(lambda f, p=p: np.fft.ifftn(1j * p * np.fft.fftn(f)), shape) for p in ps]


def _gain_medium(shape, seed):
    rng = np.random.default_rng(seed)
    k0 = np.pi / 2
    n = 1.0 + 0.2 * rng.uniform(size=shape)
    kappa = 0.3 * (rng.uniform(size=shape) - 0.5)        # gain where kappa < 0
    S = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    return k0 ** 2 * (n ** 2 + 1j * kappa), S


def test_antisymmetric_structure_and_inverse():
    shape, dx = (6, 8), 1.0
    k2, S = _gain_medium(shape, 1)
    assert np.min(k2.imag) < 0 < np.max(k2.imag)   # the raw range spans both half planes
    cf = ov.antisymmetric_helmholtz(k2, S, dx)
    op = ov.Antisymmetric(cf)
    assert np.max(np.abs(cf["v"])) == pytest.approx(0.95, rel=1e-12)
    rng = np.random.default_rng(2)
    z = rng.standard_normal((2,) + shape) + 1j * rng.standard_normal((2,) + shape)
    w = rng.standard_normal((2,) + shape) + 1j * rng.standard_normal((2,) + shape)
    # A = L + V skew-Hermitian: <z, A w> = -<A z, w>
    Aw, Az = ov.apply_A(op, w), ov.apply_A(op, z)
    assert np.vdot(z, Aw) == pytest.approx(-np.vdot(Az, w), rel=1e-12)
    # closed-form (L+I)^-1 inverts the forward L + I
    t = op.LpI_inv(z)
    assert np.allclose(op.L(t) + t, z, atol=1e-12)


def test_antisymmetric_solves_the_raw_problem_and_its_adjoint():
    """psi solves laplacian psi + k^2 psi = -S (dense elimination of the raw,
    non-accretive operator); psi' solves the adjoint problem with -S'."""
    shape, dx = (24,), 1.0
    k2, S = _gain_medium(shape, 3)
    Sa = np.random.default_rng(4).standard_normal(shape) + 0j
    cf = ov.antisymmetric_helmholtz(k2, S, dx, S_adj=Sa)
    op = ov.Antisymmetric(cf)
    x, hist, ok = ov.solve(op, cf["y"], op.alpha_star(), 1e-11, 200000)
    assert ok
    lap = _dense_from(lambda f: np.fft.ifftn(-sum(p * p for p in ov.momenta(shape, dx))
                                             * np.fft.fftn(f)), shape)
    A0 = lap + np.diag(k2.ravel())
    psi = np.linalg.solve(A0, -S.ravel())
    psia = np.linalg.solve(A0.conj().T, -Sa.ravel())
    assert np.linalg.norm(x[0].ravel() - psi) / np.linalg.norm(psi) < 1e-8
    assert np.linalg.norm(x[1].ravel() - psia) / np.linalg.norm(psia) < 1e-8
    # Algorithm 1 contracts: the residual history decreases overall
    assert hist[-1] < 1e-11 and hist[0] > hist[len(hist) // 2] > hist[-1]


def _diffusion_medium(shape, seed, vary_D=True):
    rng = np.random.default_rng(seed)
    eta = 0.05 * np.exp(0.5 * rng.standard_normal(shape))
    D = 1.0 + (0.5 * rng.uniform(size=shape) if vary_D else 0.0)
    S = np.zeros(shape)
    S[tuple(n // 2 for n in shape)] = 1.0
    return eta, D, S


def test_flux_structure_and_inverse():
    shape, dx = (6, 8), 1.0
    eta, D, S = _diffusion_medium(shape, 5)
    cf = ov.flux_diffusion(eta, D, S, dx)
    op = ov.Flux(cf)
    assert op.K == 3
    assert max(np.max(np.abs(cf["Vu"])), np.max(np.abs(cf["VJ"]))) == pytest.approx(0.95)
    rng = np.random.default_rng(6)
    z = rng.standard_normal((3,) + shape) + 1j * rng.standard_normal((3,) + shape)
    # L accretive: its Hermitian part is diag(etabar/c_u, Dinvbar/c_J) >= 0
    assert np.real(np.vdot(z, op.L(z))) >= 0
    assert np.real(np.vdot(z, ov.apply_A(op, z))) >= 0
    t = op.LpI_inv(z)
    assert np.allclose(op.L(t) + t, z, atol=1e-12)


def test_flux_form_solves_variable_D_diffusion():
    """u of the flux form solves -div(D grad u) + eta u = S with the same
    spectral derivatives (dense elimination of the raw second-order form)."""
    shape, dx = (8, 6), 1.0
    eta, D, S = _diffusion_medium(shape, 7)
    cf = ov.flux_diffusion(eta, D, S, dx)
    op = ov.Flux(cf)
    x, _, ok = ov.solve(op, cf["y"], op.alpha_star(), 1e-12, 100000)
    assert ok
    G = _grad_ops(shape, dx)
    Dd = np.diag(D.ravel())
    M = -sum(g @ Dd @ g for g in G) + np.diag(eta.ravel())
    u = np.linalg.solve(M, S.ravel())
    assert np.linalg.norm(op.density(x).ravel() - u) / np.linalg.norm(u) < 1e-9


def test_flux_form_matches_scalar_form_for_constant_D():
    shape, dx = (16, 12), 1.0
    eta, _, S = _diffusion_medium(shape, 8, vary_D=False)
    cf = ov.flux_diffusion(eta, 1.7, S, dx)
    op = ov.Flux(cf)
    x, _, ok = ov.solve(op, cf["y"], op.alpha_star(), 1e-12, 100000)
    assert ok
    cs = canon.diffusion(eta, 1.7, S, dx)
    Lh = uo.lhat(shape, dx, cs["a"], cs["b"])
    xs, _, ok2 = uo.solve(cs["V"], cs["y"], Lh, uo.alpha_star(cs["V"]), 1e-12, 100000)
    assert ok2
    assert np.linalg.norm(op.density(x) - xs) / np.linalg.norm(xs) < 1e-9


def test_slab_with_mixed_boundary_condition():
    """Sec. 3.2's check: a slab [xa, xb] without absorption inside and
    eta = D / z_e^2 outside obeys u = -z_e n.grad u at its faces, so inside
    the slab u is the Green's function of -D u'' with those Robin conditions:
    linear on each side of the source, u = A (x - xa + z_e) left of it and
    u = B (xb + z_e - x) right of it, A + B = 1/D."""
    # z_e spans several pixels so the exponential tail outside is resolved
    n, dx, D, ze = 256, 1.0, 1.0, 8.0
    xa, xb, x0 = 96, 160, 120
    x = np.arange(n) * dx
    eta = np.where((x >= xa) & (x <= xb), 0.0, D / ze ** 2)
    S = np.zeros(n)
    S[x0] = 1.0 / dx
    cf = ov.flux_diffusion(eta, D, S, dx)
    op = ov.Flux(cf)
    xs, _, ok = ov.solve(op, cf["y"], op.alpha_star(), 1e-10, 200000)
    assert ok
    u = op.density(xs).real
    # the slab covers pixels xa..xb, so its faces lie half a pixel outside
    fa, fb = xa - 0.5 * dx, xb + 0.5 * dx
    Leff = fb - fa + 2 * ze
    A = (fb + ze - x0) / (D * Leff)
    B = (x0 - fa + ze) / (D * Leff)
    ua = np.where(x <= x0, A * (x - fa + ze), B * (fb + ze - x))
    inside = (x >= xa + 4) & (x <= xb - 4) & (np.abs(x - x0) > 3)
    assert np.max(np.abs(u[inside] - ua[inside])) / np.max(ua[inside]) < 1e-3
    # outside the solution decays with the extrapolation length
    ratio = u[xa - 9] / u[xa - 5]
    assert ratio == pytest.approx(np.exp(-4 * dx / ze), rel=0.05)


@pytest.mark.parametrize("form", ["antisymmetric", "flux"])
def test_iterate_follows_the_dense_recurrence(form):
    """Algorithm 1 in the block forms: x_{i+1} = x_i + alpha B (L+I)^-1 (y - A x_i)
    (Sec. 2.1), with (L+I)^-1 taken as the dense inverse of L + I rather than
    the closed form; the history is ||Delta_i|| / ||Delta_1|| at x0 = 0, so its
    first entry is exactly 1."""
    shape, dx = (6, 4), 1.0
    if form == "antisymmetric":
        k2, S = _gain_medium(shape, 11)
        cf = ov.antisymmetric_helmholtz(k2, S, dx)
        op = ov.Antisymmetric(cf)
    else:
        eta, D, S = _diffusion_medium(shape, 12)
        cf = ov.flux_diffusion(eta, D, S, dx)
        op = ov.Flux(cf)
    y = cf["y"]
    full = y.shape
    L = _dense_from(op.L, full)
    Vd = _dense_from(op.V, full)
    Bd = _dense_from(op.B, full)
    A = L + Vd
    LpI_inv = np.linalg.inv(L + np.eye(L.shape[0]))
    alpha, n_iter = 0.7, 9
    x, hist = ov.iterate(op, y, alpha, n_iter)
    xd = np.zeros(y.size, np.complex128)
    ref = np.linalg.norm(Bd @ LpI_inv @ y.ravel())
    hd = []
    for _ in range(n_iter):
        d = Bd @ LpI_inv @ (y.ravel() - A @ xd)
        xd = xd + alpha * d
        hd.append(np.linalg.norm(d) / ref)
    assert hist[0] == pytest.approx(1.0, rel=1e-12)
    assert np.allclose(hist, hd, rtol=1e-10)
    assert np.linalg.norm(x.ravel() - xd) / np.linalg.norm(xd) < 1e-11
    assert ov.reference_norm(op, y) == pytest.approx(ref, rel=1e-12)
