"""The block variants (usp_variant_*) against the FP64 oracle
(oracle/variants.py), through the C ABI: the antisymmetrised form of a
Helmholtz medium with gain (not accretive in its raw form) and the flux form
of diffusion with a spatially varying D, on 1-, 2- and 3-D grids including
radix-3 lengths.  Tolerances as for the scalar path: relative L2 <= 1e-5 on
the iterate after the same number of iterations, 1e-4 on the history."""

import numpy as np
import pytest

from oracle import variants as ov
from paper_2207_14222_gb300 import _lib, canon, inputs

pytestmark = pytest.mark.gpu

TOL_X = 1e-5
TOL_HIST = 1e-4


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2207_14222_gb300 import build
    build.build()
    _lib.lib()
    return torch


def _rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b))


def _antisym(shape, seed):
    prob = inputs.gain_helmholtz(shape, seed)
    cp = canon.antisymmetric(prob["k2"], prob["S"])
    co = ov.antisymmetric_helmholtz(prob["k2"], prob["S"], 1.0)
    # the oracle runs on the rounded inputs the GPU sees
    co["v"] = cp["V"].astype(np.complex128)
    co["y"] = cp["y"].astype(np.complex128)
    return cp, co, ov.Antisymmetric(co)


def _flux(shape, seed):
    prob = inputs.variable_diffusion(shape, seed)
    S = np.real(prob["S"])
    cp = canon.flux_diffusion(prob["eta"], prob["D"], S)
    co = ov.flux_diffusion(prob["eta"], prob["D"], S, 1.0)
    co["Vu"] = cp["V"][0].astype(np.float64)
    co["VJ"] = cp["V"][1].astype(np.float64)
    co["y"] = cp["y"].astype(np.complex128)
    return cp, co, ov.Flux(co)


def _gpu(torch, shape, cp, n_iter=None, tol=0.0, maxit=None, alpha=0.0, schedule=0):
    from paper_2207_14222_gb300.solver import VariantSolver
    with VariantSolver(shape, cp["kind"], cp["params"], torch.from_numpy(cp["V"]).cuda(),
                       alpha=alpha, schedule=schedule) as s:
        x, r = s.solve(torch.from_numpy(cp["y"]).cuda(), tol=tol,
                       maxit=maxit if maxit else n_iter)
        return x.cpu().numpy().astype(np.complex128), r, s.history()


def _check(torch, shape, cp, op, n_iter, schedule=0):
    xg, r, hg = _gpu(torch, shape, cp, n_iter, schedule=schedule)
    assert r["iterations"] == n_iter
    assert r["alpha"] == pytest.approx(op.alpha_star(), rel=1e-6)
    xo, ho = ov.iterate(op, cp["y"].astype(np.complex128), r["alpha"], n_iter)
    assert _rel(xg, xo) <= TOL_X
    far = ho > 1e-3
    assert np.max(np.abs(hg[far] - ho[far]) / ho[far]) <= TOL_HIST
    assert r["ref_norm"] == pytest.approx(ov.reference_norm(op, cp["y"].astype(np.complex128)),
                                          rel=1e-5)


@pytest.mark.parametrize("shape", [(64,), (96,), (32, 32), (96, 64), (16, 8, 32), (8, 12 * 8, 16)])
def test_antisymmetric_trajectory(torch_cuda, shape):
    cp, co, op = _antisym(shape, 11)
    assert np.min(np.imag(inputs.gain_helmholtz(shape, 11)["k2"])) < 0   # gain present
    _check(torch_cuda, shape, cp, op, 40)


@pytest.mark.parametrize("shape", [(128,), (64, 32), (192, 16), (16, 16, 32), (8, 8, 96)])
def test_flux_trajectory(torch_cuda, shape):
    cp, co, op = _flux(shape, 12)
    _check(torch_cuda, shape, cp, op, 40)


# ---- square 2-D grids up to 128^2: the K component fields on chip (one
# cluster per problem, one launch per solve), and the passes for comparison

@pytest.mark.parametrize("kind, n, schedule", [
    ("antisymmetric", 32, 3), ("antisymmetric", 64, 3), ("antisymmetric", 128, 3),
    ("antisymmetric", 32, 1), ("flux", 32, 3), ("flux", 64, 3), ("flux", 128, 3), ("flux", 64, 1)])
def test_variant_square_grids_by_schedule(torch_cuda, kind, n, schedule):
    shape = (n, n)
    cp, co, op = (_antisym if kind == "antisymmetric" else _flux)(shape, 16 + n)
    _check(torch_cuda, shape, cp, op, 40, schedule=schedule)


def test_variant_onchip_warm_start_and_reference_pass(torch_cuda):
    """use_x0 without a reference norm: the reference pass runs on chip too,
    and the second solve continues the first one's trajectory."""
    torch = torch_cuda
    from paper_2207_14222_gb300.solver import VariantSolver
    shape = (64, 64)
    cp, co, op = _antisym(shape, 17)
    y = torch.from_numpy(cp["y"]).cuda()
    with VariantSolver(shape, cp["kind"], cp["params"], torch.from_numpy(cp["V"]).cuda(),
                       schedule=3) as s:
        x, r1 = s.solve(y, tol=0.0, maxit=15)
        x, r2 = s.solve(y, x=x, use_x0=True, tol=0.0, maxit=15)
    assert r2["ref_norm"] == pytest.approx(r1["ref_norm"], rel=1e-5)
    xo, _ = ov.iterate(op, cp["y"].astype(np.complex128), r1["alpha"], 30)
    assert _rel(x.cpu().numpy().astype(np.complex128), xo) <= TOL_X


def test_variant_onchip_schedule_validation(torch_cuda):
    torch = torch_cuda
    from paper_2207_14222_gb300.solver import VariantSolver
    for shape in ((64, 32), (16, 16, 16), (256, 256), (96, 96)):
        cp, _, _ = _antisym(shape, 18)
        with pytest.raises(_lib.UspError) as e:
            VariantSolver(shape, cp["kind"], cp["params"], torch.from_numpy(cp["V"]).cuda(),
                          schedule=3)
        assert e.value.status == _lib.ERR_UNSUPPORTED_SIZE


def test_antisymmetric_converged_solution_solves_raw_problem(torch_cuda):
    """Plain FP32 Algorithm 1 to 1e-5: the iterate agrees with the oracle's
    solve to the same tolerance, and its first component approximates the
    solution of the raw, non-accretive problem laplacian psi + k^2 psi = -S
    (dense elimination with the same spectral Laplacian)."""
    shape = (32, 32)
    prob = inputs.gain_helmholtz(shape, 13)
    cp, co, op = _antisym(shape, 13)
    xg, r, _ = _gpu(torch_cuda, shape, cp, tol=1e-5, maxit=200000)
    assert r["converged"] == 1 and r["status"] == "USP_OK"
    xo, ho, ok = ov.solve(op, cp["y"].astype(np.complex128), r["alpha"], 1e-5, 200000)
    assert ok and abs(len(ho) - r["iterations"]) <= max(3, len(ho) // 100)
    assert _rel(xg, xo) < 1e-4
    n = int(np.prod(shape))
    p2 = sum(p * p for p in ov.momenta(shape, 1.0)).ravel()
    F = np.fft.fft(np.eye(shape[0]))
    F2 = np.kron(F, np.fft.fft(np.eye(shape[1])))
    lap = np.linalg.solve(F2, (-p2)[:, None] * F2)
    A0 = lap + np.diag(prob["k2"].ravel())
    psi = np.linalg.solve(A0, -prob["S"].ravel()).reshape(shape)
    assert n == psi.size and _rel(xg[0], psi) < 1e-2


def test_flux_slab_on_gpu(torch_cuda):
    """The slab with the mixed boundary condition (Sec. 3.2), solved on the
    GPU in FP32: within 1e-3 of the analytic Robin Green's function."""
    n, D, ze = 256, 1.0, 8.0
    xa, xb, x0 = 96, 160, 120
    x = np.arange(n, dtype=np.float64)
    eta = np.where((x >= xa) & (x <= xb), 0.0, D / ze ** 2)
    S = np.zeros(n)
    S[x0] = 1.0
    cp = canon.flux_diffusion(eta, D, S)
    xg, r, _ = _gpu(torch_cuda, (n,), cp, tol=1e-5, maxit=200000)
    assert r["converged"] == 1
    u = (xg[0] / np.sqrt(cp["scales"][0])).real
    fa, fb = xa - 0.5, xb + 0.5
    Leff = fb - fa + 2 * ze
    A, B = (fb + ze - x0) / (D * Leff), (x0 - fa + ze) / (D * Leff)
    ua = np.where(x <= x0, A * (x - fa + ze), B * (fb + ze - x))
    inside = (x >= xa + 4) & (x <= xb - 4) & (np.abs(x - x0) > 3)
    assert np.max(np.abs(u[inside] - ua[inside])) / np.max(ua[inside]) < 1e-3


def test_variant_validation(torch_cuda):
    torch = torch_cuda
    from paper_2207_14222_gb300.solver import VariantSolver
    shape = (32, 32)
    cp, _, _ = _antisym(shape, 14)
    V = cp["V"].copy()
    V[3, 4] = 1.2
    with pytest.raises(_lib.UspError) as e:
        VariantSolver(shape, "antisymmetric", cp["params"], torch.from_numpy(V).cuda())
    assert e.value.status == _lib.ERR_V_NOT_CONTRACTIVE
    cf, _, _ = _flux(shape, 15)
    bad = cf["params"].copy()
    bad[0] = 0.5      # Re L would be negative
    with pytest.raises(_lib.UspError) as e:
        VariantSolver(shape, "flux", bad, torch.from_numpy(cf["V"]).cuda())
    assert e.value.status == _lib.ERR_NOT_ACCRETIVE
