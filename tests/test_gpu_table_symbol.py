"""The tabulated symbol (usp_lsymbol kind USP_LSYM_TABLE): Algorithm 1 with
an arbitrary translation-invariant L given by its values Lhat(p) on the
grid, against the FP64 oracle fed the same table.  The table is the symbol
of a finite-difference advection-diffusion operator (odd in p, so a
mirrored or transposed frequency index fails)."""

import numpy as np
import pytest

from oracle import canon as ocanon
from oracle import usp_oracle as uo
from paper_2207_14222_gb300 import _lib, inputs
from symbol_tables import stencil_symbol

pytestmark = pytest.mark.gpu

TOL_X = 1e-5
TOL_TC = 5e-5


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2207_14222_gb300 import build
    build.build()
    _lib.lib()
    return torch


def _problem(shape, seed, vreal=False):
    prob = inputs.random_diffusion(shape, seed, sigma_px=2.0) if vreal else \
        inputs.white_helmholtz(shape, seed)
    cf = ocanon.canonical(prob)
    V = cf["V"].real.astype(np.float32) if vreal else cf["V"].astype(np.complex64)
    y = cf["y"].astype(np.complex64)
    drift = tuple(c * abs(cf["a"]) / cf["dx"] for c in (0.6, -0.4, 0.25))
    T = stencil_symbol(shape, cf["dx"], cf["a"], cf["b"], drift)
    return cf, V, y, T


def _solver(torch, shape, cf, V, T, **kw):
    from paper_2207_14222_gb300.solver import Solver
    dev = torch.device("cuda:0")
    # a and b are deliberately wrong: the table alone defines L
    return Solver(shape, 9.0, -0.5, torch.from_numpy(V).to(dev), dx=cf["dx"],
                  lhat_table=torch.from_numpy(T).to(dev), **kw)


def _check(torch, shape, seed, n_iter, tol_x=TOL_X, vreal=False, **kw):
    cf, V, y, T = _problem(shape, seed, vreal)
    with _solver(torch, shape, cf, V, T, plain=True, **kw) as s:
        x, res = s.solve(torch.from_numpy(y).cuda(), tol=0.0, maxit=n_iter)
        hg = s.history()
        xg = x.cpu().numpy().astype(np.complex128)
    T64, V64, y64 = T.astype(np.complex128), V.astype(np.complex128), y.astype(np.complex128)
    xo, ho = uo.iterate(V64, y64, T64, res["alpha"], n_iter)
    assert res["iterations"] == n_iter
    assert res["ref_norm"] == pytest.approx(uo.reference_norm(y64, V64, T64), rel=1e-5)
    err = np.linalg.norm(xg - xo) / np.linalg.norm(xo)
    assert err <= tol_x, err
    far = ho > 1e-3
    assert np.max(np.abs(hg[far] - ho[far]) / ho[far]) <= 1e-4
    return err


@pytest.mark.parametrize("shape", [(256,), (96,), (64, 96), (96, 64), (16, 32, 8),
                                   (8, 16, 384), (32, 64, 64)])
def test_table_symbol_trajectory(torch_cuda, shape):
    """Line pass (1-D), strided TMA pass (2-D, 3-D), radix-3 lengths."""
    _check(torch_cuda, shape, 50 + len(shape), 30)


def test_table_symbol_real_potential(torch_cuda):
    _check(torch_cuda, (32, 32, 32), 61, 40, vreal=True)


def test_table_symbol_untiled_strided_pass(torch_cuda):
    """The strided pass without TMA staging."""
    _check(torch_cuda, (32, 64), 62, 30, no_tma=True)
    _check(torch_cuda, (16, 8, 32), 63, 30, no_tma=True)


def test_table_symbol_fused_schedule(torch_cuda):
    """Plane-cluster schedule: the z pass works on column-blocked planes."""
    _check(torch_cuda, (4, 256, 256), 64, 15, schedule=2)


def test_table_symbol_tensor_core_dft(torch_cuda):
    _check(torch_cuda, (256, 8, 32), 65, 25, tol_x=TOL_TC, tc_dft=True)


def test_table_symbol_solve_with_refinement(torch_cuda):
    """To 1e-6 with FP64 refinement (the FP64 passes read the same table)."""
    torch = torch_cuda
    shape = (64, 96)
    cf, V, y, T = _problem(shape, 66)
    with _solver(torch, shape, cf, V, T) as s:
        x, res = s.solve(torch.from_numpy(y).cuda(), tol=1e-6, maxit=5000,
                         allow_not_converged=False)
        xg = x.cpu().numpy().astype(np.complex128)
    T64, V64, y64 = T.astype(np.complex128), V.astype(np.complex128), y.astype(np.complex128)
    d = uo.residual_delta(xg, y64, V64, T64)
    assert np.linalg.norm(d) / res["ref_norm"] < 1.5e-6
    xo, _, ok = uo.solve(V64, y64, T64, res["alpha"], 1e-6, 5000)
    assert ok and np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= TOL_X


def test_table_symbol_apply_A(torch_cuda):
    torch = torch_cuda
    for shape in ((128,), (32, 64), (16, 16, 32)):
        cf, V, y, T = _problem(shape, 67)
        x = inputs.random_field(shape, 68).astype(np.complex64)
        with _solver(torch, shape, cf, V, T) as s:
            Ax = s.apply_A(torch.from_numpy(x).cuda()).cpu().numpy()
        Ao = uo.apply_A(x.astype(np.complex128), V.astype(np.complex128), T.astype(np.complex128))
        assert np.linalg.norm(Ax - Ao) / np.linalg.norm(Ao) < 1e-6


def test_table_symbol_matches_quadratic_symbol(torch_cuda):
    """A table holding a |p|^2 + b gives the quadratic symbol's iteration."""
    torch = torch_cuda
    from paper_2207_14222_gb300.solver import Solver
    shape = (32, 64, 64)
    prob = inputs.white_helmholtz(shape, 69)
    cf = ocanon.canonical(prob)
    V = torch.from_numpy(cf["V"].astype(np.complex64)).cuda()
    y = torch.from_numpy(cf["y"].astype(np.complex64)).cuda()
    T = torch.from_numpy(uo.lhat(shape, cf["dx"], cf["a"], cf["b"]).astype(np.complex64)).cuda()
    with Solver(shape, cf["a"], cf["b"], V, dx=cf["dx"], plain=True) as s:
        x1, _ = s.solve(y, tol=0.0, maxit=40)
    with Solver(shape, 0.0, 0.0, V, dx=cf["dx"], plain=True, lhat_table=T) as s:
        x2, _ = s.solve(y, tol=0.0, maxit=40)
    assert (torch.linalg.norm(x1 - x2) / torch.linalg.norm(x1)).item() < TOL_X


def test_table_symbol_rejections(torch_cuda):
    torch = torch_cuda
    shape = (16, 32)
    cf, V, y, T = _problem(shape, 70)
    bad = T.copy()
    bad[3, 5] = -1.5 + 0.2j                 # Re(Lhat + 1) < 0 at one frequency
    with pytest.raises(_lib.UspError) as e:
        _solver(torch, shape, cf, V, bad)
    assert e.value.status == _lib.ERR_NOT_ACCRETIVE
    bad = T.copy()
    bad[0, 7] = np.nan
    with pytest.raises(_lib.UspError) as e:
        _solver(torch, shape, cf, V, bad)
    assert e.value.status == _lib.ERR_NONFINITE
    with pytest.raises(ValueError):
        _solver(torch, shape, cf, V, T[:, :16].copy())
