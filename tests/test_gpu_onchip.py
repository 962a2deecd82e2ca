"""The on-chip schedule: square 2-D grids n x n (n = 32, 64, 128, 256) held
in the shared memory of one thread-block cluster per problem, a whole phase
of Algorithm 1 per launch.  Trajectories against the FP64 oracle, the
reference pass, warm starts, refinement, real potentials, tabulated symbols
and the edge cases of the state machine."""

import numpy as np
import pytest

from oracle import canon as ocanon
from oracle import usp_oracle as uo
from paper_2207_14222_gb300 import _lib, inputs

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


def _prep(prob, vreal=False):
    cf = ocanon.canonical(prob)
    V = cf["V"].real.astype(np.float32) if vreal else cf["V"].astype(np.complex64)
    return cf, V, cf["y"].astype(np.complex64)


def _solver(torch, shape, cf, V, **kw):
    from paper_2207_14222_gb300.solver import Solver
    return Solver(shape, cf["a"], cf["b"], torch.from_numpy(V).cuda(), dx=cf["dx"], **kw)


def _lh(shape, cf):
    return uo.lhat(shape, cf["dx"], cf["a"], cf["b"])


def _trajectory(torch, shape, prob, n_iter, vreal=False, **kw):
    cf, V, y = _prep(prob, vreal)
    with _solver(torch, shape, cf, V, plain=True, schedule=3, **kw) as s:
        x, res = s.solve(torch.from_numpy(y).cuda(), tol=0.0, maxit=n_iter)
        hg = s.history()
        xg = x.cpu().numpy().astype(np.complex128)
    V64, y64 = V.astype(np.complex128), y.astype(np.complex128)
    assert res["iterations"] == n_iter and len(hg) == n_iter
    assert res["alpha"] == pytest.approx(uo.alpha_star(V64), rel=1e-6)
    xo, ho = uo.iterate(V64, y64, _lh(shape, cf), res["alpha"], n_iter)
    err = np.linalg.norm(xg - xo) / np.linalg.norm(xo)
    assert err <= TOL_X, err
    far = ho > 1e-3
    assert np.max(np.abs(hg[far] - ho[far]) / ho[far]) <= TOL_HIST
    assert res["ref_norm"] == pytest.approx(uo.reference_norm(y64, V64, _lh(shape, cf)), rel=1e-5)
    return xg


@pytest.mark.parametrize("n", [32, 64, 96, 128, 192, 256])
def test_onchip_trajectory(torch_cuda, n):
    _trajectory(torch_cuda, (n, n), inputs.white_helmholtz((n, n), 200 + n), 40)


def test_onchip_helmholtz_128_workload(torch_cuda):
    """The 2-D 128 x 128 workload (sigma 4 px, amplitude 0.3, ABL 16 px,
    centre point source), 300 iterations."""
    _trajectory(torch_cuda, (128, 128), inputs.helmholtz_2d(128, seed=0), 300)


def test_onchip_real_potential(torch_cuda):
    _trajectory(torch_cuda, (128, 128), inputs.random_diffusion((128, 128), 201, sigma_px=3.0), 60,
                vreal=True)


def test_onchip_fixed_alpha(torch_cuda):
    torch = torch_cuda
    shape = (64, 64)
    cf, V, y = _prep(inputs.random_helmholtz(shape, 202, sigma_px=2.0))
    with _solver(torch, shape, cf, V, alpha=0.8, plain=True, schedule=3) as s:
        x, res = s.solve(torch.from_numpy(y).cuda(), tol=0.0, maxit=50)
    xo, _ = uo.iterate(V.astype(np.complex128), y.astype(np.complex128), _lh(shape, cf), 0.8, 50)
    assert np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo) <= TOL_X


def test_onchip_is_the_automatic_choice_and_matches_pencil(torch_cuda):
    """Schedule 0 takes the on-chip path for square 2-D grids; the pencil
    passes (schedule 1) compute the same iteration."""
    torch = torch_cuda
    shape = (128, 128)
    cf, V, y = _prep(inputs.random_helmholtz(shape, 203, sigma_px=3.0))
    yd = torch.from_numpy(y).cuda()
    out = {}
    for sched in (0, 1):
        with _solver(torch, shape, cf, V, plain=True, schedule=sched) as s:
            x, _ = s.solve(yd, tol=0.0, maxit=80)
            out[sched] = (x.cpu().numpy(), s.history(),
                          [p["name"] for p in s.time_passes(yd, torch.zeros_like(yd), 3)])
    assert out[0][2] == ["onchip_iteration"] and "onchip_iteration" not in out[1][2]
    assert np.linalg.norm(out[0][0] - out[1][0]) / np.linalg.norm(out[1][0]) < 2e-6
    assert np.max(np.abs(out[0][1] - out[1][1]) / out[1][1]) < 1e-5


def test_onchip_solve_with_refinement(torch_cuda):
    """To 1e-6: FP32 phases on chip, the FP64 residual y - A x between them."""
    torch = torch_cuda
    shape = (128, 128)
    cf, V, y = _prep(inputs.helmholtz_2d(128, seed=1))
    with _solver(torch, shape, cf, V, schedule=3) as s:
        x, res = s.solve(torch.from_numpy(y).cuda(), tol=1e-6, maxit=5000,
                         allow_not_converged=False)
    xg = x.cpu().numpy().astype(np.complex128)
    V64, y64 = V.astype(np.complex128), y.astype(np.complex128)
    d = uo.residual_delta(xg, y64, V64, _lh(shape, cf))
    assert np.linalg.norm(d) / res["ref_norm"] < 1.5e-6
    xo, ho, ok = uo.solve(V64, y64, _lh(shape, cf), res["alpha"], 1e-6, 5000)
    assert ok and np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= TOL_X
    assert abs(res["iterations"] - len(ho)) <= max(5, len(ho) // 20)


def test_onchip_warm_start_and_reference_pass(torch_cuda):
    """use_x0 without a reference norm: the reference pass (Delta at x = 0,
    no update) runs on chip, then the phase continues the trajectory."""
    torch = torch_cuda
    shape = (64, 64)
    cf, V, y = _prep(inputs.white_helmholtz(shape, 204))
    yd = torch.from_numpy(y).cuda()
    with _solver(torch, shape, cf, V, plain=True, schedule=3) as s:
        x, r1 = s.solve(yd, tol=0.0, maxit=20)
        x, r2 = s.solve(yd, x=x, use_x0=True, tol=0.0, maxit=20)
        x3, r3 = s.solve(yd, x=x.clone(), use_x0=True, tol=0.0, maxit=5, ref_norm=r1["ref_norm"])
    assert r2["ref_norm"] == pytest.approx(r1["ref_norm"], rel=1e-5)
    assert r3["ref_norm"] == r1["ref_norm"]
    xo, ho = uo.iterate(V.astype(np.complex128), y.astype(np.complex128), _lh(shape, cf),
                        r1["alpha"], 40)
    assert np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo) <= TOL_X


def test_onchip_table_symbol(torch_cuda):
    torch = torch_cuda
    from symbol_tables import stencil_symbol
    shape = (64, 64)
    cf, V, y = _prep(inputs.white_helmholtz(shape, 205))
    drift = (0.6 * abs(cf["a"]), -0.4 * abs(cf["a"]))
    T = stencil_symbol(shape, cf["dx"], cf["a"], cf["b"], drift)
    with _solver(torch, shape, cf, V, plain=True, schedule=3,
                 lhat_table=torch.from_numpy(T).cuda()) as s:
        x, res = s.solve(torch.from_numpy(y).cuda(), tol=0.0, maxit=30)
    xo, _ = uo.iterate(V.astype(np.complex128), y.astype(np.complex128), T.astype(np.complex128),
                       res["alpha"], 30)
    assert np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo) <= TOL_X


def test_onchip_edges(torch_cuda):
    """maxit 1; a zero source converges at once; a non-finite source is
    reported; the history stops at the limit."""
    torch = torch_cuda
    shape = (32, 32)
    cf, V, y = _prep(inputs.random_helmholtz(shape, 206))
    with _solver(torch, shape, cf, V, plain=True, schedule=3) as s:
        x, r = s.solve(torch.from_numpy(y).cuda(), tol=1e-6, maxit=1)
        assert r["status"] == "USP_ERR_NOT_CONVERGED" and r["iterations"] == 1
        xo, _ = uo.iterate(V.astype(np.complex128), y.astype(np.complex128), _lh(shape, cf),
                           r["alpha"], 1)
        assert np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo) <= TOL_X
        z = torch.zeros(shape, dtype=torch.complex64, device="cuda:0")
        x, r = s.solve(z, tol=1e-6, maxit=10)
        assert r["status"] == "USP_OK" and torch.count_nonzero(x).item() == 0
        yb = y.copy()
        yb[3, 5] = np.nan
        with pytest.raises(_lib.UspError) as e:
            s.solve(torch.from_numpy(yb).cuda(), tol=1e-6, maxit=50)
        assert e.value.status == _lib.ERR_NONFINITE
        x, r = s.solve(torch.from_numpy(y).cuda(), tol=0.0, maxit=7)
        assert r["iterations"] == 7 and len(s.history()) == 7


def test_onchip_deterministic(torch_cuda):
    torch = torch_cuda
    shape = (128, 128)
    cf, V, y = _prep(inputs.random_helmholtz(shape, 207))
    outs = []
    for _ in range(2):
        with _solver(torch, shape, cf, V, schedule=3) as s:
            x, r = s.solve(torch.from_numpy(y).cuda(), tol=1e-6, maxit=3000)
            outs.append((x.cpu().numpy(), s.history()))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


def test_onchip_rejected_where_it_does_not_apply(torch_cuda):
    torch = torch_cuda
    for shape in ((64, 128), (384, 384), (16, 16), (8, 32, 32)):
        cf, V, y = _prep(inputs.white_helmholtz(shape, 208))
        with pytest.raises(_lib.UspError) as e:
            _solver(torch, shape, cf, V, schedule=3)
        assert e.value.status == _lib.ERR_UNSUPPORTED_SIZE


def test_onchip_bounded_wait_reports_timeout(torch_cuda):
    """Failure detection without a fault: with the test hook the first exchange
    expects bytes that no CTA sends, every wait gives up after its limit, the
    CTAs meet at the final barrier and the solve reports the timeout; the
    same solver then solves normally (the context is intact)."""
    torch = torch_cuda
    shape = (64, 64)
    cf, V, y = _prep(inputs.white_helmholtz(shape, 209))
    yd = torch.from_numpy(y).cuda()
    with _solver(torch, shape, cf, V, plain=True, schedule=3) as s:
        s.set_options(plain=True, schedule=3, test_wait_fault=True)
        with pytest.raises(_lib.UspError) as e:
            s.solve(yd, tol=1e-6, maxit=50)
        assert e.value.status == _lib.ERR_CUDA and "timed out" in str(e.value)
        s.set_options(plain=True, schedule=3)
        x, res = s.solve(yd, tol=0.0, maxit=20)
    assert res["iterations"] == 20
    xo, _ = uo.iterate(V.astype(np.complex128), y.astype(np.complex128), _lh(shape, cf),
                       res["alpha"], 20)
    assert np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo) <= TOL_X


@pytest.mark.parametrize("n, rows", [(96, 8), (96, 16)])
def test_onchip_radix3_rows_per_cta(torch_cuda, n, rows):
    """Radix-3 lines (96 = 3 x 32) with 8 or 16 rows per CTA (12 or 6 CTAs)."""
    _trajectory(torch_cuda, (n, n), inputs.white_helmholtz((n, n), 210 + rows), 30, onchip_rows=rows)

