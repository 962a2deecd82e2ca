"""The split-y two-pass schedule (schedule 4: grids nz x 256 x 256) against
the FP64 oracle, through the C ABI.

The rows pass does the x transform and the 16-point y1 stage of each tile
of 16 rows (y = 16 y1 + y2); the column pass the 16-point y2 stage, the z
transform and the multiply.  Every test compares element by element with the
oracle's Algorithm 1 on the same complex64 (or float32) inputs, at the
complex64 bar (rel-L2 1e-5 on x, 1e-4 on the residual history).
"""

import os

import numpy as np
import pytest
import scipy.fft as sfft

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


def _run(torch, shape, cf, V, y, n_iter, schedule=4, **opts):
    from paper_2207_14222_gb300.solver import Solver
    dev = torch.device("cuda:0")
    with Solver(shape, cf["a"], cf["b"], torch.from_numpy(V).to(dev), dx=cf["dx"], plain=True,
                schedule=schedule, **opts) as s:
        x, res = s.solve(torch.from_numpy(y).to(dev), tol=0.0, maxit=n_iter)
        hist = s.history()
        torch.cuda.synchronize()
        return x.cpu().numpy().astype(np.complex128), res, hist


def _check(torch, shape, prob, n_iter, vreal=False, **opts):
    cf, V, y = _prep(prob, vreal)
    xg, res, hg = _run(torch, shape, cf, V, y, n_iter, **opts)
    assert res["iterations"] == n_iter
    Lh = uo.lhat(shape, cf["dx"], cf["a"], cf["b"])
    V64, y64 = V.astype(np.complex128), y.astype(np.complex128)
    assert res["alpha"] == pytest.approx(uo.alpha_star(V64), rel=1e-6)
    # the oracle's transform on every host core (its arithmetic does not
    # depend on the worker count)
    with sfft.set_workers(os.cpu_count() or 1):
        xo, ho = uo.iterate(V64, y64, Lh, res["alpha"], n_iter)
    err = np.linalg.norm(xg - xo) / np.linalg.norm(xo)
    assert err <= TOL_X, err
    far = ho > 1e-3
    herr = np.max(np.abs(hg[far] - ho[far]) / ho[far])
    assert herr <= TOL_HIST, herr
    assert res["ref_norm"] == pytest.approx(uo.reference_norm(y64, V64, Lh), rel=1e-5)
    return xg


@pytest.mark.parametrize("nz", [32, 64, 128])
def test_split_parity_shapes(torch_cuda, nz):
    """Every column-pass variant (nz = 32, 64, 128: 4, 8, 8 threads per
    z column) on an unsmoothed random medium."""
    shape = (nz, 256, 256)
    _check(torch_cuda, shape, inputs.white_helmholtz(shape, 50 + nz), 20)


def test_split_parity_real_potential(torch_cuda):
    shape = (64, 256, 256)
    _check(torch_cuda, shape, inputs.random_diffusion(shape, 51, sigma_px=3.0), 20, vreal=True)


def test_split_parity_full_size_helmholtz(torch_cuda):
    """The benchmark's workload (3-D Helmholtz 256^3, a beam source in one
    plane, so the rows pass copies 0.4% of the source rows) on the split
    schedule, every output compared with the oracle after 20 iterations."""
    shape = (256, 256, 256)
    _check(torch_cuda, shape, inputs.helmholtz_3d(256, seed=0), 20)


def test_split_parity_full_size_diffusion(torch_cuda):
    """The 3-D diffusion workload (real V, a point source) after 20
    iterations."""
    shape = (256, 256, 256)
    _check(torch_cuda, shape, inputs.diffusion_3d(256, seed=0), 20, vreal=True)


def test_split_and_pencil_schedules_agree(torch_cuda):
    """Both schedules compute the same iteration; they differ only in the
    order of FP32 rounding."""
    torch = torch_cuda
    shape = (32, 256, 256)
    cf, V, y = _prep(inputs.random_helmholtz(shape, 52, sigma_px=3.0, abl_width=4))
    x1, r1, h1 = _run(torch, shape, cf, V, y, 50, schedule=1)
    x2, r2, h2 = _run(torch, shape, cf, V, y, 50, schedule=4)
    assert np.linalg.norm(x1 - x2) / np.linalg.norm(x1) < 2e-6
    assert np.max(np.abs(h1 - h2) / h1) < 1e-5


def test_split_warm_start_and_reference_pass(torch_cuda):
    """x0 given (use_x0): the reference norm comes from a separate pass
    (Delta at x = 0, no update), then the iteration continues from x0."""
    torch = torch_cuda
    from paper_2207_14222_gb300.solver import Solver
    shape = (32, 256, 256)
    cf, V, y = _prep(inputs.white_helmholtz(shape, 53))
    dev = torch.device("cuda:0")
    yd = torch.from_numpy(y).to(dev)
    with Solver(shape, cf["a"], cf["b"], torch.from_numpy(V).to(dev), plain=True,
                schedule=4) as s:
        x, r1 = s.solve(yd, tol=0.0, maxit=15)
        x, r2 = s.solve(yd, x=x, use_x0=True, tol=0.0, maxit=15)
    assert r2["ref_norm"] == pytest.approx(r1["ref_norm"], rel=1e-5)
    Lh = uo.lhat(shape, cf["dx"], cf["a"], cf["b"])
    xo, _ = uo.iterate(V.astype(np.complex128), y.astype(np.complex128), Lh, r1["alpha"], 30)
    assert np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo) <= TOL_X


def test_split_table_symbol(torch_cuda):
    """A tabulated symbol (odd in p: a mirrored or transposed frequency
    index fails) through the column pass's multiply."""
    torch = torch_cuda
    from symbol_tables import stencil_symbol
    from paper_2207_14222_gb300.solver import Solver
    shape = (32, 256, 256)
    cf, V, y = _prep(inputs.white_helmholtz(shape, 54))
    drift = tuple(c * abs(cf["a"]) / cf["dx"] for c in (0.6, -0.4, 0.25))
    T = stencil_symbol(shape, cf["dx"], cf["a"], cf["b"], drift)
    dev = torch.device("cuda:0")
    n_iter = 20
    with Solver(shape, 9.0, -0.5, torch.from_numpy(V).to(dev), dx=cf["dx"],
                lhat_table=torch.from_numpy(T).to(dev), plain=True, schedule=4) as s:
        x, res = s.solve(torch.from_numpy(y).to(dev), tol=0.0, maxit=n_iter)
        xg = x.cpu().numpy().astype(np.complex128)
    xo, _ = uo.iterate(V.astype(np.complex128), y.astype(np.complex128),
                       T.astype(np.complex128), res["alpha"], n_iter)
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= TOL_X


def test_split_solve_with_refinement(torch_cuda):
    """FP32 iteration on the split schedule with FP64 refinement, to 1e-6:
    the oracle's preconditioned residual of the returned field is below
    1.5e-6 and the field is within 1e-5 of the oracle's solve."""
    torch = torch_cuda
    from paper_2207_14222_gb300.solver import Solver
    shape = (32, 256, 256)
    cf, V, y = _prep(inputs.random_helmholtz(shape, 55, sigma_px=3.0, abl_width=4))
    dev = torch.device("cuda:0")
    with Solver(shape, cf["a"], cf["b"], torch.from_numpy(V).to(dev), schedule=4) as s:
        x, res = s.solve(torch.from_numpy(y).to(dev), tol=1e-6, maxit=20000,
                         allow_not_converged=False)
        xg = x.cpu().numpy().astype(np.complex128)
    Lh = uo.lhat(shape, cf["dx"], cf["a"], cf["b"])
    V64, y64 = V.astype(np.complex128), y.astype(np.complex128)
    d = uo.residual_delta(xg, y64, V64, Lh)
    assert np.linalg.norm(d) / res["ref_norm"] < 1.5e-6
    xo, _, ok = uo.solve(V64, y64, Lh, res["alpha"], 1e-6, 20000)
    assert ok and np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= TOL_X


def test_split_schedule_refuses_other_grids(torch_cuda):
    torch = torch_cuda
    from paper_2207_14222_gb300.solver import Solver
    for shape in ((16, 256, 256), (32, 128, 256), (64, 64)):
        cf, V, y = _prep(inputs.white_helmholtz(shape, 56))
        with pytest.raises(_lib.UspError):
            Solver(shape, cf["a"], cf["b"], torch.from_numpy(V).cuda(), schedule=4)


def test_split_general_complex_symbol(torch_cuda):
    """A symbol a |p|^2 + b with both a and b complex (neither the Helmholtz
    form, a purely imaginary, nor the real diffusion form) through the column
    pass's general multiply."""
    torch = torch_cuda
    from paper_2207_14222_gb300.solver import Solver
    shape = (32, 256, 256)
    cf, V, y = _prep(inputs.white_helmholtz(shape, 57))
    a, b = complex(0.04, 0.25), complex(0.15, -0.35)
    dev = torch.device("cuda:0")
    n_iter = 20
    with Solver(shape, a, b, torch.from_numpy(V).to(dev), dx=cf["dx"], plain=True,
                schedule=4) as s:
        x, res = s.solve(torch.from_numpy(y).to(dev), tol=0.0, maxit=n_iter)
        xg = x.cpu().numpy().astype(np.complex128)
    Lh = uo.lhat(shape, cf["dx"], a, b)
    xo, _ = uo.iterate(V.astype(np.complex128), y.astype(np.complex128), Lh, res["alpha"], n_iter)
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= TOL_X


def _sparse_rows_source(shape, seed, keep=0.1):
    """A random source with all but a random tenth of its rows (x lines) set
    to zero, so that tiles hold every mix of copied and skipped rows."""
    rng = np.random.default_rng(seed)
    prob = inputs.white_helmholtz(shape, seed)
    rows = rng.uniform(size=shape[:-1]) < keep
    rows[0, 0] = rows[-1, -1] = True
    prob["S"] = prob["S"] * rows[..., None]
    return prob, rows


def test_split_source_row_mask(torch_cuda):
    """The rows pass copies only the source rows that hold a nonzero value;
    the others enter as zeros.  A source with 90% of its rows zero (random
    rows, both ends set) follows the oracle, and the pass's byte count drops
    by the skipped rows' 8 B per point."""
    torch = torch_cuda
    from paper_2207_14222_gb300.solver import Solver
    shape = (32, 256, 256)
    prob, rows = _sparse_rows_source(shape, 58)
    _check(torch, shape, prob, 20)
    cf, V, y = _prep(prob)
    assert np.array_equal(np.any(y != 0, axis=-1), rows)
    dev = torch.device("cuda:0")
    yd = torch.from_numpy(y).to(dev)
    with Solver(shape, cf["a"], cf["b"], torch.from_numpy(V).to(dev), plain=True,
                schedule=4) as s:
        x = torch.zeros_like(yd)
        s.solve(yd, x=x, tol=0.0, maxit=2)
        passes = {p["name"]: p for p in s.time_passes(yd, x, iters=2)}
    npts = int(np.prod(shape))
    expect = (24.0 + 8.0 * rows.mean() + 8.0 + 8.0) * npts   # scratch, x, V (complex)
    assert passes["split_rows_full"]["bytes"] == pytest.approx(expect, rel=1e-12)


def test_split_source_mask_follows_the_source(torch_cuda):
    """The mask is rebuilt from the source at every phase: the same device
    buffer refilled with a different source between two solves gives the
    second source's solution, and a NaN placed in a row that was zero
    before is still reported."""
    torch = torch_cuda
    from paper_2207_14222_gb300.solver import Solver
    shape = (32, 256, 256)
    prob1, _ = _sparse_rows_source(shape, 59, keep=0.02)
    prob2, _ = _sparse_rows_source(shape, 60, keep=0.5)
    cf1, V, y1 = _prep(prob1)
    cf2 = ocanon.canonical(dict(prob2, k2=prob1["k2"]))
    y2 = cf2["y"].astype(np.complex64)
    dev = torch.device("cuda:0")
    yd = torch.from_numpy(y1).to(dev)
    n_iter = 20
    with Solver(shape, cf1["a"], cf1["b"], torch.from_numpy(V).to(dev), plain=True,
                schedule=4) as s:
        s.solve(yd, tol=0.0, maxit=n_iter)
        yd.copy_(torch.from_numpy(y2))
        x, res = s.solve(yd, tol=0.0, maxit=n_iter)
        xg = x.cpu().numpy().astype(np.complex128)
        yb = y2.copy()
        zero_rows = np.argwhere(~np.any(y2 != 0, axis=-1))
        z, yy = zero_rows[len(zero_rows) // 2]
        yb[z, yy, 7] = np.nan
        yd.copy_(torch.from_numpy(yb))
        with pytest.raises(_lib.UspError) as e:
            s.solve(yd, tol=1e-6, maxit=10)
        assert e.value.status == _lib.ERR_NONFINITE
    Lh = uo.lhat(shape, cf1["dx"], cf1["a"], cf1["b"])
    xo, _ = uo.iterate(V.astype(np.complex128), y2.astype(np.complex128), Lh, res["alpha"], n_iter)
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= TOL_X
