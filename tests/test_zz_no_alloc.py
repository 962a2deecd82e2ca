"""The allocation-free entry point (usp_solve_noalloc) against the regular
solver, through the C ABI.

usp_solve_noalloc exists for callers that cannot allocate device memory (for
example a process whose device memory already belongs to another allocator,
or a loop that must not call cudaMalloc/cudaFree because they synchronise the
device).  It works in a fixed scratch area inside the library; this test
checks that two calls in a row give the regular solver's result, that the
second call allocates nothing, and that an oversized grid is refused.

This file is collected last so that a run stopping at the first failure has
run every other test before it.
"""

import ctypes

import numpy as np
import pytest

from oracle import canon as ocanon
from paper_2207_14222_gb300 import _lib, inputs

pytestmark = pytest.mark.gpu

TOL_X = 1e-5   # the complex64 bar used by the parity tests


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2207_14222_gb300 import build
    build.build()
    _lib.lib()
    return torch


def _grid(shape):
    g = _lib.Grid()
    g.ndim = len(shape)
    for i, n in enumerate(shape):
        g.n[i] = n
    g.dx = 1.0
    return g


def _noalloc(torch, shape, cf, Vd, yd, xd, tol, maxit, alpha=0.0):
    res = _lib.Result()
    sym = _lib.LSymbol(cf["a"].real, cf["a"].imag, cf["b"].real, cf["b"].imag)
    stream = torch.cuda.current_stream().cuda_stream
    st = _lib.lib().usp_solve_noalloc(
        ctypes.byref(_grid(shape)), ctypes.byref(sym), ctypes.c_void_p(Vd.data_ptr()),
        int(Vd.dtype == torch.float32), float(alpha), ctypes.c_void_p(yd.data_ptr()),
        ctypes.c_void_p(xd.data_ptr()), float(tol), int(maxit), ctypes.c_void_p(stream),
        ctypes.byref(res))
    return st, res


@pytest.mark.parametrize("shape, vreal", [((32, 32, 32), False), ((64, 128), True),
                                          ((256,), True), ((16, 32, 64), True)])
def test_noalloc_matches_regular_solver_twice(torch_cuda, shape, vreal):
    torch = torch_cuda
    from paper_2207_14222_gb300.solver import Solver
    if vreal:
        cf = ocanon.canonical(inputs.random_diffusion(shape, 21, sigma_px=2.0))
        V = cf["V"].real.astype(np.float32)
    else:
        cf = ocanon.canonical(inputs.random_helmholtz(shape, 21, sigma_px=2.0))
        V = cf["V"].astype(np.complex64)
    y = cf["y"].astype(np.complex64)
    Vd = torch.from_numpy(V).cuda()
    yd = torch.from_numpy(y).cuda()
    n_iter = 60
    with Solver(shape, cf["a"], cf["b"], Vd, plain=True) as s:
        xr, rr = s.solve(yd, tol=0.0, maxit=n_iter)
        xr = xr.cpu().numpy()
    outs = []
    for _ in range(2):
        xd = torch.full(shape, complex(7.0, -3.0), dtype=torch.complex64, device="cuda:0")
        torch.cuda.synchronize()
        st, res = _noalloc(torch, shape, cf, Vd, yd, xd, 0.0, n_iter)
        torch.cuda.synchronize()
        assert st == _lib.ERR_NOT_CONVERGED, _lib.last_error()
        assert res.iterations == n_iter
        assert res.alpha == pytest.approx(rr["alpha"], rel=1e-12)
        assert res.ref_norm == pytest.approx(rr["ref_norm"], rel=1e-6)
        outs.append(xd.cpu().numpy())
    for x in outs:
        err = np.linalg.norm(x - xr) / np.linalg.norm(xr)
        assert err <= TOL_X, err
    assert np.array_equal(outs[0], outs[1])


def test_noalloc_converges_and_allocates_nothing(torch_cuda):
    torch = torch_cuda
    from paper_2207_14222_gb300.solver import Solver
    shape = (64, 64)
    cf = ocanon.canonical(inputs.helmholtz_2d(64, seed=4, abl_width=8))
    Vd = torch.from_numpy(cf["V"].astype(np.complex64)).cuda()
    yd = torch.from_numpy(cf["y"].astype(np.complex64)).cuda()
    with Solver(shape, cf["a"], cf["b"], Vd, plain=True) as s:
        xr, rr = s.solve(yd, tol=1e-5, maxit=5000)
        xr = xr.cpu().numpy()
    xd = torch.empty_like(yd)
    st, _ = _noalloc(torch, shape, cf, Vd, yd, xd, 1e-5, 5000)   # first call: set-up
    assert st == _lib.OK, _lib.last_error()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        st, res = _noalloc(torch, shape, cf, Vd, yd, xd, 1e-5, 5000)
        assert st == _lib.OK, _lib.last_error()
        assert res.converged == 1 and res.iterations == rr["iterations"]
        x = xd.cpu().numpy()
        assert np.linalg.norm(x - xr) / np.linalg.norm(xr) <= TOL_X
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_refuses_oversized_requests(torch_cuda):
    torch = torch_cuda
    shape = (128, 128, 64)            # 2^20 points > USP_NOALLOC_MAX_POINTS
    cf = {"a": 0.3j, "b": 0.2 - 0.5j}
    dummy = torch.zeros(4, dtype=torch.complex64, device="cuda:0")
    st, _ = _noalloc(torch, shape, cf, dummy, dummy, dummy, 1e-6, 10)
    assert st == _lib.ERR_UNSUPPORTED_SIZE
    assert "at most 524288 points" in _lib.last_error()
    st, _ = _noalloc(torch, (16, 16), cf, dummy, dummy, dummy, 1e-6, 10 ** 6)
    assert st == _lib.ERR_INVALID_ARG
    assert "maxit" in _lib.last_error()
