"""CUDA path vs the FP64 oracle, through the C ABI.

Both sides get the same inputs: the oracle's canonical V and y rounded to
complex64 (float32 for a real potential), upcast again for the oracle, so
the comparison measures the solver's arithmetic only.

Tolerance: relative L2 error <= 1e-5 on the iterate after the same number
of iterations (the complex64 bar), and 1e-4 relative on the residual
history while it is far above the FP32 floor.
"""

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
    if vreal:
        V = cf["V"].real.astype(np.float32)
    else:
        V = cf["V"].astype(np.complex64)
    y = cf["y"].astype(np.complex64)
    return cf, V, y


def _gpu_iterate(torch, shape, cf, V, y, n_iter, alpha=0.0, schedule=0, **opts):
    from paper_2207_14222_gb300.solver import Solver
    dev = torch.device("cuda:0")
    Vd = torch.from_numpy(V).to(dev)
    yd = torch.from_numpy(y).to(dev)
    with Solver(shape, cf["a"], cf["b"], Vd, alpha=alpha, dx=cf["dx"], plain=True,
                schedule=schedule, **opts) as s:
        x, res = s.solve(yd, tol=0.0, maxit=n_iter)
        hist = s.history()
        torch.cuda.synchronize()
        return x.cpu().numpy().astype(np.complex128), res, hist


def _oracle_iterate(shape, cf, V, y, n_iter, alpha):
    Lh = uo.lhat(shape, cf["dx"], cf["a"], cf["b"])
    return uo.iterate(V.astype(np.complex128), y.astype(np.complex128), Lh, alpha, n_iter)


def _check_trajectory(torch, shape, prob, n_iter, vreal=False, alpha=0.0, schedule=0,
                      tol_x=TOL_X, **opts):
    cf, V, y = _prep(prob, vreal)
    xg, res, hg = _gpu_iterate(torch, shape, cf, V, y, n_iter, alpha, schedule, **opts)
    assert res["iterations"] == n_iter
    a = res["alpha"]
    if alpha <= 0:
        assert a == pytest.approx(uo.alpha_star(V.astype(np.complex128)), rel=1e-6)
    xo, ho = _oracle_iterate(shape, cf, V, y, n_iter, a)
    err = np.linalg.norm(xg - xo) / np.linalg.norm(xo)
    assert err <= tol_x, err
    far = ho > 1e-3
    herr = np.max(np.abs(hg[far] - ho[far]) / ho[far])
    assert herr <= TOL_HIST, herr
    assert res["ref_norm"] == pytest.approx(
        uo.reference_norm(y.astype(np.complex128), V.astype(np.complex128),
                          uo.lhat(shape, cf["dx"], cf["a"], cf["b"])), rel=1e-5)
    return err


# ------------------------------------------------------------- shapes ---

@pytest.mark.parametrize("shape", [(2,), (8,), (256,)])
def test_parity_1d(torch_cuda, shape):
    _check_trajectory(torch_cuda, shape, inputs.white_helmholtz(shape, 1), 40)


@pytest.mark.parametrize("shape", [(2, 2), (4, 32), (16, 256), (256, 8), (64, 64)])
def test_parity_2d_shapes(torch_cuda, shape):
    _check_trajectory(torch_cuda, shape, inputs.white_helmholtz(shape, 2), 30)


def test_parity_2d_helmholtz_128(torch_cuda):
    """The 2-D 128x128 workload (sigma 4 px, amplitude 0.3, ABL 16 px,
    centre point source), 300 iterations."""
    prob = inputs.helmholtz_2d(128, seed=0)
    _check_trajectory(torch_cuda, (128, 128), prob, 300)


@pytest.mark.parametrize("shape", [(2, 4, 8), (8, 16, 32), (32, 32, 32), (16, 2, 64),
                                   (4, 256, 2), (64, 64, 64)])
def test_parity_3d_shapes(torch_cuda, shape):
    _check_trajectory(torch_cuda, shape, inputs.white_helmholtz(shape, 3), 25)


@pytest.mark.parametrize("shape", [(96,), (192,), (384,), (512,),
                                   (96, 96), (192, 128), (384, 32), (512, 64), (64, 512),
                                   (32, 384), (96, 8, 16), (4, 16, 384), (6 * 16, 512, 2)])
def test_parity_radix3_and_512_lengths(torch_cuda, shape):
    """Axis lengths 3 * 2^k and 512, transformed through the radix-3 / radix-2
    outer stage, on every kind of pass (line pass, strided pass, both)."""
    _check_trajectory(torch_cuda, shape, inputs.white_helmholtz(shape, 4), 25)


def test_solve_with_refinement_radix3(torch_cuda):
    """FP32 iteration + FP64 refinement (FP64 transforms of the same lengths)
    on a 192 x 96 medium, to 1e-6, against the oracle's solve."""
    torch = torch_cuda
    from paper_2207_14222_gb300.solver import Solver
    shape = (192, 96)
    cf, V, y = _prep(inputs.random_helmholtz(shape, 21, sigma_px=3.0, amplitude=0.3))
    dev = torch.device("cuda:0")
    with Solver(shape, cf["a"], cf["b"], torch.from_numpy(V).to(dev)) as s:
        x, res = s.solve(torch.from_numpy(y).to(dev), tol=1e-6, maxit=5000,
                         allow_not_converged=False)
        xg = x.cpu().numpy().astype(np.complex128)
    Lh = uo.lhat(shape, cf["dx"], cf["a"], cf["b"])
    V64, y64 = V.astype(np.complex128), y.astype(np.complex128)
    xo, ho, ok = uo.solve(V64, y64, Lh, res["alpha"], 1e-6, 5000)
    assert ok and res["converged"] == 1
    # the correction phase restarts from z = 0 at 8 tol and repeats the slow
    # first steps of a fresh iteration: a few percent more iterations
    assert abs(res["iterations"] - len(ho)) <= max(5, len(ho) // 20)
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= TOL_X
    d = uo.residual_delta(xg, y64, V64, Lh)
    assert np.linalg.norm(d) / res["ref_norm"] < 1.5e-6


def test_parity_3d_helmholtz_64(torch_cuda):
    """The 3-D Helmholtz medium generator at 64^3 (lengths scaled by 1/4)."""
    prob = inputs.helmholtz_3d(64, seed=0)
    _check_trajectory(torch_cuda, (64, 64, 64), prob, 100)


def test_parity_diffusion_real_potential(torch_cuda):
    prob = inputs.random_diffusion((32, 32, 32), 4, sigma_px=2.0)
    _check_trajectory(torch_cuda, (32, 32, 32), prob, 60, vreal=True)
    prob = inputs.random_diffusion((64, 128), 5, sigma_px=3.0)
    _check_trajectory(torch_cuda, (64, 128), prob, 60, vreal=True)


def test_parity_fixed_alpha(torch_cuda):
    prob = inputs.random_helmholtz((32, 64), 6, sigma_px=2.0)
    for alpha in (1.0, 0.7):
        _check_trajectory(torch_cuda, (32, 64), prob, 40, alpha=alpha)


# ----------------------------------------- fused two-pass schedule ---

@pytest.mark.parametrize("nz", [2, 16])
def test_parity_fused_schedule(torch_cuda, nz):
    """Grids nz x 256 x 256 on the plane-cluster + z-pencil schedule."""
    shape = (nz, 256, 256)
    _check_trajectory(torch_cuda, shape, inputs.white_helmholtz(shape, 30 + nz), 20, schedule=2)


def test_parity_fused_real_potential(torch_cuda):
    shape = (8, 256, 256)
    prob = inputs.random_diffusion(shape, 33, sigma_px=3.0)
    _check_trajectory(torch_cuda, shape, prob, 20, vreal=True, schedule=2)


def test_fused_and_pencil_schedules_agree(torch_cuda):
    """Both schedules compute the same iteration; they differ only in the
    order of FP32 rounding."""
    torch = torch_cuda
    shape = (32, 256, 256)
    cf, V, y = _prep(inputs.random_helmholtz(shape, 34, sigma_px=3.0, abl_width=4))
    x1, r1, h1 = _gpu_iterate(torch, shape, cf, V, y, 50, schedule=1)
    x2, r2, h2 = _gpu_iterate(torch, shape, cf, V, y, 50, schedule=2)
    assert np.linalg.norm(x1 - x2) / np.linalg.norm(x1) < 2e-6
    assert np.max(np.abs(h1 - h2) / h1) < 1e-5


def test_fused_warm_start_and_reference_pass(torch_cuda):
    torch = torch_cuda
    from paper_2207_14222_gb300.solver import Solver
    shape = (4, 256, 256)
    cf, V, y = _prep(inputs.white_helmholtz(shape, 35))
    dev = torch.device("cuda:0")
    yd = torch.from_numpy(y).to(dev)
    with Solver(shape, cf["a"], cf["b"], torch.from_numpy(V).to(dev), plain=True,
                schedule=2) as s:
        x, r1 = s.solve(yd, tol=0.0, maxit=15)
        x, r2 = s.solve(yd, x=x, use_x0=True, tol=0.0, maxit=15)   # reference pass
    assert r2["ref_norm"] == pytest.approx(r1["ref_norm"], rel=1e-5)
    xo, _ = _oracle_iterate(shape, cf, V, y, 30, r1["alpha"])
    assert np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo) <= TOL_X


@pytest.mark.parametrize("schedule", [0, 1])
def test_parity_full_size_256_bench_configuration(torch_cuda, schedule):
    """The benchmark's workload (3-D Helmholtz 256^3) in the benchmark's
    launch configuration (automatic schedule: the split-y passes) and on the
    pencil passes, every output compared with the oracle after 3 iterations."""
    shape = (256, 256, 256)
    prob = inputs.helmholtz_3d(256, seed=0)
    _check_trajectory(torch_cuda, shape, prob, 3, schedule=schedule)


@pytest.mark.parametrize("schedule", [0, 1])
def test_parity_full_size_256_diffusion(torch_cuda, schedule):
    """The second full-size workload (3-D steady diffusion 256^3, Sec. 3.2 in
    its scalar form: real float32 V), automatic schedule (split-y) and the
    pencil passes, every output compared with the oracle after 4 iterations."""
    shape = (256, 256, 256)
    prob = inputs.diffusion_3d(256, seed=0)
    _check_trajectory(torch_cuda, shape, prob, 4, vreal=True, schedule=schedule)


@pytest.mark.parametrize("workload", ["helmholtz", "diffusion"])
def test_full_size_256_solve_reaches_tolerance(torch_cuda, workload):
    """The benchmark's solve at 256^3 (FP32 iteration with FP64 refinement,
    automatic schedule) to 1e-6: the oracle's own preconditioned residual of
    the returned field (one FP64 evaluation of Algorithm 1's Delta) is below
    1.5e-6 of the oracle's reference norm, and the reported reference norm
    matches the oracle's."""
    torch = torch_cuda
    from paper_2207_14222_gb300.solver import Solver
    shape = (256, 256, 256)
    if workload == "helmholtz":
        cf, V, y = _prep(inputs.helmholtz_3d(256, seed=0))
    else:
        cf, V, y = _prep(inputs.diffusion_3d(256, seed=0), vreal=True)
    dev = torch.device("cuda:0")
    with Solver(shape, cf["a"], cf["b"], torch.from_numpy(V).to(dev), dx=cf["dx"]) as s:
        x, res = s.solve(torch.from_numpy(y).to(dev), tol=1e-6, maxit=20000,
                         allow_not_converged=False)
        torch.cuda.synchronize()
        xg = x.cpu().numpy().astype(np.complex128)
    del x
    assert res["converged"] == 1 and res["final_rel_residual"] < 1e-6
    Lh = uo.lhat(shape, cf["dx"], cf["a"], cf["b"])
    V64, y64 = V.astype(np.complex128), y.astype(np.complex128)
    ref = uo.reference_norm(y64, V64, Lh)
    assert res["ref_norm"] == pytest.approx(ref, rel=1e-5)
    d = uo.residual_delta(xg, y64, V64, Lh)
    assert np.linalg.norm(d) / ref < 1.5e-6


# The TF32 three-product split rounds each 16-point stage at about twice
# FP32's error, so the raw trajectory gets 5e-5; the path's bar (1e-5 to the
# oracle) applies after refinement, in the converged-solve test below.
TOL_TC = 5e-5


@pytest.mark.parametrize("shape", [(256, 64), (256, 8, 32), (256, 256, 16)])
def test_parity_tensor_core_dft(torch_cuda, shape):
    """The 256-point strided-axis transforms on the tensor cores (TF32 split
    into three products): the oracle's trajectory on 2-D and 3-D grids (one
    or both strided axes of length 256)."""
    _check_trajectory(torch_cuda, shape, inputs.random_helmholtz(shape, 31), 25,
                      tol_x=TOL_TC, tc_dft=True)


def test_parity_tensor_core_dft_bench_configuration(torch_cuda):
    shape = (256, 256, 256)
    _check_trajectory(torch_cuda, shape, inputs.helmholtz_3d(256, seed=0), 3, tol_x=TOL_TC,
                      tc_dft=True)


def test_tensor_core_dft_solve_with_refinement(torch_cuda):
    """To 1e-6 with the tensor-core transforms and FP64 refinement: the
    oracle's preconditioned residual of the result is below 1.5e-6."""
    torch = torch_cuda
    from paper_2207_14222_gb300.solver import Solver
    shape = (256, 128)
    cf, V, y = _prep(inputs.random_helmholtz(shape, 32, sigma_px=4.0))
    dev = torch.device("cuda:0")
    with Solver(shape, cf["a"], cf["b"], torch.from_numpy(V).to(dev), tc_dft=True) as s:
        x, res = s.solve(torch.from_numpy(y).to(dev), tol=1e-6, maxit=20000,
                         allow_not_converged=False)
    Lh = uo.lhat(shape, cf["dx"], cf["a"], cf["b"])
    xg = x.cpu().numpy().astype(np.complex128)
    V64, y64 = V.astype(np.complex128), y.astype(np.complex128)
    d = uo.residual_delta(xg, y64, V64, Lh)
    assert np.linalg.norm(d) / res["ref_norm"] < 1.5e-6
    # the tensor-core path's bar: within 1e-5 of the oracle's solve after refinement
    xo, _, ok = uo.solve(V64, y64, Lh, res["alpha"], 1e-6, 20000)
    assert ok and np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= TOL_X


# ------------------------------------------------------ full solves ---

def test_solve_to_tolerance_with_refinement(torch_cuda):
    """GPU (FP32 + FP64 refinement) to 1e-6 against the oracle's solve to
    the same tolerance: same iteration count within a few, same field."""
    torch = torch_cuda
    from paper_2207_14222_gb300.solver import Solver
    shape = (128, 128)
    cf, V, y = _prep(inputs.helmholtz_2d(128, seed=1))
    dev = torch.device("cuda:0")
    with Solver(shape, cf["a"], cf["b"], torch.from_numpy(V).to(dev)) as s:
        x, res = s.solve(torch.from_numpy(y).to(dev), tol=1e-6, maxit=5000,
                         allow_not_converged=False)
        xg = x.cpu().numpy().astype(np.complex128)
        hg = s.history()
        _, rel = s.residual(x, torch.from_numpy(y).to(dev))
    assert res["converged"] == 1 and res["final_rel_residual"] < 1e-6
    Lh = uo.lhat(shape, cf["dx"], cf["a"], cf["b"])
    V64, y64 = V.astype(np.complex128), y.astype(np.complex128)
    xo, ho, ok = uo.solve(V64, y64, Lh, res["alpha"], 1e-6, 5000)
    assert ok
    # the refinement restart may shift the stopping step by a few iterations
    assert abs(res["iterations"] - len(ho)) <= max(5, len(ho) // 50)
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= TOL_X
    # the true preconditioned residual of the returned field
    d = uo.residual_delta(xg, y64, V64, Lh)
    assert np.linalg.norm(d) / res["ref_norm"] < 1.5e-6
    assert rel == pytest.approx(uo.relative_residual(xg, y64, V64, Lh), rel=1e-3)
    assert len(hg) == res["iterations"]


def test_plain_mode_reports_stagnation_floor(torch_cuda):
    """Plain FP32 Algorithm 1 with a tolerance below its rounding floor ends
    NOT_CONVERGED at maxit, x still valid (close to the oracle's)."""
    torch = torch_cuda
    from paper_2207_14222_gb300.solver import Solver
    shape = (64, 64)
    cf, V, y = _prep(inputs.helmholtz_2d(64, seed=2, abl_width=8))
    dev = torch.device("cuda:0")
    with Solver(shape, cf["a"], cf["b"], torch.from_numpy(V).to(dev), plain=True) as s:
        x, res = s.solve(torch.from_numpy(y).to(dev), tol=1e-12, maxit=600)
    assert res["status"] == "USP_ERR_NOT_CONVERGED" and res["iterations"] == 600
    Lh = uo.lhat(shape, cf["dx"], cf["a"], cf["b"])
    xo, _, _ = uo.solve(V.astype(np.complex128), y.astype(np.complex128), Lh, res["alpha"],
                        1e-10, 5000)
    xg = x.cpu().numpy()
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) < 1e-4


def test_warm_start_continues_trajectory(torch_cuda):
    """x0 from 40 iterations + 40 more with the stored reference norm equals
    80 oracle iterations; with ref_norm <= 0 the reference pass recomputes
    ||B (L+I)^-1 y|| (Algorithm 1's denominator)."""
    torch = torch_cuda
    from paper_2207_14222_gb300.solver import Solver
    shape = (32, 32, 32)
    cf, V, y = _prep(inputs.random_helmholtz(shape, 9, sigma_px=2.0))
    dev = torch.device("cuda:0")
    yd = torch.from_numpy(y).to(dev)
    with Solver(shape, cf["a"], cf["b"], torch.from_numpy(V).to(dev), plain=True) as s:
        x, r1 = s.solve(yd, tol=0.0, maxit=40)
        x, r2 = s.solve(yd, x=x, use_x0=True, tol=0.0, maxit=40, ref_norm=r1["ref_norm"])
        x2 = x.clone()
        _, r3 = s.solve(yd, x=x2, use_x0=True, tol=0.0, maxit=1)
    xo, ho = _oracle_iterate(shape, cf, V, y, 80, r1["alpha"])
    assert np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo) <= TOL_X
    assert r3["ref_norm"] == pytest.approx(r1["ref_norm"], rel=1e-5)


def test_host_api_matches_device_api(torch_cuda):
    torch = torch_cuda
    from paper_2207_14222_gb300.solver import Solver
    shape = (64, 64)
    cf, V, y = _prep(inputs.helmholtz_2d(64, seed=3, abl_width=8))
    dev = torch.device("cuda:0")
    with Solver(shape, cf["a"], cf["b"], torch.from_numpy(V).to(dev)) as s:
        xd, rd = s.solve(torch.from_numpy(y).to(dev), tol=1e-6, maxit=3000)
        yh = torch.from_numpy(y).pin_memory()
        xh = torch.empty_like(yh).pin_memory()
        xh, rh = s.solve_host(yh, xh, tol=1e-6, maxit=3000)
    assert rd["iterations"] == rh["iterations"]
    assert torch.equal(xd.cpu(), xh)


def test_deterministic(torch_cuda):
    torch = torch_cuda
    from paper_2207_14222_gb300.solver import Solver
    shape = (16, 32, 64)
    cf, V, y = _prep(inputs.random_helmholtz(shape, 10))
    dev = torch.device("cuda:0")
    out = []
    for _ in range(2):
        with Solver(shape, cf["a"], cf["b"], torch.from_numpy(V).to(dev)) as s:
            x, r = s.solve(torch.from_numpy(y).to(dev), tol=1e-5, maxit=2000)
            out.append((x.cpu(), s.history()))
    assert torch.equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])


def test_apply_A_and_residual_fp64(torch_cuda):
    torch = torch_cuda
    from paper_2207_14222_gb300.solver import Solver
    for shape, vreal in (((128,), False), ((32, 64), False), ((16, 16, 32), True)):
        if vreal:
            cf, V, y = _prep(inputs.random_diffusion(shape, 11), vreal=True)
        else:
            cf, V, y = _prep(inputs.random_helmholtz(shape, 11))
        x = inputs.random_field(shape, 12).astype(np.complex64)
        dev = torch.device("cuda:0")
        with Solver(shape, cf["a"], cf["b"], torch.from_numpy(V).to(dev)) as s:
            Ax = s.apply_A(torch.from_numpy(x).to(dev)).cpu().numpy()
            r, rel = s.residual(torch.from_numpy(x).to(dev), torch.from_numpy(y).to(dev))
        Lh = uo.lhat(shape, cf["dx"], cf["a"], cf["b"])
        Ao = uo.apply_A(x.astype(np.complex128), V.astype(np.complex128), Lh)
        assert np.linalg.norm(Ax - Ao) / np.linalg.norm(Ao) < 1e-6
        ro = y.astype(np.complex128) - Ao
        assert np.linalg.norm(r.cpu().numpy() - ro) / np.linalg.norm(ro) < 1e-6
        assert rel == pytest.approx(np.linalg.norm(ro) / np.linalg.norm(y), rel=1e-9)


@pytest.mark.parametrize("fp64", [False, True])
def test_refinement_residual_below_fp32_rounding(torch_cuda, fp64):
    """The refinement residual r = y - A x with y = A x up to complex64
    rounding, so that ||r|| is about 1e-7 ||y||: r comes out right only if
    the residual's arithmetic carries far more than FP32 (the same residual
    with complex64 transforms is checked to miss it).  Double-float (default)
    and FP64; line lengths 384 (radix-3 lines), 96 x 128, 8 x 192 x 256 and
    16 x 32 x 64 with a real V."""
    torch = torch_cuda
    import scipy.fft as sfft
    from paper_2207_14222_gb300.solver import Solver
    dev = torch.device("cuda:0")
    cases = ((384,), False), ((96, 128), False), ((8, 192, 256), False), ((16, 32, 64), True)
    for shape, vreal in cases:
        if vreal:
            cf, V, _ = _prep(inputs.random_diffusion(shape, 21), vreal=True)
        else:
            cf, V, _ = _prep(inputs.random_helmholtz(shape, 21))
        Lh = uo.lhat(shape, cf["dx"], cf["a"], cf["b"])
        x = inputs.random_field(shape, 22).astype(np.complex64)
        x64, V64 = x.astype(np.complex128), V.astype(np.complex128)
        y = uo.apply_A(x64, V64, Lh).astype(np.complex64)
        y64 = y.astype(np.complex128)
        ro = y64 - uo.apply_A(x64, V64, Lh)
        rel_o = np.linalg.norm(ro) / np.linalg.norm(y64)
        assert 1e-9 < rel_o < 1e-6, rel_o
        # complex64 transforms cannot resolve it
        r32 = y - (sfft.ifftn(Lh.astype(np.complex64) * sfft.fftn(x)) + V.astype(np.complex64) * x)
        assert np.linalg.norm(r32 - ro) / np.linalg.norm(ro) > 0.1
        with Solver(shape, cf["a"], cf["b"], torch.from_numpy(V).to(dev), dx=cf["dx"],
                    residual_fp64=fp64) as s:
            r, rel = s.residual(torch.from_numpy(x).to(dev), torch.from_numpy(y).to(dev))
        r = r.cpu().numpy()
        assert np.linalg.norm(r - ro) / np.linalg.norm(ro) < 1e-3, shape
        assert rel == pytest.approx(rel_o, rel=1e-3)


def test_refinement_residual_full_size(torch_cuda):
    """The refinement residual at the benchmark's size (3-D Helmholtz 256^3,
    double-float arithmetic, the automatic schedule's solver): y = A x up to
    complex64 rounding, r within 1e-3 of the FP64 oracle's."""
    torch = torch_cuda
    import os
    import scipy.fft as sfft
    from paper_2207_14222_gb300.solver import Solver
    shape = (256, 256, 256)
    cf, V, _ = _prep(inputs.helmholtz_3d(256, seed=0))
    Lh = uo.lhat(shape, cf["dx"], cf["a"], cf["b"])
    x = inputs.random_field(shape, 23).astype(np.complex64)
    x64, V64 = x.astype(np.complex128), V.astype(np.complex128)
    with sfft.set_workers(os.cpu_count() or 1):
        y = uo.apply_A(x64, V64, Lh).astype(np.complex64)
        y64 = y.astype(np.complex128)
        ro = y64 - uo.apply_A(x64, V64, Lh)
    dev = torch.device("cuda:0")
    with Solver(shape, cf["a"], cf["b"], torch.from_numpy(V).to(dev), dx=cf["dx"]) as s:
        r, rel = s.residual(torch.from_numpy(x).to(dev), torch.from_numpy(y).to(dev))
    r = r.cpu().numpy()
    assert np.linalg.norm(r - ro) / np.linalg.norm(ro) < 1e-3
    assert rel == pytest.approx(np.linalg.norm(ro) / np.linalg.norm(y64), rel=1e-3)


# ------------------------------------------------------ edge cases ---

def _solver(torch, shape, cf, V, **kw):
    from paper_2207_14222_gb300.solver import Solver
    return Solver(shape, cf["a"], cf["b"], torch.from_numpy(V).to("cuda:0"), **kw)


def test_edge_maxit_one_and_zero_source(torch_cuda):
    torch = torch_cuda
    shape = (16, 16)
    cf, V, y = _prep(inputs.random_helmholtz(shape, 13))
    with _solver(torch, shape, cf, V, plain=True) as s:
        x, r = s.solve(torch.from_numpy(y).cuda(), tol=1e-6, maxit=1)
        assert r["status"] == "USP_ERR_NOT_CONVERGED" and r["iterations"] == 1
        xo, _ = _oracle_iterate(shape, cf, V, y, 1, r["alpha"])
        assert np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo) < TOL_X
        z = torch.zeros(shape, dtype=torch.complex64, device="cuda:0")
        x, r = s.solve(z, tol=1e-6, maxit=10)
        assert r["status"] == "USP_OK" and r["converged"] == 1
        assert torch.count_nonzero(x).item() == 0


def test_edge_nonfinite_source_and_potential(torch_cuda):
    torch = torch_cuda
    shape = (8, 32)
    cf, V, y = _prep(inputs.random_helmholtz(shape, 14))
    yb = y.copy()
    yb[3, 5] = np.nan
    with _solver(torch, shape, cf, V) as s:
        with pytest.raises(_lib.UspError) as e:
            s.solve(torch.from_numpy(yb).cuda(), tol=1e-6, maxit=50)
        assert e.value.status == _lib.ERR_NONFINITE
    Vb = V.copy()
    Vb[0, 0] = np.inf
    with pytest.raises(_lib.UspError) as e:
        _solver(torch, shape, cf, Vb)
    assert e.value.status == _lib.ERR_NONFINITE


def test_edge_potential_not_contractive(torch_cuda):
    torch = torch_cuda
    shape = (8, 8)
    cf, V, y = _prep(inputs.random_helmholtz(shape, 15))
    with pytest.raises(_lib.UspError) as e:
        _solver(torch, shape, cf, (V * 1.1).astype(np.complex64))
    assert e.value.status == _lib.ERR_V_NOT_CONTRACTIVE


def test_edge_non_accretive_diverges(torch_cuda):
    """A = L + V with Re A < 0 everywhere (outside Thm 1): the iteration
    grows and the solver reports USP_ERR_DIVERGED."""
    torch = torch_cuda
    shape = (16, 16)
    rng = np.random.default_rng(16)
    V = (0.1 + 0.05 * rng.uniform(size=shape)).astype(np.float32)
    y = inputs.random_field(shape, 17).astype(np.complex64)
    from paper_2207_14222_gb300.solver import Solver
    with Solver(shape, 0.0, -0.5, torch.from_numpy(V).cuda(), alpha=1.0, plain=True) as s:
        with pytest.raises(_lib.UspError) as e:
            s.solve(torch.from_numpy(y).cuda(), tol=1e-6, maxit=500)
    assert e.value.status == _lib.ERR_DIVERGED


def test_residual_history_is_monotone(torch_cuda):
    """Thm 1: ||Delta_i|| decreases monotonically (until the FP32 floor)."""
    torch = torch_cuda
    shape = (64, 64, 64)
    cf, V, y = _prep(inputs.helmholtz_3d(64, seed=1))
    with _solver(torch, shape, cf, V, plain=True) as s:
        s.solve(torch.from_numpy(y).cuda(), tol=1e-5, maxit=2000)
        h = s.history()
    h = h[h > 2e-5]
    assert np.all(np.diff(h) < 0)
