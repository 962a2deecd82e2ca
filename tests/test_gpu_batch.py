"""Batches of problems on one grid (usp_batch_create / usp_batch_solve)
against the FP64 oracle, problem by problem, through the C ABI.

Every problem of a batch has its own medium, symbol, step, convergence test
and refinement; each must follow the trajectory the oracle computes for it
alone (relative L2 <= 1e-5 on the iterate, 1e-4 on the residual history far
above the FP32 floor), and a converged batch must agree with solving each
problem on its own.
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


def _prep(probs, vreal=False):
    cfs, Vs, ys = [], [], []
    for prob in probs:
        cf = ocanon.canonical(prob)
        cfs.append(cf)
        Vs.append(cf["V"].real.astype(np.float32) if vreal else cf["V"].astype(np.complex64))
        ys.append(cf["y"].astype(np.complex64))
    return cfs, np.stack(Vs), np.stack(ys)


def _batch(torch, shape, cfs, V, **kw):
    from paper_2207_14222_gb300.solver import BatchSolver
    return BatchSolver(shape, [cf["a"] for cf in cfs], [cf["b"] for cf in cfs],
                       torch.from_numpy(V).to("cuda:0"), dx=cfs[0]["dx"], **kw)


def _lh(shape, cf):
    return uo.lhat(shape, cf["dx"], cf["a"], cf["b"])


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _check_trajectories(torch, shape, probs, n_iter, vreal=False, schedule=0):
    cfs, V, y = _prep(probs, vreal)
    with _batch(torch, shape, cfs, V, plain=True, schedule=schedule) as s:
        x, res = s.solve(torch.from_numpy(y).to("cuda:0"), tol=0.0, maxit=n_iter)
        hists = [s.history(j) for j in range(len(probs))]
        xg = x.cpu().numpy().astype(np.complex128)
    for j, cf in enumerate(cfs):
        r = res[j]
        assert r["iterations"] == n_iter and len(hists[j]) == n_iter
        V64, y64 = V[j].astype(np.complex128), y[j].astype(np.complex128)
        assert r["alpha"] == pytest.approx(uo.alpha_star(V64), rel=1e-6)
        xo, ho = uo.iterate(V64, y64, _lh(shape, cf), r["alpha"], n_iter)
        assert _rel(xg[j], xo) <= TOL_X, (j, _rel(xg[j], xo))
        far = ho > 1e-3
        herr = np.max(np.abs(hists[j][far] - ho[far]) / ho[far])
        assert herr <= TOL_HIST, (j, herr)
        assert r["ref_norm"] == pytest.approx(uo.reference_norm(y64, V64, _lh(shape, cf)),
                                              rel=1e-5)


@pytest.mark.parametrize("shape, count, schedule", [
    ((64, 64), 5, 1),          # plain line passes
    ((128, 128), 3, 1),        # staged line pass, 2 tiles per problem
    ((16, 64, 64), 2, 0),
    ((8, 128, 128), 2, 0),     # staged line and column passes
    ((96, 96), 3, 1),          # radix-3 lines
    ((96, 96), 3, 0),          # on-chip, radix-3 lines
    ((192, 192), 2, 0),
    ((512, 64), 2, 0),         # radix-2 outer stage on the strided axis
    ((16, 512), 3, 1),         # staged 512-point line pass, two 8-row tiles per problem
    ((32, 384), 2, 1),         # staged 384-point line pass, four 8-row tiles per problem
    ((64, 64), 5, 0),          # on-chip: one cluster per problem
    ((128, 128), 3, 0),
    ((256, 256), 2, 0),
])
def test_batch_trajectories_match_oracle(torch_cuda, shape, count, schedule):
    probs = [inputs.random_helmholtz(shape, 100 + j, sigma_px=2.0 + j,
                                     amplitude=0.1 + 0.1 * j) for j in range(count)]
    _check_trajectories(torch_cuda, shape, probs, 30, schedule=schedule)


def test_batch_full_size_problems_256(torch_cuda):
    """Two 256 x 256 problems: staged 32-line tiles, 8 per problem."""
    probs = [inputs.helmholtz_2d(256, seed=j, abl_width=32) for j in range(2)]
    _check_trajectories(torch_cuda, (256, 256), probs, 40)


def test_batch_diffusion_real_potential(torch_cuda):
    probs = [inputs.random_diffusion((64, 128), 20 + j, sigma_px=2.0 + j,
                                     median_eta=0.02 + 0.02 * j) for j in range(3)]
    _check_trajectories(torch_cuda, (64, 128), probs, 40, vreal=True)


def test_batch_mixed_kinds_converge_like_single_solves(torch_cuda):
    """Helmholtz media of different contrast and a diffusion problem (real V
    stored as complex) in one batch, solved to 1e-6 with refinement: every
    problem stops at its own iteration count, and matches both the solve of
    that problem alone and the oracle's solve."""
    torch = torch_cuda
    from paper_2207_14222_gb300.solver import Solver
    shape = (128, 128)
    probs = [inputs.helmholtz_2d(128, seed=1),
             inputs.helmholtz_2d(128, seed=2, amplitude=0.1),
             inputs.random_diffusion(shape, 3, sigma_px=4.0),
             inputs.helmholtz_2d(128, seed=4, amplitude=0.2, abl_width=8)]
    cfs, V, y = _prep(probs)
    dev = torch.device("cuda:0")
    with _batch(torch, shape, cfs, V) as s:
        x, res = s.solve(torch.from_numpy(y).to(dev), tol=1e-6, maxit=5000,
                         allow_failed=False)
        hists = [s.history(j) for j in range(len(probs))]
        xb = x.cpu().numpy().astype(np.complex128)
    its = [r["iterations"] for r in res]
    assert len(set(its)) > 1, its   # the problems really stop independently
    for j, cf in enumerate(cfs):
        r = res[j]
        assert r["converged"] == 1 and r["final_rel_residual"] < 1e-6
        assert len(hists[j]) == r["iterations"]
        with Solver(shape, cf["a"], cf["b"], torch.from_numpy(V[j]).to(dev)) as s1:
            x1, r1 = s1.solve(torch.from_numpy(y[j]).to(dev), tol=1e-6, maxit=5000)
        # same arithmetic; only the order of the norm's partial sums differs
        assert abs(r1["iterations"] - r["iterations"]) <= 2, (j, r1["iterations"], its)
        assert r1["refinements"] == r["refinements"]
        assert _rel(xb[j], x1.cpu().numpy().astype(np.complex128)) <= 2e-6
        V64, y64 = V[j].astype(np.complex128), y[j].astype(np.complex128)
        xo, ho, ok = uo.solve(V64, y64, _lh(shape, cf), r["alpha"], 1e-6, 5000)
        assert ok
        assert _rel(xb[j], xo) <= TOL_X
        d = uo.residual_delta(xb[j], y64, V64, _lh(shape, cf))
        assert np.linalg.norm(d) / r["ref_norm"] < 1.5e-6


def test_batch_of_one_is_the_single_solver(torch_cuda):
    torch = torch_cuda
    from paper_2207_14222_gb300.solver import Solver
    shape = (16, 32, 64)
    cfs, V, y = _prep([inputs.random_helmholtz(shape, 30)])
    dev = torch.device("cuda:0")
    with _batch(torch, shape, cfs, V) as s:
        xb, rb = s.solve(torch.from_numpy(y).to(dev), tol=1e-5, maxit=2000)
        hb = s.history(0)
    with Solver(shape, cfs[0]["a"], cfs[0]["b"], torch.from_numpy(V[0]).to(dev)) as s1:
        x1, r1 = s1.solve(torch.from_numpy(y[0]).to(dev), tol=1e-5, maxit=2000)
        h1 = s1.history()
    assert rb[0]["iterations"] == r1["iterations"]
    assert torch.equal(xb[0].cpu(), x1.cpu())
    assert np.array_equal(hb, h1)


def test_batch_failures_stay_in_their_problem(torch_cuda):
    """A non-finite source in one problem and a zero source in another:
    those two end with their own status, the rest converge unchanged."""
    torch = torch_cuda
    shape = (64, 64)
    probs = [inputs.random_helmholtz(shape, 40 + j) for j in range(4)]
    cfs, V, y = _prep(probs)
    y[1, 10, 10] = np.nan
    y[2] = 0
    dev = torch.device("cuda:0")
    with _batch(torch, shape, cfs, V) as s:
        x, res = s.solve(torch.from_numpy(y).to(dev), tol=1e-6, maxit=3000)
        xb = x.cpu().numpy().astype(np.complex128)
    assert [r["status"] for r in res] == ["USP_OK", "USP_ERR_NONFINITE", "USP_OK", "USP_OK"]
    assert np.count_nonzero(xb[2]) == 0 and res[2]["converged"] == 1
    for j in (0, 3):
        V64, y64 = V[j].astype(np.complex128), y[j].astype(np.complex128)
        xo, _, ok = uo.solve(V64, y64, _lh(shape, cfs[j]), res[j]["alpha"], 1e-6, 5000)
        assert ok and _rel(xb[j], xo) <= TOL_X
    with pytest.raises(_lib.UspError) as e:
        with _batch(torch, shape, cfs, V) as s:
            s.solve(torch.from_numpy(y).to(dev), tol=1e-6, maxit=3000, allow_failed=False)
    assert e.value.status == _lib.ERR_NONFINITE and "problem 1" in str(e.value)


def test_batch_rejects_bad_problem_potential(torch_cuda):
    torch = torch_cuda
    shape = (64, 64)
    cfs, V, y = _prep([inputs.random_helmholtz(shape, 50 + j) for j in range(3)])
    Vb = V.copy()
    Vb[2, 3, 3] = 1.5
    with pytest.raises(_lib.UspError) as e:
        _batch(torch, shape, cfs, Vb)
    assert e.value.status == _lib.ERR_V_NOT_CONTRACTIVE and "problem 2" in str(e.value)
    with _batch(torch, shape, cfs, V) as s:
        r = _lib.Result()
        yd = torch.from_numpy(y).cuda()
        st = _lib.lib().usp_solve(s._h, yd.data_ptr(), yd.data_ptr(), 0, 1e-6, 10, 0.0, r)
        assert st == _lib.ERR_INVALID_ARG


def test_batch_warm_start_and_reference_norms(torch_cuda):
    """40 + 40 iterations with stored reference norms equal 80 oracle
    iterations; with one norm given and one left automatic, the reference
    pass recomputes only the missing one."""
    torch = torch_cuda
    shape = (32, 64)
    cfs, V, y = _prep([inputs.random_helmholtz(shape, 60 + j, sigma_px=2.0 + j)
                       for j in range(2)])
    yd = torch.from_numpy(y).to("cuda:0")
    with _batch(torch, shape, cfs, V, plain=True) as s:
        x, r1 = s.solve(yd, tol=0.0, maxit=40)
        refs = [r["ref_norm"] for r in r1]
        x, r2 = s.solve(yd, x=x, use_x0=True, tol=0.0, maxit=40, ref_norms=refs)
        xg = x.cpu().numpy().astype(np.complex128)
        x3 = x.clone()
        _, r3 = s.solve(yd, x=x3, use_x0=True, tol=0.0, maxit=1, ref_norms=[refs[0], 0.0])
    for j, cf in enumerate(cfs):
        xo, _ = uo.iterate(V[j].astype(np.complex128), y[j].astype(np.complex128),
                           _lh(shape, cf), r1[j]["alpha"], 80)
        assert _rel(xg[j], xo) <= TOL_X
        assert r3[j]["ref_norm"] == pytest.approx(refs[j], rel=1e-5)


def test_batch_apply_A_and_residual(torch_cuda):
    torch = torch_cuda
    shape = (32, 64)
    cfs, V, y = _prep([inputs.random_helmholtz(shape, 70 + j) for j in range(3)])
    x = np.stack([inputs.random_field(shape, 80 + j) for j in range(3)]).astype(np.complex64)
    with _batch(torch, shape, cfs, V) as s:
        Ax = s.apply_A(torch.from_numpy(x).cuda()).cpu().numpy()
        r, rel = s.residual(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda())
        r = r.cpu().numpy()
    num = den = 0.0
    for j, cf in enumerate(cfs):
        Ao = uo.apply_A(x[j].astype(np.complex128), V[j].astype(np.complex128), _lh(shape, cf))
        assert _rel(Ax[j], Ao) < 1e-6
        ro = y[j].astype(np.complex128) - Ao
        assert _rel(r[j], ro) < 1e-6
        num += np.linalg.norm(ro) ** 2
        den += np.linalg.norm(y[j].astype(np.complex128)) ** 2
    assert rel == pytest.approx(np.sqrt(num / den), rel=1e-9)


def _mixed_indices(per_side=2, limit=200):
    """Indices of the mixed-size batch generator covering every side."""
    got = {}
    for i in range(limit):
        n = inputs.batch_problem(i)["S"].shape[0]
        if len(got.setdefault(n, [])) < per_side:
            got[n].append(i)
    assert len(got) == len(inputs.BATCH_SIDES)
    return got


def test_mixed_sizes_solved_concurrently(torch_cuda):
    """Two problems of every side 64-512 (Helmholtz and diffusion), one
    autotuned batch solver per side, all solved at once: each converged
    field has the oracle's preconditioned residual below 1.5e-6, matches
    the problem solved alone, and (for the sides the oracle solves quickly)
    the oracle's own solve."""
    torch = torch_cuda
    from paper_2207_14222_gb300.solver import BatchSolver, Solver, solve_many
    dev = torch.device("cuda:0")
    groups = _mixed_indices()
    sides = sorted(groups)
    probs = {n: [inputs.batch_problem(i) for i in groups[n]] for n in sides}
    kinds = {p["kind"] for n in sides for p in probs[n]}
    assert kinds == {"helmholtz", "diffusion"}
    data = {}
    for n in sides:
        cfs = [ocanon.canonical(p) for p in probs[n]]
        V = np.stack([cf["V"].astype(np.complex64) for cf in cfs])
        y = np.stack([cf["y"].astype(np.complex64) for cf in cfs])
        data[n] = (cfs, V, y)
    solvers = [_batch(torch, (n, n), data[n][0], data[n][1]) for n in sides]
    try:
        ys = [torch.from_numpy(data[n][2]).to(dev) for n in sides]
        tuned = [sv.autotune(y, iters=2) for sv, y in zip(solvers, ys)]
        assert all(t["chunk"] >= 4 for t in tuned)
        xs, res = solve_many(solvers, ys, tol=1e-6, maxit=20000)
    finally:
        for sv in solvers:
            sv.close()
    for gi, n in enumerate(sides):
        cfs, V, y = data[n]
        xg = xs[gi].cpu().numpy().astype(np.complex128)
        for j, cf in enumerate(cfs):
            r = res[gi][j]
            assert r["status"] == "USP_OK" and r["converged"] == 1, (n, j, r)
            V64, y64 = V[j].astype(np.complex128), y[j].astype(np.complex128)
            Lh = _lh((n, n), cf)
            d = uo.residual_delta(xg[j], y64, V64, Lh)
            assert np.linalg.norm(d) / r["ref_norm"] < 1.5e-6, (n, j)
            with Solver((n, n), cf["a"], cf["b"], torch.from_numpy(V[j]).to(dev)) as s1:
                x1, r1 = s1.solve(torch.from_numpy(y[j]).to(dev), tol=1e-6, maxit=20000)
            assert abs(r1["iterations"] - r["iterations"]) <= 2, (n, j)
            assert _rel(xg[j], x1.cpu().numpy().astype(np.complex128)) <= 2e-6, (n, j)
            if n <= 96:
                xo, _, ok = uo.solve(V64, y64, Lh, r["alpha"], 1e-6, 20000)
                assert ok and _rel(xg[j], xo) <= TOL_X, (n, j)


def test_autotune_choice_is_cached_per_shape(torch_cuda):
    torch = torch_cuda
    shape = (128, 128)
    cfs, V, y = _prep([inputs.random_helmholtz(shape, 90 + j) for j in range(2)])
    yd = torch.from_numpy(y).to("cuda:0")
    with _batch(torch, shape, cfs, V) as s:
        t1 = s.autotune(yd, iters=2)
        x, res = s.solve(yd, tol=1e-6, maxit=5000, allow_failed=False)
    with _batch(torch, shape, cfs, V) as s:
        t2 = s.autotune(yd, iters=2)
    assert t1 == t2
    # square 128^2: the on-chip schedule (several times faster than the passes)
    assert t1["schedule"] == 3 and 4 <= t1["chunk"] <= 64
    for j, cf in enumerate(cfs):
        V64, y64 = V[j].astype(np.complex128), y[j].astype(np.complex128)
        d = uo.residual_delta(x[j].cpu().numpy().astype(np.complex128), y64, V64, _lh(shape, cf))
        assert np.linalg.norm(d) / res[j]["ref_norm"] < 1.5e-6
