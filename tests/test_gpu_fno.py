"""The warm-start network's CUDA kernels against the FP64 oracle
(oracle/fno.py) through the C ABI: forward pass, every parameter gradient,
the Adam step; then its purpose: trained on solver output, its estimate as
x0 shortens the solve, and the solve still returns the iteration's own
answer.

Tolerances: forward relative L2 <= 1e-5 (FP32 arithmetic over sums of a few
thousand terms); gradients per tensor relative L2 <= 1e-4.
"""

import numpy as np
import pytest

from oracle import fno as ofno
from oracle import usp_oracle as uo
from paper_2207_14222_gb300 import _lib, inputs

pytestmark = pytest.mark.gpu


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


def _setup(torch, h, w, c_in, width, layers, modes, batch, seed):
    from paper_2207_14222_gb300.fno import FNO
    net = FNO(h, w, c_in, width, layers, modes, max_batch=batch, seed=seed)
    rng = np.random.default_rng(seed)
    flat = net.params.astype(np.float64)
    # larger spectral weights than the initialiser's, so every path matters
    prm = ofno.unpack(flat, c_in, width, layers, modes)
    for l in range(layers):
        prm["R%d" % l] = rng.standard_normal(prm["R%d" % l].shape) * (0.5 / width)
        prm["b%d" % l] = rng.standard_normal(width) * 0.1
    prm["q"] = rng.standard_normal(2) * 0.1
    flat = ofno.pack(prm, c_in, width, layers, modes).astype(np.float32)
    net.params = flat
    a = rng.standard_normal((batch, c_in, h, w)).astype(np.float32)
    x = (rng.standard_normal((batch, h, w)) + 1j * rng.standard_normal((batch, h, w))).astype(np.complex64)
    return net, flat.astype(np.float64), a, x


@pytest.mark.parametrize("cfg", [
    (32, 32, 3, 8, 3, 8, 3),
    (16, 64, 2, 5, 2, 4, 2),       # non-square, odd width
    (128, 128, 3, 32, 4, 16, 2),   # the warm-start configuration
])
def test_forward_and_gradients_match_oracle(torch_cuda, cfg):
    torch = torch_cuda
    h, w, c_in, width, layers, modes, batch = cfg
    net, flat, a, x = _setup(torch, h, w, c_in, width, layers, modes, batch, seed=7)
    with net:
        ad = torch.from_numpy(a).cuda()
        xd = torch.from_numpy(x).cuda()
        xh = net.predict(ad).cpu().numpy()
        loss, g = net.gradients(ad, xd)
        loss2, g2 = net.gradients(ad, xd)
    prm = ofno.unpack(flat, c_in, width, layers, modes)
    u, cache = ofno.forward(prm, a.astype(np.float64), layers, modes)
    assert _rel(xh, ofno.field(u)) <= 1e-5
    xo = x.astype(np.complex128)
    lo = ofno.loss(u, xo)
    assert loss == pytest.approx(lo, rel=1e-5)
    go = ofno.backward(prm, cache, u, xo, layers, modes)
    gg = ofno.unpack(g.astype(np.float64), c_in, width, layers, modes)
    for name, _ in ofno.shapes(c_in, width, layers, modes):
        assert _rel(gg[name], go[name]) <= 1e-4, name
    # deterministic reductions: bit-identical on a second call
    assert loss2 == loss and np.array_equal(g, g2)


def test_adam_step_matches_oracle(torch_cuda):
    torch = torch_cuda
    cfg = (32, 32, 3, 8, 2, 8, 2)
    h, w, c_in, width, layers, modes, batch = cfg
    net, flat, a, x = _setup(torch, h, w, c_in, width, layers, modes, batch, seed=8)
    lr = 1e-3
    with net:
        ad, xd = torch.from_numpy(a).cuda(), torch.from_numpy(x).cuda()
        _, g = net.gradients(ad, xd)
        l1 = net.train_step(ad, xd, lr)
        l2 = net.train_step(ad, xd, lr)
        p2 = net.params.astype(np.float64)
    m = np.zeros_like(flat)
    v = np.zeros_like(flat)
    p = flat
    prm = ofno.unpack(p, c_in, width, layers, modes)
    for t in (1, 2):
        prm = ofno.unpack(p, c_in, width, layers, modes)
        u, cache = ofno.forward(prm, a.astype(np.float64), layers, modes)
        go = ofno.pack(ofno.backward(prm, cache, u, x.astype(np.complex128), layers, modes),
                       c_in, width, layers, modes)
        p, m, v = ofno.adam(p, go, m, v, t, lr)
    # Adam's early steps are about lr * sign(g): compare where the gradient
    # is well above the FP32 noise of its computation
    big = np.abs(go) > 1e-3 * np.sqrt(np.mean(go ** 2))
    assert np.max(np.abs(p2 - p)[big]) <= 1e-2 * lr
    assert l2 < l1


def _helmholtz_dataset(torch, n, seeds, abl=8):
    """Media of the 2-D workload's distribution at n x n, their features and
    their solutions from the batch solver (tol 1e-6)."""
    from paper_2207_14222_gb300 import canon
    from paper_2207_14222_gb300.fno import features
    from paper_2207_14222_gb300.solver import BatchSolver
    probs = [inputs.helmholtz_2d(n, seed=s, abl_width=abl) for s in seeds]
    cfs = [canon.canonical(p) for p in probs]
    V = torch.from_numpy(np.stack([cf["V"] for cf in cfs])).cuda()
    y = torch.from_numpy(np.stack([cf["y"] for cf in cfs])).cuda()
    with BatchSolver((n, n), [cf["a"] for cf in cfs], [cf["b"] for cf in cfs], V) as s:
        x, res = s.solve(y, tol=1e-6, maxit=20000, allow_failed=False)
    a = torch.from_numpy(np.stack([features(p) for p in probs])).cuda()
    return probs, cfs, a, x, res


def test_trained_network_shortens_the_solve(torch_cuda):
    """Train on 1024 solved 64 x 64 media (40 epochs), then solve 8 held-out
    media from the network's estimate and from zero: the loss falls tenfold,
    the estimates are within 50% (median relative L2), the warm starts need
    fewer iterations, and each converges to the iteration's own answer with
    the same reference norm."""
    torch = torch_cuda
    from paper_2207_14222_gb300.fno import FNO
    from paper_2207_14222_gb300.solver import Solver
    n = 64
    _, _, a, x, _ = _helmholtz_dataset(torch, n, range(10000, 11024))
    probs_t, cfs_t, at, xt, res_t = _helmholtz_dataset(torch, n, range(90000, 90008))
    losses = []
    with FNO(n, n, width=32, layers=4, modes=16, max_batch=32, seed=3) as net:
        for epoch in range(40):
            perm = torch.randperm(a.shape[0], generator=torch.Generator().manual_seed(epoch))
            ep = []
            for k in range(0, a.shape[0], 32):
                idx = perm[k:k + 32].cuda()
                ep.append(net.train_step(a[idx], x[idx], lr=2e-3 * 0.5 ** (epoch // 15)))
            losses.append(np.mean(ep))
        x0 = net.predict(at)
    err = [_rel(x0[j].cpu().numpy(), xt[j].cpu().numpy()) for j in range(8)]
    assert losses[-1] < 0.2 * losses[0] and np.median(err) < 0.5, (losses, err)
    gain = []
    for j, cf in enumerate(cfs_t):
        V = torch.from_numpy(cf["V"]).cuda()
        y = torch.from_numpy(cf["y"]).cuda()
        with Solver((n, n), cf["a"], cf["b"], V) as s:
            xw, rw = s.solve(y, x=x0[j].clone(), use_x0=True, tol=1e-6, maxit=20000)
            _, rz = s.solve(y, tol=1e-6, maxit=20000)
        assert rw["converged"] == 1
        # the stopping test keeps Algorithm 1's denominator: same ref norm
        assert rw["ref_norm"] == pytest.approx(rz["ref_norm"], rel=1e-5)
        Lh = uo.lhat((n, n), cf["dx"], cf["a"], cf["b"])
        d = uo.residual_delta(xw.cpu().numpy().astype(np.complex128),
                              cf["y"].astype(np.complex128), cf["V"].astype(np.complex128), Lh)
        assert np.linalg.norm(d) / rw["ref_norm"] < 1.5e-6
        gain.append(rz["iterations"] - rw["iterations"])
    assert np.median(gain) > 0, gain
