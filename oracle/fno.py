"""Oracle: the Fourier neural operator that proposes a warm start x0.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import anything under ``oracle/``.  Plain
NumPy in FP64, sharing no code with the CUDA path.

The paper has no counterpart: Algorithm 1 accepts any initial estimate x0
(Sec. 2.1 starts from x0 = 0 as one choice), and this network supplies one.
The iteration's stopping test keeps the alpha-free denominator ||B (L+I)^-1 y||
whatever x0 is, so a warm start changes where the iteration starts, never what
it converges to.

The network (a Fourier neural operator, Li et al. 2020, restated here):
  input  a   : (batch, c_in, H, W) real channels
  lift       : v0 = P a + p                      (per pixel, P: width x c_in)
  layer l    : z_l = W_l v_l + b_l + K_l v_l;    v_{l+1} = gelu(z_l) for
               l < layers - 1, v_layers = z_{layers-1}
  spectral   : K_l v = Re( F^-1 [ S^T R_l S F v ] ), F the unnormalised 2-D
               DFT (exponent -i), F^-1 its inverse (factor 1/(H W)), S the
               selection of the modes x modes lowest frequencies (index k of
               each axis in [0, modes/2) or [n - modes/2, n)), and R_l one
               complex width x width matrix per retained mode
  project    : u = Q v_layers + q                (Q: 2 x width); the field
               estimate is u[0] + i u[1]
  gelu(x) = x Phi(x) = x (1 + erf(x / sqrt 2)) / 2
  loss       : mean over the batch of ||u0 + i u1 - x||^2 / ||x||^2

The backward pass is derived by hand (adjoints of each linear map): for the
spectral map, d v = Re(F^-1 S^T R^H S F g) and dR[o, c, m] =
sum_batch (F g_o)(m) conj((F v_c)(m)) / (H W).

Flat parameter layout (the order of ``pack``/``unpack``): P [width][c_in],
p [width]; per layer W [width][width] (out, in), b [width], R
[width(out)][width(in)][modes(axis H)][modes(axis W)][re, im]; Q [2][width],
q [2].
"""

import math

import numpy as np


def mode_index(n, modes):
    """FFT index of mode slot s in [0, modes): s for the first half, then the
    highest indices n - modes + s (the negative frequencies)."""
    h = modes // 2
    return np.array([s if s < h else n - modes + s for s in range(modes)])


def shapes(c_in, width, layers, modes):
    out = [("P", (width, c_in)), ("p", (width,))]
    for l in range(layers):
        out += [("W%d" % l, (width, width)), ("b%d" % l, (width,)),
                ("R%d" % l, (width, width, modes, modes, 2))]
    out += [("Q", (2, width)), ("q", (2,))]
    return out


def unpack(flat, c_in, width, layers, modes):
    prm, k = {}, 0
    for name, sh in shapes(c_in, width, layers, modes):
        n = int(np.prod(sh))
        prm[name] = np.asarray(flat[k:k + n], dtype=np.float64).reshape(sh)
        k += n
    assert k == len(flat)
    return prm


def pack(prm, c_in, width, layers, modes):
    return np.concatenate([np.asarray(prm[name], np.float64).ravel()
                           for name, _ in shapes(c_in, width, layers, modes)])


def gelu(x):
    erf = np.vectorize(math.erf)
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    erf = np.vectorize(math.erf)
    cdf = 0.5 * (1.0 + erf(x / math.sqrt(2.0)))
    pdf = np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)
    return cdf + x * pdf


def _complex_R(R):
    return R[..., 0] + 1j * R[..., 1]


def spectral(v, R, modes, adjoint=False):
    """K v (or K^T v with adjoint): v (batch, c, H, W) real; R (o, c, modes,
    modes, 2).  Returns (result, the retained modes of F v)."""
    _, _, H, W = v.shape
    ih, iw = mode_index(H, modes), mode_index(W, modes)
    Fv = np.fft.fft2(v)[:, :, ih][:, :, :, iw]          # (batch, c, m1, m2)
    Rc = _complex_R(R)                                  # (o, c, m1, m2)
    if adjoint:
        Z = np.einsum("ocmn,bomn->bcmn", np.conj(Rc), Fv)
    else:
        Z = np.einsum("ocmn,bcmn->bomn", Rc, Fv)
    full = np.zeros(Z.shape[:2] + (H, W), complex)
    full[:, :, ih[:, None], iw[None, :]] = Z
    return np.real(np.fft.ifft2(full)), Fv


def conv1x1(v, Wm, b=None):
    out = np.einsum("oc,bchw->bohw", Wm, v)
    if b is not None:
        out = out + b[None, :, None, None]
    return out


def forward(prm, a, layers, modes):
    """Returns (u, cache); u (batch, 2, H, W)."""
    v = conv1x1(a, prm["P"], prm["p"])
    cache = {"a": a, "v": [], "z": [], "Fv": []}
    for l in range(layers):
        ks, Fv = spectral(v, prm["R%d" % l], modes)
        z = conv1x1(v, prm["W%d" % l], prm["b%d" % l]) + ks
        cache["v"].append(v)
        cache["z"].append(z)
        cache["Fv"].append(Fv)
        v = gelu(z) if l < layers - 1 else z
    cache["vL"] = v
    u = conv1x1(v, prm["Q"], prm["q"])
    return u, cache


def field(u):
    return u[:, 0] + 1j * u[:, 1]


def loss(u, x):
    """Mean relative squared error of the field estimate against x
    (batch, H, W) complex."""
    d = field(u) - x
    num = np.sum(np.abs(d) ** 2, axis=(1, 2))
    den = np.sum(np.abs(x) ** 2, axis=(1, 2))
    return float(np.mean(num / den))


def backward(prm, cache, u, x, layers, modes):
    """Gradients of ``loss`` with respect to every parameter (dict of the
    same shapes)."""
    B, _, H, W = u.shape
    d = field(u) - x
    den = np.sum(np.abs(x) ** 2, axis=(1, 2))
    gu = np.stack([np.real(d), np.imag(d)], axis=1) * (2.0 / (B * den))[:, None, None, None]
    g = {}
    vL = cache["vL"]
    g["Q"] = np.einsum("bkhw,bchw->kc", gu, vL)
    g["q"] = np.sum(gu, axis=(0, 2, 3))
    gv = conv1x1(gu, prm["Q"].T)
    ih, iw = mode_index(H, modes), mode_index(W, modes)
    for l in reversed(range(layers)):
        z, v, Fv = cache["z"][l], cache["v"][l], cache["Fv"][l]
        gz = gv * gelu_grad(z) if l < layers - 1 else gv
        g["W%d" % l] = np.einsum("bohw,bchw->oc", gz, v)
        g["b%d" % l] = np.sum(gz, axis=(0, 2, 3))
        Fg = np.fft.fft2(gz)[:, :, ih][:, :, :, iw]      # (batch, o, m1, m2)
        dR = np.einsum("bomn,bcmn->ocmn", Fg, np.conj(Fv)) / (H * W)
        g["R%d" % l] = np.stack([np.real(dR), np.imag(dR)], axis=-1)
        ks_adj, _ = spectral(gz, prm["R%d" % l], modes, adjoint=True)
        gv = conv1x1(gz, prm["W%d" % l].T) + ks_adj
    g["P"] = np.einsum("bkhw,bchw->kc", gv, cache["a"])
    g["p"] = np.sum(gv, axis=(0, 2, 3))
    return g


def adam(params, grads, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma and Ba 2015) on flat vectors; t counts steps
    from 1.  Returns the new (params, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grads
    v = beta2 * v + (1.0 - beta2) * grads * grads
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v
