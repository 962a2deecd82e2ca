"""Pins of the FP64 Fourier-neural-operator oracle (oracle/fno.py) against
definitions, closed forms and identities that do not come from the oracle's
own backward pass: the Gaussian error function, band-limited signals, the
adjoint identity of the spectral map, central finite differences of the
loss, and Adam's closed-form first step."""

import numpy as np
import pytest

from oracle import fno

C_IN, WIDTH, LAYERS, MODES, H, W = 3, 4, 2, 4, 8, 16


def _params(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    n = sum(int(np.prod(sh)) for _, sh in fno.shapes(C_IN, WIDTH, LAYERS, MODES))
    return rng.standard_normal(n) * scale


def test_gelu_values_and_derivative():
    assert fno.gelu(np.array([0.0]))[0] == 0.0
    # x Phi(x) with Phi the standard normal CDF
    assert fno.gelu(np.array([1.0]))[0] == pytest.approx(0.8413447460685429, abs=1e-15)
    assert fno.gelu(np.array([-1.0]))[0] == pytest.approx(-0.15865525393145707, abs=1e-15)
    assert fno.gelu(np.array([10.0]))[0] == pytest.approx(10.0, abs=1e-12)
    x = np.linspace(-4, 4, 17)
    h = 1e-6
    fd = (fno.gelu(x + h) - fno.gelu(x - h)) / (2 * h)
    assert np.max(np.abs(fno.gelu_grad(x) - fd)) < 1e-8


def test_mode_index():
    assert list(fno.mode_index(16, 4)) == [0, 1, 14, 15]
    assert list(fno.mode_index(128, 16)) == list(range(8)) + list(range(120, 128))


def _identity_R(c):
    R = np.zeros((c, c, MODES, MODES, 2))
    for k in range(c):
        R[k, k, :, :, 0] = 1.0
    return R


def test_spectral_identity_keeps_retained_band_only():
    i = np.arange(H)[:, None]
    j = np.arange(W)[None, :]
    # frequencies +-1 on both axes: retained in both signs (the band is
    # [-modes/2, modes/2), so +-2 would lose its positive half)
    low = np.cos(2 * np.pi * (i / H + j / W)) + 0.5 * np.sin(2 * np.pi * (-i / H + j / W))
    high = np.cos(2 * np.pi * 3 * j / W)        # |k| = 3 > modes / 2
    v = np.stack([low + high, 2 * low])[None]
    out, _ = fno.spectral(v, _identity_R(2), MODES)
    assert np.allclose(out[0, 0], low, atol=1e-12)
    assert np.allclose(out[0, 1], 2 * low, atol=1e-12)


def test_spectral_single_mode_closed_form():
    """One complex weight r on mode (0, 1) maps cos(2 pi j / W) to
    Re(r e^{2 pi i j/W}) / 2 (the mode (0, -1) carries the other half, with
    weight zero)."""
    r = 0.7 - 0.4j
    R = np.zeros((1, 1, MODES, MODES, 2))
    R[0, 0, 0, 1] = [r.real, r.imag]
    j = np.arange(W)[None, :] + np.zeros((H, 1))
    v = np.cos(2 * np.pi * j / W)[None, None]
    out, _ = fno.spectral(v, R, MODES)
    assert np.allclose(out[0, 0], np.real(r * np.exp(2j * np.pi * j / W)) / 2, atol=1e-12)


def test_spectral_adjoint_identity():
    rng = np.random.default_rng(3)
    R = rng.standard_normal((WIDTH, 3, MODES, MODES, 2))
    v = rng.standard_normal((2, 3, H, W))
    g = rng.standard_normal((2, WIDTH, H, W))
    Kv, _ = fno.spectral(v, R, MODES)
    # the adjoint maps the output space (WIDTH channels) back to 3 channels
    KTg, _ = fno.spectral(g, R, MODES, adjoint=True)
    assert KTg.shape == v.shape
    assert np.sum(Kv * g) == pytest.approx(np.sum(v * KTg), rel=1e-12)


def test_gradients_match_central_differences():
    rng = np.random.default_rng(5)
    flat = _params(1)
    a = rng.standard_normal((2, C_IN, H, W))
    x = rng.standard_normal((2, H, W)) + 1j * rng.standard_normal((2, H, W))

    def L(f):
        prm = fno.unpack(f, C_IN, WIDTH, LAYERS, MODES)
        u, _ = fno.forward(prm, a, LAYERS, MODES)
        return fno.loss(u, x)

    prm = fno.unpack(flat, C_IN, WIDTH, LAYERS, MODES)
    u, cache = fno.forward(prm, a, LAYERS, MODES)
    g = fno.pack(fno.backward(prm, cache, u, x, LAYERS, MODES), C_IN, WIDTH, LAYERS, MODES)
    # every tensor gets probed
    offs, k = [], 0
    for _, sh in fno.shapes(C_IN, WIDTH, LAYERS, MODES):
        n = int(np.prod(sh))
        offs += list(k + rng.choice(n, size=min(n, 6), replace=False))
        k += n
    h = 1e-6
    for i in offs:
        e = np.zeros_like(flat)
        e[i] = h
        fd = (L(flat + e) - L(flat - e)) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-9), i


def test_loss_zero_at_truth_and_scale_free():
    rng = np.random.default_rng(6)
    x = rng.standard_normal((2, H, W)) + 1j * rng.standard_normal((2, H, W))
    u = np.stack([x.real, x.imag], axis=1)
    assert fno.loss(u, x) == 0.0
    assert fno.loss(3 * u, 3 * x) == 0.0
    assert fno.loss(np.zeros_like(u), x) == pytest.approx(1.0)


def test_adam_first_step_closed_form():
    g = np.array([0.5, -2.0, 1e-3])
    p, m, v = fno.adam(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    # bias-corrected moments are g and g^2 after one step
    assert np.allclose(p, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_pack_unpack_round_trip():
    flat = _params(2)
    prm = fno.unpack(flat, C_IN, WIDTH, LAYERS, MODES)
    assert prm["R1"].shape == (WIDTH, WIDTH, MODES, MODES, 2)
    assert np.array_equal(fno.pack(prm, C_IN, WIDTH, LAYERS, MODES), flat)
