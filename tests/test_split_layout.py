"""Host-side model of the split-y schedule's data movement (no GPU): the
factorisation of the 256-point y transform into the rows pass's y1 stage and
the column pass's y2 stage, the scratch layout S[k1][z][y2][kx] that the rows
pass writes, the 4-D tensor-map view the column pass gathers its tiles
through, and the column-major arrangement of a tile in shared memory --
restated from the kernels' index rules and checked for the properties the
kernels rely on:

* the two 16-point stages with the W_256^(y2 k1) factor between them give
  the 256-point DFT (and the inverse stages its inverse);
* the rows pass's store offsets and the tensor map's element offsets name
  the same element, and every element of the scratch is written once and
  gathered once per iteration;
* the column tile's shared-memory positions (as the box arrives: [y2][z][xi])
  and the column-major positions of the z transform are bijections, and the
  y2 stage's stores land where the z transform reads;
* one whole application of (L+I)^-1 through these layouts equals the
  oracle's spectral division.

A change to an index rule that breaks one of these would mix up points of
the field; this catches it on the CPU."""

import numpy as np
import pytest

from oracle import usp_oracle as uo

N = 256          # nx = ny
R1 = R2 = 16     # y = 16 y1 + y2, k = k1 + 16 k2
XB = 2           # kx per column tile


def w(n, e):
    return np.exp(-2j * np.pi * np.asarray(e) / n)


def rows_stage(t):
    """Rows pass on the y axis (axis -2 of length 256): for each residue y2,
    the 16-point DFT over y1, then the factor W_256^(y2 k1).  Returns
    A[..., y2, k1, x]."""
    s = t.reshape(t.shape[:-2] + (R1, R2, t.shape[-1]))           # [.., y1, y2, x]
    a = np.fft.fft(s, axis=-3)                                     # y1 -> k1
    a = np.moveaxis(a, -3, -2)                                     # [.., y2, k1, x]
    y2 = np.arange(R2)[:, None, None]
    k1 = np.arange(R1)[None, :, None]
    return a * w(N, y2 * k1)


def cols_stage(a):
    """Column pass's y2 stage: 16-point DFT over y2 -> k2, giving
    Y[k1 + 16 k2]."""
    b = np.fft.fft(a, axis=-3)                                     # [.., k2, k1, x]
    return b.reshape(a.shape[:-3] + (N, a.shape[-1]))              # k = 16 k2 + k1


def rows_stage_inv(y):
    """Inverse of cols_stage then rows_stage (unnormalised, as the kernels):
    inverse y2 stage, then conj factor and the inverse 16-point DFT over k1."""
    b = y.reshape(y.shape[:-2] + (R2, R1, y.shape[-1]))           # [.., k2, k1, x]
    a = np.fft.ifft(b, axis=-3) * R2                               # k2 -> y2
    y2 = np.arange(R2)[:, None, None]
    k1 = np.arange(R1)[None, :, None]
    a = a * np.conj(w(N, y2 * k1))
    s = np.fft.ifft(a, axis=-2) * R1                               # k1 -> y1: [.., y2, y1, x]
    s = np.moveaxis(s, -2, -3)                                     # [.., y1, y2, x]
    return s.reshape(y.shape)


def test_factorisation_is_the_256_point_dft():
    rng = np.random.default_rng(0)
    t = rng.standard_normal((3, N, 5)) + 1j * rng.standard_normal((3, N, 5))
    y = cols_stage(rows_stage(t))
    assert np.max(np.abs(y - np.fft.fft(t, axis=-2))) < 1e-11 * np.max(np.abs(y))
    back = rows_stage_inv(y)
    assert np.max(np.abs(back - N * t)) < 1e-11 * np.max(np.abs(back))


def rows_store_offset(nz, z, y2, k1, kx):
    """Rows pass: tile u = 16 z + y2 stores element (k1, kx) at
    buf + u * 256 + kx + k1 * (nz * 16) * 256."""
    u = R2 * z + y2
    tiles = nz * R2
    return u * N + kx + k1 * tiles * N


def map_offset(nz, kx, z, y2, k1):
    """The column pass's 4-D view {kx 256, z nz, y2 16, k1 16} with byte
    strides (z, y2, k1) = (16 * 256 * 8, 256 * 8, nz * 16 * 256 * 8), in
    8-byte elements."""
    return kx + z * (R2 * N) + y2 * N + k1 * (nz * R2 * N)


@pytest.mark.parametrize("nz", [32, 64, 128, 256])
def test_rows_stores_and_map_name_the_same_elements(nz):
    z, y2, k1, kx = np.meshgrid(np.arange(nz), np.arange(R2), np.arange(R1), np.arange(N),
                                indexing="ij")
    a = rows_store_offset(nz, z, y2, k1, kx)
    b = map_offset(nz, kx, z, y2, k1)
    assert np.array_equal(a, b)
    # every element of the scratch written once
    assert np.array_equal(np.sort(a.ravel()), np.arange(nz * R2 * R1 * N))


@pytest.mark.parametrize("nz", [32, 64, 128, 256])
def test_column_tiles_gather_each_element_once(nz):
    """Tile t = (k1, xb), t = 128 k1 + xb: the box {2, nz, 16, 1} at
    (2 xb, 0, 0, k1); shared-memory position xi + 2 (z + nz y2)."""
    seen = np.zeros(nz * R2 * R1 * N, np.int32)
    xi, zz, yy = np.meshgrid(np.arange(XB), np.arange(nz), np.arange(R2), indexing="ij")
    smem = (xi + XB * (zz + nz * yy)).ravel()
    assert np.array_equal(np.sort(smem), np.arange(XB * nz * R2))
    for t in range(R1 * (N // XB)):
        k1, xb = divmod(t, N // XB)
        off = map_offset(nz, XB * xb + xi, zz, yy, k1).ravel()
        seen[off] += 1
    assert np.all(seen == 1)


def colpos(nz, c, z):
    return c * nz + (z ^ (8 * (c & 1)))


@pytest.mark.parametrize("nz", [32, 64, 128, 256])
def test_column_major_positions(nz):
    """The y2 stage of pair (z, xi) stores k2 at colpos(xi, z) + 2 nz k2,
    which is column c = 2 k2 + xi at position z (XOR-swizzled); the positions
    are a bijection onto the tile, and for nz = 256 the z transform's thread g
    of column c reads z = g + 16 q at c nz + (g ^ 8 (c & 1)) + 16 q."""
    c_all = np.arange(XB * R2)[:, None]
    z_all = np.arange(nz)[None, :]
    pos = colpos(nz, c_all, z_all)
    assert np.array_equal(np.sort(pos.ravel()), np.arange(XB * R2 * nz))
    for xi in range(XB):
        for k2 in range(R2):
            z = np.arange(nz)
            assert np.array_equal(colpos(nz, xi, z) + 2 * nz * k2, colpos(nz, 2 * k2 + xi, z))
    if nz == 256:
        g = np.arange(16)[:, None]
        q = np.arange(16)[None, :]
        for c in range(XB * R2):
            cbase = c * nz + (g ^ (8 * (c & 1)))
            assert np.array_equal(cbase + 16 * q, colpos(nz, c, g + 16 * q))


def test_two_pass_model_applies_l_plus_i_inverse():
    """One application of (L+I)^-1 through the schedule's steps and layouts
    (nz = 32): rows pass forward (x FFT, y1 stage, stores into S), column
    pass (gather by tiles, y2 stage, z FFT, x 1/(N (Lhat + 1)), inverse,
    scatter), rows pass inverse -- against the oracle's spectral division."""
    nz = 32
    shape = (nz, N, N)
    rng = np.random.default_rng(1)
    t = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    a, b = 0.3j, 0.55 - 1.7j
    Lh = uo.lhat(shape, 1.0, a, b)
    # rows pass: FFT x, then the y1 stage per tile (z, y2); store into S
    tx = np.fft.fft(t, axis=2)
    A = rows_stage(tx)                                  # [z, y2, k1, kx]
    S = np.empty(nz * R2 * R1 * N, complex)
    z, y2, k1, kx = np.meshgrid(np.arange(nz), np.arange(R2), np.arange(R1), np.arange(N),
                                indexing="ij")
    S[rows_store_offset(nz, z, y2, k1, kx)] = A[z, y2, k1, kx]
    # column pass, tile by tile
    xi, zz, yy = np.meshgrid(np.arange(XB), np.arange(nz), np.arange(R2), indexing="ij")
    for tt in range(R1 * (N // XB)):
        k1t, xb = divmod(tt, N // XB)
        off = map_offset(nz, XB * xb + xi, zz, yy, k1t)         # [xi, z, y2]
        tile = S[off]
        spec = np.fft.fft(np.fft.fft(tile, axis=2), axis=1)     # y2 -> k2, z -> kz
        kxx = XB * xb + np.arange(XB)[:, None, None]
        ky = k1t + R1 * np.arange(R2)[None, None, :]
        kz = np.arange(nz)[None, :, None]
        spec = spec / (nz * N * N * (Lh[kz, ky, kxx] + 1))
        back = np.fft.ifft(np.fft.ifft(spec, axis=1), axis=2) * (nz * R2)
        S[off] = back
    # rows pass inverse: gather rows, inverse y1 stage, inverse FFT x
    Ai = S[rows_store_offset(nz, z, y2, k1, kx)]                 # [z, y2, k1, kx]
    Ai = Ai * np.conj(w(N, y2 * k1))
    s = np.fft.ifft(Ai, axis=2) * R1                             # k1 -> y1: [z, y2, y1, kx]
    s = np.moveaxis(s, 2, 1).reshape(nz, N, N)                   # y = 16 y1 + y2
    u = np.fft.ifft(s, axis=2) * N
    ref = uo.apply_L_plus_I_inverse(t, Lh)
    assert np.max(np.abs(u - ref)) < 1e-12 * np.max(np.abs(ref))
