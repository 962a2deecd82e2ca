"""Canonical form of physical problems, computed by the library on the host
in FP64 (usp_canon_helmholtz / usp_canon_diffusion; paper Sec. 2.2, 3.1, 3.2).

Input: a problem dict from ``inputs`` (physical fields).  Output: complex64
V and y ready for the GPU plus the symbol coefficients a, b.
"""

import ctypes

import numpy as np

from . import _lib


def canonical(problem, norm_v=0.95):
    L = _lib.lib()
    shape = np.shape(problem["S"])
    n = int(np.prod(shape))
    S = np.ascontiguousarray(problem["S"], dtype=np.complex128)
    y = np.empty(shape, np.complex64)
    sym = _lib.LSymbol()
    c = np.zeros(2)
    bias = np.zeros(2)
    if problem["kind"] == "helmholtz":
        k2 = np.ascontiguousarray(problem["k2"], dtype=np.complex128)
        V = np.empty(shape, np.complex64)
        st = L.usp_canon_helmholtz(k2.ctypes.data, S.ctypes.data, n, float(norm_v),
                                   V.ctypes.data, y.ctypes.data, ctypes.byref(sym),
                                   c.ctypes.data, bias.ctypes.data)
    else:
        eta = np.ascontiguousarray(problem["eta"], dtype=np.float64)
        V = np.empty(shape, np.float32)
        st = L.usp_canon_diffusion(eta.ctypes.data, float(problem["D"]), S.ctypes.data, n,
                                   float(norm_v), V.ctypes.data, y.ctypes.data,
                                   ctypes.byref(sym), c.ctypes.data, bias.ctypes.data)
    if st != _lib.OK:
        raise _lib.UspError(st, "canonical form failed")
    return dict(V=V, y=y, a=complex(sym.a_re, sym.a_im), b=complex(sym.b_re, sym.b_im),
                c=complex(c[0], c[1]), bias=complex(bias[0], bias[1]), dx=problem["dx"],
                kind=problem["kind"])


def antisymmetric(k2, S, dx=1.0, S_adj=None, norm_v=0.95):
    """Antisymmetrised canonical form of laplacian psi + k^2 psi = -S (and of
    the adjoint problem with source -S_adj): v (complex64 grid), y (complex64,
    2 planes), params (a_re, a_im, b_re, b_im of l = a|p|^2 + b), c."""
    L = _lib.lib()
    k2 = np.ascontiguousarray(k2, dtype=np.complex128)
    shape = k2.shape
    n = int(np.prod(shape))
    S = np.ascontiguousarray(S, dtype=np.complex128)
    Sa = None if S_adj is None else np.ascontiguousarray(S_adj, dtype=np.complex128)
    v = np.empty(shape, np.complex64)
    y = np.empty((2,) + shape, np.complex64)
    params = np.zeros(4)
    c = np.zeros(1)
    st = L.usp_canon_antisymmetric(k2.ctypes.data, S.ctypes.data,
                                   None if Sa is None else Sa.ctypes.data, n, float(norm_v),
                                   v.ctypes.data, y.ctypes.data,
                                   params.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                   c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if st != _lib.OK:
        raise _lib.UspError(st, "antisymmetrised canonical form failed")
    return dict(kind="antisymmetric", V=v, y=y, params=params, c=float(c[0]), dx=dx)


def flux_diffusion(eta, D, S, dx=1.0, norm_v=0.95):
    """Flux canonical form of -div(D grad u) + eta u = S: V (float32, 2
    planes Vu, VJ), y (complex64, 1 + ndim planes), params (alpha, beta, s),
    scales (c_u, c_J); u = x[0] / sqrt(c_u)."""
    L = _lib.lib()
    eta = np.ascontiguousarray(eta, dtype=np.float64)
    shape = eta.shape
    n = int(np.prod(shape))
    D = np.ascontiguousarray(np.broadcast_to(np.asarray(D, np.float64), shape))
    S = np.ascontiguousarray(np.real(S), dtype=np.float64)
    V = np.empty((2,) + shape, np.float32)
    y = np.empty((1 + len(shape),) + shape, np.complex64)
    params = np.zeros(3)
    scales = np.zeros(2)
    st = L.usp_canon_flux_diffusion(eta.ctypes.data, D.ctypes.data, S.ctypes.data, n,
                                    len(shape), float(norm_v), V.ctypes.data, y.ctypes.data,
                                    params.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                    scales.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if st != _lib.OK:
        raise _lib.UspError(st, "flux canonical form failed")
    return dict(kind="flux", V=V, y=y, params=params, scales=scales, dx=dx)
