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
