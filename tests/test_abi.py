"""The C ABI without a GPU: the library loads, exports every function that
include/usp.h declares, rejects bad arguments before touching the device,
and its host-side canonical form agrees with the oracle's."""

import ctypes

import numpy as np
import pytest

from oracle import canon as ocanon
from paper_2207_14222_gb300 import _lib, inputs
from paper_2207_14222_gb300 import build as pkg_build
from paper_2207_14222_gb300 import canon as pcanon


@pytest.fixture(scope="module")
def L():
    pkg_build.build()
    return _lib.lib()


def test_exports_every_declared_function(L):
    names = _lib.header_functions()
    assert len(names) >= 14
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    # the binding declares a signature for every one of them
    assert set(names) == set(_lib._SIGNATURES), set(names) ^ set(_lib._SIGNATURES)


def test_status_strings(L):
    for code, name in _lib.STATUS.items():
        assert L.usp_status_string(code).decode() == name
    assert L.usp_version() >= 100


def _grid(shape, dx=1.0):
    g = _lib.Grid()
    g.ndim = len(shape)
    for i, n in enumerate(shape[:3]):
        g.n[i] = n
    g.dx = dx
    return g


def _create(L, shape, sym=(0.0, 0.3, 0.2, -0.5), V=1, alpha=0.0, dx=1.0):
    g = _grid(shape, dx)
    s = _lib.LSymbol(*sym)
    h = ctypes.c_void_p()
    st = L.usp_solver_create(ctypes.byref(g), ctypes.byref(s), ctypes.c_void_p(V), 0,
                             alpha, None, ctypes.byref(h))
    return st


@pytest.mark.parametrize("shape, expect", [
    ((), _lib.ERR_INVALID_ARG),                 # ndim 0
    ((4, 4, 4, 4), _lib.ERR_INVALID_ARG),       # ndim 4
    ((0, 8), _lib.ERR_INVALID_ARG),             # empty axis
    ((100,), _lib.ERR_UNSUPPORTED_SIZE),        # not a power of two
    ((1024, 2), _lib.ERR_UNSUPPORTED_SIZE),     # above 512
    ((48, 8), _lib.ERR_UNSUPPORTED_SIZE),       # 3 * 16: radix-3 lengths start at 96
    ((768,), _lib.ERR_UNSUPPORTED_SIZE),        # 3 * 256
    ((1, 8), _lib.ERR_UNSUPPORTED_SIZE),        # length-1 axis
])
def test_create_rejects_bad_grids(L, shape, expect):
    assert _create(L, shape) == expect


def test_create_rejects_bad_arguments(L):
    assert _create(L, (8, 8), V=0) == _lib.ERR_INVALID_ARG                 # NULL V
    assert _create(L, (8, 8), dx=0.0) == _lib.ERR_INVALID_ARG
    assert _create(L, (8, 8), dx=float("nan")) == _lib.ERR_INVALID_ARG
    # Re(Lhat + 1) <= 0 somewhere on the grid (Corollary needs Re[L+I] > 0)
    assert _create(L, (8, 8), sym=(0.0, 1.0, -1.5, 0.0)) == _lib.ERR_NOT_ACCRETIVE
    assert _create(L, (8, 8), sym=(-1.0, 0.0, 0.0, 0.0)) == _lib.ERR_NOT_ACCRETIVE
    assert _create(L, (8, 8), sym=(float("inf"), 0, 0, 0)) == _lib.ERR_INVALID_ARG
    assert _create(L, (8, 8), alpha=2.5) == _lib.ERR_ALPHA_RANGE
    assert _create(L, (8, 8), alpha=float("nan")) == _lib.ERR_ALPHA_RANGE
    assert "alpha" in _lib.last_error()


def test_null_handles_are_rejected(L):
    """Entry points that take a solver handle refuse NULL without touching the
    device (no GPU here)."""
    o = _lib.Options()
    assert L.usp_solver_set_options(None, ctypes.byref(o)) == _lib.ERR_INVALID_ARG
    assert L.usp_variant_set_schedule(None, 0) == _lib.ERR_INVALID_ARG
    a = ctypes.c_double()
    assert L.usp_solver_alpha(None, ctypes.byref(a)) == _lib.ERR_INVALID_ARG
    n = ctypes.c_int32()
    assert L.usp_residual_history(None, None, 0, ctypes.byref(n)) == _lib.ERR_INVALID_ARG


def test_table_symbol_rejections(L):
    """A tabulated symbol needs a table, one problem, and a known kind; the
    allocation-free entry point takes the quadratic symbol only."""
    g = _grid((8, 8))
    h = ctypes.c_void_p()
    s = _lib.LSymbol(0.0, 0.0, 0.0, 0.0, 1, None)          # kind TABLE, NULL table
    assert L.usp_solver_create(ctypes.byref(g), ctypes.byref(s), ctypes.c_void_p(1), 0, 0.0,
                               None, ctypes.byref(h)) == _lib.ERR_INVALID_ARG
    assert "table" in _lib.last_error()
    s = _lib.LSymbol(0.0, 0.3, 0.2, -0.5, 7, None)         # unknown kind
    assert L.usp_solver_create(ctypes.byref(g), ctypes.byref(s), ctypes.c_void_p(1), 0, 0.0,
                               None, ctypes.byref(h)) == _lib.ERR_INVALID_ARG
    g = _grid((64, 64))
    arr = (_lib.LSymbol * 2)(_lib.LSymbol(0.0, 0.3, 0.2, -0.5, 1, 16),
                             _lib.LSymbol(0.0, 0.3, 0.2, -0.5))
    al = (ctypes.c_double * 2)(0.0, 0.0)
    assert L.usp_batch_create(ctypes.byref(g), 2, arr, ctypes.c_void_p(1), 0, al, None,
                              ctypes.byref(h)) == _lib.ERR_INVALID_ARG
    assert "single-problem" in _lib.last_error()
    s = _lib.LSymbol(0.0, 0.3, 0.2, -0.5, 1, 16)
    r = _lib.Result()
    assert L.usp_solve_noalloc(ctypes.byref(g), ctypes.byref(s), ctypes.c_void_p(1), 0, 0.0,
                               ctypes.c_void_p(1), ctypes.c_void_p(1), 1e-5, 10, None,
                               ctypes.byref(r)) == _lib.ERR_INVALID_ARG


def _batch_create(L, shape, syms, alphas=None, V=1):
    g = _grid(shape)
    count = len(syms)
    arr = (_lib.LSymbol * max(1, count))(*[_lib.LSymbol(*sy) for sy in syms])
    al = (ctypes.c_double * max(1, count))(*(alphas or [0.0] * count))
    h = ctypes.c_void_p()
    return L.usp_batch_create(ctypes.byref(g), count, arr, ctypes.c_void_p(V), 0, al, None,
                              ctypes.byref(h))


def test_batch_create_rejects_bad_arguments(L):
    good = (0.0, 0.3, 0.2, -0.5)
    assert _batch_create(L, (64, 64), []) == _lib.ERR_INVALID_ARG           # count 0
    assert _batch_create(L, (64, 64), [good, good], V=0) == _lib.ERR_INVALID_ARG
    # every problem's symbol is validated (Corollary: Re[L+I] > 0)
    bad = (0.0, 1.0, -1.5, 0.0)
    assert _batch_create(L, (64, 64), [good, good, bad]) == _lib.ERR_NOT_ACCRETIVE
    assert "problem 2" in _lib.last_error()
    assert _batch_create(L, (64, 64), [good, good], alphas=[0.5, 3.0]) == _lib.ERR_ALPHA_RANGE
    # a batch needs whole blocks of lines per problem: 1-D and thin grids are refused
    assert _batch_create(L, (256,), [good, good]) == _lib.ERR_UNSUPPORTED_SIZE
    assert _batch_create(L, (8, 256), [good, good]) == _lib.ERR_UNSUPPORTED_SIZE
    assert _batch_create(L, (4, 4), [good, good]) == _lib.ERR_UNSUPPORTED_SIZE


def test_canonical_variants_match_oracle(L):
    from oracle import variants as ov
    prob = inputs.gain_helmholtz((8, 12), 3)
    Sa = inputs.random_field((8, 12), 4)
    cp = pcanon.antisymmetric(prob["k2"], prob["S"], S_adj=Sa)
    co = ov.antisymmetric_helmholtz(prob["k2"], prob["S"], 1.0, S_adj=Sa)
    assert np.allclose(cp["V"], co["v"], rtol=1e-6, atol=1e-6)
    assert np.allclose(cp["y"], co["y"], rtol=1e-6, atol=1e-6 * np.abs(co["y"]).max())
    assert np.allclose(cp["params"], [np.real(co["a"]), np.imag(co["a"]),
                                      np.real(co["b"]), np.imag(co["b"])], rtol=1e-12)
    assert cp["c"] == pytest.approx(co["c"], rel=1e-12)
    d = inputs.variable_diffusion((6, 10), 5)
    S = np.real(d["S"])
    fp = pcanon.flux_diffusion(d["eta"], d["D"], S)
    fo = ov.flux_diffusion(d["eta"], d["D"], S, 1.0)
    assert np.allclose(fp["V"][0], fo["Vu"], atol=1e-6) and np.allclose(fp["V"][1], fo["VJ"], atol=1e-6)
    assert np.allclose(fp["params"], [fo["alpha"], fo["beta"], fo["s"]], rtol=1e-12)
    assert np.allclose(fp["scales"], [fo["c_u"], fo["c_J"]], rtol=1e-12)
    assert np.allclose(fp["y"], fo["y"], rtol=1e-6, atol=1e-7)


def test_fno_config_validation(L):
    def count(*cfg):
        return L.usp_fno_param_count(ctypes.byref(_lib.FnoConfig(*cfg)))
    # P, p; per layer W, b, R (complex per mode); Q, q
    assert count(128, 128, 3, 32, 4, 16, 8) == 32 * 3 + 32 + 4 * (32 * 32 + 32 + 32 * 32 * 256 * 2) + 64 + 2
    assert count(128, 128, 3, 32, 4, 12, 8) == -1      # modes not a power of two
    assert count(128, 128, 3, 65, 4, 16, 8) == -1      # width above 64
    assert count(4, 128, 3, 8, 1, 2, 1) == -1          # image below 8
    assert count(128, 128, 9, 8, 1, 16, 1) == -1       # too many input channels
    h = ctypes.c_void_p()
    assert L.usp_fno_create(ctypes.byref(_lib.FnoConfig(128, 128, 3, 8, 0, 16, 1)), 0, None,
                            ctypes.byref(h)) == _lib.ERR_INVALID_ARG
    L.usp_fno_destroy(None)


def test_null_handles(L):
    r = _lib.Result()
    assert L.usp_solve(None, None, None, 0, 1e-6, 10, 0.0, ctypes.byref(r)) == _lib.ERR_INVALID_ARG
    n = ctypes.c_int32()
    assert L.usp_residual_history(None, None, 0, ctypes.byref(n)) == _lib.ERR_INVALID_ARG
    assert L.usp_batch_history(None, 0, None, 0, ctypes.byref(n)) == _lib.ERR_INVALID_ARG
    assert L.usp_batch_solve(None, None, None, 0, 1e-6, 10, None, None,
                             None) == _lib.ERR_INVALID_ARG
    L.usp_solver_destroy(None)


@pytest.mark.parametrize("make", [
    lambda: inputs.helmholtz_2d(64, 2, abl_width=8),
    lambda: inputs.random_helmholtz((8, 16, 16), 5),
])
def test_canonical_helmholtz_matches_oracle(L, make):
    prob = make()
    p = pcanon.canonical(prob)
    o = ocanon.canonical(prob)
    assert p["bias"] == pytest.approx(o["bias"], rel=1e-12, abs=1e-12)
    assert p["c"] == pytest.approx(o["c"], rel=1e-12)
    assert p["a"] == pytest.approx(o["a"], rel=1e-12)
    assert p["b"] == pytest.approx(o["b"], rel=1e-12)
    # complex64 outputs equal the rounded FP64 values to float rounding
    assert np.max(np.abs(p["V"] - o["V"])) <= 1e-7 * np.max(np.abs(o["V"]))
    assert np.max(np.abs(p["y"] - o["y"])) <= 1e-7 * np.max(np.abs(o["y"]))
    assert np.max(np.abs(p["V"])) == pytest.approx(0.95, rel=1e-6)


def test_canonical_diffusion_matches_oracle(L):
    prob = inputs.random_diffusion((16, 8, 8), 6)
    p = pcanon.canonical(prob)
    o = ocanon.canonical(prob)
    assert p["V"].dtype == np.float32
    assert p["c"].real == pytest.approx(o["c"], rel=1e-12)
    assert p["a"] == pytest.approx(o["a"], rel=1e-12)
    assert p["b"] == pytest.approx(o["b"], rel=1e-12)
    assert np.max(np.abs(p["V"] - o["V"].real)) <= 1e-7


def test_canonical_rejects_homogeneous_medium(L):
    prob = inputs.random_helmholtz((8, 8), 1)
    prob["k2"] = np.full((8, 8), 2.0 + 0.1j)
    with pytest.raises(_lib.UspError):
        pcanon.canonical(prob)
