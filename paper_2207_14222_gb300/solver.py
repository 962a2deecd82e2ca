"""Python front end of the GB300 solver: torch tensors in, torch tensors out.

Marshals arguments to the C ABI (include/usp.h); PyTorch provides device
memory and streams only.  There is no CPU path: without the built library
or a CUDA device every call raises.
"""

import ctypes

import numpy as np

from . import _lib
from ._lib import Grid, LSymbol, Options, Result, check


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def kernel_launches():
    """Kernel launches issued by the library so far in this process."""
    return int(_lib.lib().usp_kernel_launches())


class Solver:
    """Fixed-point iteration with the universal split preconditioner for the
    canonical system (L + V) x = y (Algorithm 1, forward-eliminated form).

    shape : grid shape (1-3 axes, each a power of two in [2, 256] or 96, 192,
            384, 512), last axis fastest.
    a, b  : symbol Lhat(p) = a |p|^2 + b (complex).
    V     : CUDA tensor of the potential, complex64 (or float32 for a real
            potential), copied at construction.
    alpha : step size; <= 0 selects Re[B^-1] = min Re 1/(1 - V).
    plain : True runs Algorithm 1 exactly (no FP64 refinement).
    schedule : 0 auto, 1 pencil passes, 2 fused two-pass 3-D schedule,
            3 on-chip (square 2-D grids of side 32, 64, 96, 128, 192, 256:
            the fields stay in one thread-block cluster's shared memory),
            4 split-y two-pass 3-D schedule (nz x 256 x 256, nz in 32..256).
    no_tma : True loads the strided-axis passes with plain global accesses.
    cols_tile : columns per staged strided-axis tile (8, 16, 32; 0 default).
    tc_dft : True runs the 256-point strided-axis transforms on the tensor cores.
    lhat_table : complex64 CUDA tensor of Lhat on the grid's frequencies (FFT
            order) instead of a |p|^2 + b.
    onchip_rows : rows per CTA of the on-chip schedule (8, 16; 0 default).
    residual_fp64 : True forms the refinement residual (and apply_A, residual)
            in FP64 instead of double-float.
    """

    def __init__(self, shape, a, b, V, alpha=0.0, dx=1.0, stream=None, plain=False,
                 schedule=0, chunk=0, max_refinements=0, no_tma=False, cols_tile=0,
                 tc_dft=False, lhat_table=None, onchip_rows=0, residual_fp64=False):
        """Lhat(p) = a |p|^2 + b, or, with `lhat_table` (a complex64 CUDA tensor of the
        grid's shape, k-space in FFT order), the tabulated symbol; a and b are then
        ignored."""
        import torch
        L = _lib.lib()
        if not V.is_cuda:
            raise ValueError("V must be a CUDA tensor")
        if V.dtype not in (torch.complex64, torch.float32):
            raise ValueError("V must be complex64 or float32")
        V = V.contiguous()
        self.shape = tuple(int(n) for n in shape)
        if int(np.prod(self.shape)) != V.numel():
            raise ValueError("V has %d elements, grid %s" % (V.numel(), self.shape))
        self.device = V.device
        g = Grid()
        g.ndim = len(self.shape)
        for i in range(3):
            g.n[i] = self.shape[i] if i < len(self.shape) else 1
        g.dx = float(dx)
        sym = LSymbol(complex(a).real, complex(a).imag, complex(b).real, complex(b).imag)
        if lhat_table is not None:
            if (not lhat_table.is_cuda or lhat_table.dtype != torch.complex64
                    or tuple(lhat_table.shape) != self.shape):
                raise ValueError("lhat_table must be a complex64 CUDA tensor of shape %s"
                                 % (self.shape,))
            lhat_table = lhat_table.contiguous()
            sym.kind = 1
            sym.table = _ptr(lhat_table)
        if stream is None:
            stream = torch.cuda.current_stream(self.device).cuda_stream
        self._stream = stream
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            check(L.usp_solver_create(ctypes.byref(g), ctypes.byref(sym), _ptr(V),
                                      int(V.dtype == torch.float32), float(alpha),
                                      ctypes.c_void_p(stream), ctypes.byref(h)))
        self._h = h
        self.set_options(plain=plain, schedule=schedule, chunk=chunk,
                         max_refinements=max_refinements, no_tma=no_tma, cols_tile=cols_tile,
                         tc_dft=tc_dft, onchip_rows=onchip_rows, residual_fp64=residual_fp64)

    def set_options(self, plain=False, schedule=0, chunk=0, max_refinements=0, no_tma=False,
                    cols_tile=0, tc_dft=False, onchip_rows=0, test_wait_fault=False,
                    residual_fp64=False):
        o = Options(int(bool(plain)), int(schedule), int(chunk), int(max_refinements),
                    int(bool(no_tma)), int(cols_tile), int(bool(tc_dft)), int(onchip_rows),
                    int(bool(test_wait_fault)), int(bool(residual_fp64)))
        check(_lib.lib().usp_solver_set_options(self._h, ctypes.byref(o)))

    @property
    def alpha(self):
        v = ctypes.c_double()
        check(_lib.lib().usp_solver_alpha(self._h, ctypes.byref(v)))
        return v.value

    def solve(self, y, x=None, tol=1e-6, maxit=10000, ref_norm=0.0, use_x0=False,
              allow_not_converged=True):
        """Run the iteration; returns (x, result dict).  ``x`` (a CUDA
        complex64 tensor) is updated in place and holds x0 if use_x0."""
        import torch
        y = y.contiguous()
        if x is None:
            x = torch.empty_like(y)
            use_x0 = False
        res = Result()
        allow = (_lib.OK, _lib.ERR_NOT_CONVERGED) if allow_not_converged else (_lib.OK,)
        with torch.cuda.device(self.device):
            st = _lib.lib().usp_solve(self._h, _ptr(y), _ptr(x), int(bool(use_x0)), float(tol),
                                      int(maxit), float(ref_norm), ctypes.byref(res))
        check(st, allow)
        d = res.as_dict()
        d["status"] = _lib.STATUS[st]
        return x, d

    def solve_host(self, y_host, x_host, tol=1e-6, maxit=10000, ref_norm=0.0, use_x0=False):
        """Same solve with host (CPU, ideally pinned) complex64 tensors."""
        res = Result()
        st = _lib.lib().usp_solve_host(self._h, _ptr(y_host), _ptr(x_host), int(bool(use_x0)),
                                       float(tol), int(maxit), float(ref_norm),
                                       ctypes.byref(res))
        check(st, (_lib.OK, _lib.ERR_NOT_CONVERGED))
        d = res.as_dict()
        d["status"] = _lib.STATUS[st]
        return x_host, d

    def history(self):
        n = ctypes.c_int32()
        check(_lib.lib().usp_residual_history(self._h, None, 0, ctypes.byref(n)))
        out = np.zeros(n.value, np.float64)
        if n.value:
            check(_lib.lib().usp_residual_history(
                self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n.value,
                ctypes.byref(n)))
        return out

    def time_passes(self, y, x, iters=10):
        """Per-kernel mean durations (CUDA events) of one iteration's
        kernels; returns a list of dicts {name, ms, bytes, launches}."""
        import torch
        out = (_lib.PassTime * 16)()
        n = ctypes.c_int32()
        with torch.cuda.device(self.device):
            check(_lib.lib().usp_time_passes(self._h, _ptr(y), _ptr(x), int(iters), out, 16,
                                             ctypes.byref(n)))
        return [dict(name=out[i].name.decode(), ms=out[i].ms, bytes=out[i].bytes,
                     launches=out[i].launches) for i in range(n.value)]

    def autotune(self, y, x=None, iters=5):
        """Time the pass variants this grid admits on (y, x) and keep the
        fastest (cached per grid shape for the process); returns the chosen
        options as a dict.  x, if given, is overwritten."""
        import torch
        y = y.contiguous()
        if x is None:
            x = torch.empty_like(y)
        o = Options()
        with torch.cuda.device(self.device):
            check(_lib.lib().usp_autotune(self._h, _ptr(y), _ptr(x), int(iters),
                                          ctypes.byref(o)))
        return dict(schedule=o.schedule, no_tma=bool(o.no_tma), chunk=o.chunk,
                    cols_tile=o.cols_tile)

    def apply_A(self, x):
        """A x = L x + V x in FP64 arithmetic (complex64 in and out)."""
        import torch
        x = x.contiguous()
        out = torch.empty_like(x)
        with torch.cuda.device(self.device):
            check(_lib.lib().usp_apply_A(self._h, _ptr(x), _ptr(out)))
        return out

    def residual(self, x, y):
        """(y - A x, ||y - A x|| / ||y||), FP64 arithmetic."""
        import torch
        x, y = x.contiguous(), y.contiguous()
        r = torch.empty_like(x)
        rel = ctypes.c_double()
        with torch.cuda.device(self.device):
            check(_lib.lib().usp_residual(self._h, _ptr(x), _ptr(y), _ptr(r), ctypes.byref(rel)))
        return r, rel.value

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.lib().usp_solver_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class BatchSolver(Solver):
    """``count`` independent problems (L_j + V_j) x_j = y_j on one grid, every
    pass of the iteration run once over all of them, each problem with its
    own symbol, step, convergence test, history and refinement.

    shape : grid of one problem (2 or 3 axes).
    a, b  : sequences of ``count`` symbol coefficients.
    V     : CUDA tensor (count, *shape), complex64 or float32.
    alpha : scalar or sequence of ``count`` (<= 0: automatic).
    """

    def __init__(self, shape, a, b, V, alpha=0.0, dx=1.0, stream=None, plain=False,
                 schedule=0, chunk=0, max_refinements=0, no_tma=False, onchip_rows=0):
        import torch
        L = _lib.lib()
        if not V.is_cuda:
            raise ValueError("V must be a CUDA tensor")
        if V.dtype not in (torch.complex64, torch.float32):
            raise ValueError("V must be complex64 or float32")
        V = V.contiguous()
        self.shape = tuple(int(n) for n in shape)
        self.count = int(V.shape[0])
        if int(np.prod(self.shape)) * self.count != V.numel():
            raise ValueError("V has %d elements, %d problems of grid %s"
                             % (V.numel(), self.count, self.shape))
        a, b = list(a), list(b)
        if len(a) != self.count or len(b) != self.count:
            raise ValueError("need one symbol per problem")
        alphas = list(alpha) if hasattr(alpha, "__len__") else [alpha] * self.count
        if len(alphas) != self.count:
            raise ValueError("need one alpha per problem")
        self.device = V.device
        g = Grid()
        g.ndim = len(self.shape)
        for i in range(3):
            g.n[i] = self.shape[i] if i < len(self.shape) else 1
        g.dx = float(dx)
        syms = (LSymbol * self.count)(*[
            LSymbol(complex(aj).real, complex(aj).imag, complex(bj).real, complex(bj).imag)
            for aj, bj in zip(a, b)])
        al = (ctypes.c_double * self.count)(*[float(v) for v in alphas])
        if stream is None:
            stream = torch.cuda.current_stream(self.device).cuda_stream
        self._stream = stream
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            check(L.usp_batch_create(ctypes.byref(g), self.count, syms, _ptr(V),
                                     int(V.dtype == torch.float32), al,
                                     ctypes.c_void_p(stream), ctypes.byref(h)))
        self._h = h
        self.set_options(plain=plain, schedule=schedule, chunk=chunk,
                         max_refinements=max_refinements, no_tma=no_tma, onchip_rows=onchip_rows)

    def solve(self, y, x=None, tol=1e-6, maxit=10000, ref_norms=None, use_x0=False,
              allow_failed=True):
        """Solve all problems; returns (x, list of per-problem result dicts,
        each with its own "status").  With allow_failed, a problem that did
        not converge, diverged or met a non-finite value is reported in its
        status instead of raising."""
        import torch
        y = y.contiguous()
        if x is None:
            x = torch.empty_like(y)
            use_x0 = False
        res = (Result * self.count)()
        sts = (ctypes.c_int32 * self.count)()
        refs = None
        if ref_norms is not None:
            refs = (ctypes.c_double * self.count)(*[float(v) for v in ref_norms])
        allow = ((_lib.OK, _lib.ERR_NOT_CONVERGED, _lib.ERR_DIVERGED, _lib.ERR_NONFINITE)
                 if allow_failed else (_lib.OK,))
        with torch.cuda.device(self.device):
            st = _lib.lib().usp_batch_solve(self._h, _ptr(y), _ptr(x), int(bool(use_x0)),
                                            float(tol), int(maxit), refs, res, sts)
        check(st, allow)
        out = []
        for j in range(self.count):
            d = res[j].as_dict()
            d["status"] = _lib.STATUS[sts[j]]
            out.append(d)
        return x, out

    def solve_host(self, *args, **kwargs):
        raise NotImplementedError("a batch is solved from device tensors (BatchSolver.solve)")

    def history(self, problem=0):
        n = ctypes.c_int32()
        check(_lib.lib().usp_batch_history(self._h, int(problem), None, 0, ctypes.byref(n)))
        out = np.zeros(n.value, np.float64)
        if n.value:
            check(_lib.lib().usp_batch_history(
                self._h, int(problem), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                n.value, ctypes.byref(n)))
        return out


def solve_many(solvers, ys, xs=None, tol=1e-6, maxit=10000):
    """Solve several solvers (Solver or BatchSolver, any grids) concurrently,
    one host thread and stream each (usp_solve_many).  Returns (xs, results)
    with results a list per solver of per-problem result dicts."""
    import torch
    n = len(solvers)
    if len(ys) != n:
        raise ValueError("one source per solver")
    ys = [y.contiguous() for y in ys]
    use_x0 = xs is not None
    if xs is None:
        xs = [torch.empty_like(y) for y in ys]
    counts = [getattr(s, "count", 1) for s in solvers]
    total = sum(counts)
    res = (Result * total)()
    sts = (ctypes.c_int32 * total)()
    hs = (ctypes.c_void_p * n)(*[s._h.value for s in solvers])
    yp = (ctypes.c_void_p * n)(*[y.data_ptr() for y in ys])
    xp = (ctypes.c_void_p * n)(*[x.data_ptr() for x in xs])
    st = _lib.lib().usp_solve_many(hs, n, yp, xp, int(use_x0), float(tol), int(maxit), res,
                                   sts)
    check(st, (_lib.OK, _lib.ERR_NOT_CONVERGED, _lib.ERR_DIVERGED, _lib.ERR_NONFINITE))
    out, k = [], 0
    for c in counts:
        lst = []
        for _ in range(c):
            d = res[k].as_dict()
            d["status"] = _lib.STATUS[sts[k]]
            lst.append(d)
            k += 1
        out.append(lst)
    return xs, out


class VariantSolver:
    """Algorithm 1 on a block form of the canonical system (usp_variant_*):
    kind "antisymmetric" (K = 2) or "flux" (K = 1 + ndim).  params and V as
    returned by canon.antisymmetric / canon.flux_diffusion; V a CUDA tensor
    (complex64 grid, or float32 (2,) + grid for the flux form)."""

    KINDS = {"antisymmetric": 1, "flux": 2}

    def __init__(self, shape, kind, params, V, alpha=0.0, dx=1.0, stream=None, schedule=0):
        """schedule: 0 automatic (on chip for square 2-D grids up to 128^2), 1 the
        passes, 3 on chip."""
        import torch
        if not V.is_cuda:
            raise ValueError("V must be a CUDA tensor")
        self.shape = tuple(int(n) for n in shape)
        self.kind = kind
        self.K = 2 if kind == "antisymmetric" else 1 + len(self.shape)
        V = V.contiguous()
        self.device = V.device
        g = Grid()
        g.ndim = len(self.shape)
        for i in range(3):
            g.n[i] = self.shape[i] if i < len(self.shape) else 1
        g.dx = float(dx)
        p = (ctypes.c_double * 4)(*[float(v) for v in params] + [0.0] * (4 - len(params)))
        if stream is None:
            stream = torch.cuda.current_stream(self.device).cuda_stream
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            check(_lib.lib().usp_variant_create(ctypes.byref(g), self.KINDS[kind], p, _ptr(V),
                                                float(alpha), ctypes.c_void_p(stream),
                                                ctypes.byref(h)))
        self._h = h
        if schedule:
            try:
                check(_lib.lib().usp_variant_set_schedule(h, int(schedule)))
            except Exception:
                self.close()
                raise

    def solve(self, y, x=None, tol=1e-5, maxit=20000, ref_norm=0.0, use_x0=False,
              allow_not_converged=True):
        """y, x: CUDA complex64 tensors (K,) + grid; returns (x, result)."""
        import torch
        y = y.contiguous()
        if x is None:
            x = torch.empty_like(y)
            use_x0 = False
        res = Result()
        allow = (_lib.OK, _lib.ERR_NOT_CONVERGED) if allow_not_converged else (_lib.OK,)
        with torch.cuda.device(self.device):
            st = _lib.lib().usp_variant_solve(self._h, _ptr(y), _ptr(x), int(bool(use_x0)),
                                              float(tol), int(maxit), float(ref_norm),
                                              ctypes.byref(res))
        check(st, allow)
        d = res.as_dict()
        d["status"] = _lib.STATUS[st]
        return x, d

    def history(self):
        n = ctypes.c_int32()
        check(_lib.lib().usp_variant_history(self._h, None, 0, ctypes.byref(n)))
        out = np.zeros(n.value, np.float64)
        if n.value:
            check(_lib.lib().usp_variant_history(
                self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n.value,
                ctypes.byref(n)))
        return out

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.lib().usp_variant_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
