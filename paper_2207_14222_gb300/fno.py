"""Python front end of the warm-start network (include/usp.h, "learned
initial estimate"): argument marshalling only; every step runs in the
library's kernels.

The network maps the medium and the source of a 2-D Helmholtz problem to an
estimate of its field; a solve takes that estimate as x0 (``use_x0=True``)
and still stops on Algorithm 1's alpha-free denominator, so the converged
answer is the iteration's own.
"""

import ctypes

import numpy as np

from . import _lib
from ._lib import FnoConfig, check
from .inputs import K0_QUARTER_WAVE

C_IN = 3


def features(problem):
    """Input channels of a Helmholtz problem (host float32, 3 x H x W):
    Re k^2 / k0^2 - 1, Im k^2 / k0^2, and the real part of the source."""
    k2 = np.asarray(problem["k2"])
    k0 = problem.get("k0", K0_QUARTER_WAVE)
    return np.stack([k2.real / k0 ** 2 - 1.0, k2.imag / k0 ** 2,
                     np.real(problem["S"])]).astype(np.float32)


class FNO:
    """Fourier neural operator on h x w images (c_in input channels, width
    hidden channels, `layers` spectral layers keeping modes x modes
    frequencies), parameters drawn from `seed`."""

    def __init__(self, h=128, w=128, c_in=C_IN, width=32, layers=4, modes=16, max_batch=32,
                 seed=0, device=None, stream=None):
        import torch
        L = _lib.lib()
        self.cfg = FnoConfig(h, w, c_in, width, layers, modes, max_batch)
        self.device = torch.device(device or "cuda:0")
        self.nparam = int(L.usp_fno_param_count(ctypes.byref(self.cfg)))
        if self.nparam < 0:
            raise ValueError(_lib.last_error())
        if stream is None:
            stream = torch.cuda.current_stream(self.device).cuda_stream
        h_ = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            check(L.usp_fno_create(ctypes.byref(self.cfg), int(seed), ctypes.c_void_p(stream),
                                   ctypes.byref(h_)))
        self._h = h_

    def _check_inputs(self, a, x=None):
        import torch
        if not a.is_cuda or a.dtype != torch.float32 or a.dim() != 4:
            raise ValueError("a must be a CUDA float32 tensor (batch, c_in, h, w)")
        if tuple(a.shape[1:]) != (self.cfg.c_in, self.cfg.h, self.cfg.w):
            raise ValueError("a has shape %s" % (tuple(a.shape),))
        if x is not None and (x.dtype != torch.complex64 or
                              tuple(x.shape) != (a.shape[0], self.cfg.h, self.cfg.w)):
            raise ValueError("x must be complex64 (batch, h, w)")
        return a.contiguous(), None if x is None else x.contiguous()

    @property
    def params(self):
        out = np.empty(self.nparam, np.float32)
        check(_lib.lib().usp_fno_get_params(
            self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), self.nparam))
        return out

    @params.setter
    def params(self, value):
        v = np.ascontiguousarray(value, dtype=np.float32)
        check(_lib.lib().usp_fno_set_params(
            self._h, v.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), v.size))

    def predict(self, a):
        """Field estimates (batch, h, w) complex64 for inputs a."""
        import torch
        a, _ = self._check_inputs(a)
        x = torch.empty((a.shape[0], self.cfg.h, self.cfg.w), dtype=torch.complex64,
                        device=a.device)
        with torch.cuda.device(self.device):
            check(_lib.lib().usp_fno_predict(self._h, ctypes.c_void_p(a.data_ptr()),
                                             int(a.shape[0]), ctypes.c_void_p(x.data_ptr())))
        return x

    def gradients(self, a, x):
        """(loss, gradient vector) without an update."""
        import torch
        a, x = self._check_inputs(a, x)
        g = np.empty(self.nparam, np.float32)
        loss = ctypes.c_double()
        with torch.cuda.device(self.device):
            check(_lib.lib().usp_fno_gradients(
                self._h, ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                int(a.shape[0]), g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                ctypes.byref(loss)))
        return loss.value, g

    def train_step(self, a, x, lr=1e-3):
        """One Adam step on a batch; returns the loss before the update."""
        import torch
        a, x = self._check_inputs(a, x)
        loss = ctypes.c_double()
        with torch.cuda.device(self.device):
            check(_lib.lib().usp_fno_train_step(
                self._h, ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                int(a.shape[0]), float(lr), ctypes.byref(loss)))
        return loss.value

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.lib().usp_fno_destroy(self._h)
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
