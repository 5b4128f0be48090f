"""Python face of the learned coarse correction of libraspml (an extra
FGMRES stage; the paper has no learned component). Argument marshalling
only: the network runs in the library's tensor-core kernels.

Parameters are exchanged as one FP32 vector in the layer order of the C ABI:
per layer W[co][ci][3][3] then b[co]; `pack` and `unpack` convert to and
from a list of (W, b) arrays.
"""
from __future__ import annotations

from ctypes import byref, c_double, c_void_p

import numpy as np
import torch

from . import _lib

CHANNELS = (2, 32, 32, 32, 32, 32, 2)


def pack(params) -> np.ndarray:
    return np.concatenate([np.concatenate([np.asarray(W, np.float32).ravel(), np.asarray(b, np.float32).ravel()])
                           for W, b in params]).astype(np.float32)


def unpack(vec: np.ndarray):
    out, o = [], 0
    for l in range(len(CHANNELS) - 1):
        ci, co = CHANNELS[l], CHANNELS[l + 1]
        W = vec[o:o + co * ci * 9].reshape(co, ci, 3, 3)
        o += co * ci * 9
        out.append((W, vec[o:o + co]))
        o += co
    return out


class Net:
    """Device network for an Nc x Nc coarse grid and batches of up to `cap` images."""

    def __init__(self, Nc: int = 256, cap: int = 8, seed: int = 0, device=None,
                 stream: torch.cuda.Stream | None = None):
        self.lib = _lib.load()
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   torch.device(device).index or 0)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.Nc, self.cap = Nc, cap
        self._h = c_void_p()
        with torch.cuda.device(self.device):
            _lib.check("ras_pml_net_create", self.lib.ras_pml_net_create(
                int(Nc), int(cap), int(seed), c_void_p(self.stream.cuda_stream), byref(self._h)))
        self.nparam = self.lib.ras_pml_net_param_count(self._h)

    def set_params(self, vec: np.ndarray) -> None:
        v = np.ascontiguousarray(vec, dtype=np.float32)
        _lib.check("ras_pml_net_set_params", self.lib.ras_pml_net_set_params(
            self._h, v.ctypes.data_as(c_void_p), int(v.size)))

    def get_params(self) -> np.ndarray:
        v = np.zeros(self.nparam, dtype=np.float32)
        _lib.check("ras_pml_net_get_params", self.lib.ras_pml_net_get_params(
            self._h, v.ctypes.data_as(c_void_p), int(v.size)))
        return v

    def forward(self, x: torch.Tensor) -> torch.Tensor:
        """x: (nimg, 2, Nc, Nc) float32 on the device -> same-shaped output."""
        if not (x.is_cuda and x.dtype == torch.float32 and x.is_contiguous() and x.dim() == 4
                and tuple(x.shape[1:]) == (2, self.Nc, self.Nc)):
            raise ValueError("expected a contiguous cuda float32 tensor (nimg, 2, Nc, Nc)")
        y = torch.empty_like(x)
        _lib.check("ras_pml_net_forward", self.lib.ras_pml_net_forward(
            self._h, c_void_p(x.data_ptr()), c_void_p(y.data_ptr()), int(x.shape[0])))
        return y

    def loss_grad(self, x: torch.Tensor, t: torch.Tensor, want_grad: bool = True):
        """(loss, gradient vector or None) of the mean loss over the images of x against t."""
        for a in (x, t):
            if not (a.is_cuda and a.dtype == torch.float32 and a.is_contiguous()
                    and tuple(a.shape[1:]) == (2, self.Nc, self.Nc)):
                raise ValueError("expected contiguous cuda float32 tensors (nimg, 2, Nc, Nc)")
        loss = c_double()
        g = np.zeros(self.nparam, dtype=np.float32) if want_grad else None
        _lib.check("ras_pml_net_loss_grad", self.lib.ras_pml_net_loss_grad(
            self._h, c_void_p(x.data_ptr()), c_void_p(t.data_ptr()), int(x.shape[0]), byref(loss),
            g.ctypes.data_as(c_void_p) if want_grad else None))
        return loss.value, g

    def adam_step(self, lr: float) -> None:
        _lib.check("ras_pml_net_adam_step", self.lib.ras_pml_net_adam_step(self._h, float(lr)))

    @property
    def gamma(self) -> float:
        return float(self.lib.ras_pml_net_get_gamma(self._h))

    @gamma.setter
    def gamma(self, value: float) -> None:
        _lib.check("ras_pml_net_set_gamma", self.lib.ras_pml_net_set_gamma(self._h, float(value)))

    def train(self, solver, nrhs: int = 4, m_list=(1, 2, 3, 4, 6, 8, 12, 16), epochs: int = 100,
              lr: float = 1e-3, seed: int = 0):
        """Train on residual/error pairs of the solver's own problem; returns
        (loss per epoch, gamma)."""
        ms = np.ascontiguousarray(m_list, dtype=np.int32)
        hist = np.zeros(int(epochs), dtype=np.float32)
        g = c_double()
        _lib.check("ras_pml_net_train", self.lib.ras_pml_net_train(
            self._h, solver._h, int(nrhs), ms.ctypes.data_as(c_void_p), int(ms.size), int(epochs), float(lr),
            int(seed), hist.ctypes.data_as(c_void_p), byref(g)))
        return hist, g.value

    def close(self) -> None:
        if getattr(self, "_h", None) and self._h.value:
            self.lib.ras_pml_net_destroy(self._h)
            self._h = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
