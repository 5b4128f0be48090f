"""Python face of libraspml: one RAS-PML Helmholtz problem on one GPU.

Argument marshalling only. Torch supplies device memory and the CUDA stream;
every step of the method runs in the library's CUDA kernels.
"""
from __future__ import annotations

import ctypes
from ctypes import byref, c_double, c_int, c_void_p

import numpy as np
import torch

from . import _lib

PARAM_KEYS = ("k", "x0", "y0", "x1", "y1", "kappa_g", "h", "px", "py", "ovlp_cells", "pml_cells",
              "g_amp", "g_ramp", "local_bc")


def make_params(params: dict, factor_prec: int = 0, ortho: int = 0) -> _lib.Params:
    p = _lib.Params()
    for key in PARAM_KEYS:
        setattr(p, key, params[key])
    p.factor_prec = int(factor_prec)
    p.ortho = int(ortho)
    p.g_profile = int(params.get("g_profile", 0))
    p.form = int(params.get("form", 0))
    return p


def tune_dict(rep: _lib.TuneReport) -> dict:
    """The tuner's report; factor candidates keyed "<threads>x<rank>"."""
    return {"factor_threads": rep.factor_threads, "factor_rank": rep.factor_rank, "apply_cols": rep.apply_cols,
            "factor_ms": {f"{rep.factor_cand_threads[i]}x{rep.factor_cand_rank[i]}": rep.factor_ms[i]
                          for i in range(rep.n_factor)},
            "apply_ms": {rep.apply_cand[i]: rep.apply_ms[i] for i in range(rep.n_apply)},
            "wide_cluster": rep.wide_cluster,
            "wide_ms": {rep.wide_cand[i]: rep.wide_ms[i] for i in range(rep.n_wide)}}


def _dev_ptr(t: torch.Tensor, n: int) -> int:
    if not (t.is_cuda and t.dtype == torch.complex128 and t.is_contiguous() and t.numel() == n):
        raise ValueError(f"expected a contiguous cuda complex128 tensor of {n} elements")
    return t.data_ptr()


class RasPml:
    """Handle on a set-up problem: global matrix, covering, local factors."""

    def __init__(self, params: dict, factor_prec: int = 0, ortho: int = 0, device=None,
                 stream: torch.cuda.Stream | None = None):
        self.lib = _lib.load()
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   torch.device(device).index or 0)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        p = make_params(params, factor_prec, ortho)
        self._h = c_void_p()
        with torch.cuda.device(self.device):
            _lib.check("ras_pml_setup", self.lib.ras_pml_setup(byref(p), c_void_p(self.stream.cuda_stream),
                                                               byref(self._h)))
        self.n = self.info()["n"]

    # -- queries ---------------------------------------------------------------
    def info(self) -> dict:
        inf = _lib.Info()
        _lib.check("ras_pml_info", self.lib.ras_pml_info(self._h, byref(inf)))
        return {name: getattr(inf, name) for name, _ in _lib.Info._fields_}

    def set_timing(self, enable: bool = True) -> None:
        _lib.check("ras_pml_set_timing", self.lib.ras_pml_set_timing(self._h, int(bool(enable))))

    def timing(self) -> dict:
        t = _lib.Timing()
        _lib.check("ras_pml_get_timing", self.lib.ras_pml_get_timing(self._h, byref(t)))
        return {name: getattr(t, name) for name, _ in _lib.Timing._fields_}

    def history(self) -> np.ndarray:
        cnt = c_int()
        self.lib.ras_pml_history(self._h, None, 0, byref(cnt))
        buf = np.zeros(max(cnt.value, 1))
        _lib.check("ras_pml_history", self.lib.ras_pml_history(
            self._h, buf.ctypes.data_as(c_void_p), cnt.value, byref(cnt)))
        return buf[:cnt.value]

    # -- set-up ----------------------------------------------------------------
    def empty(self) -> torch.Tensor:
        return torch.empty(self.n, dtype=torch.complex128, device=self.device)

    def assemble_rhs(self, centres, amps, width: float) -> torch.Tensor:
        cen = np.ascontiguousarray(np.asarray(centres, dtype=np.float64).reshape(-1, 2))
        amp = np.ascontiguousarray(np.asarray(amps, dtype=np.float64).ravel())
        b = self.empty()
        _lib.check("ras_pml_assemble_rhs", self.lib.ras_pml_assemble_rhs(
            self._h, cen.ctypes.data_as(c_void_p), amp.ctypes.data_as(c_void_p), int(amp.size),
            float(width), c_void_p(_dev_ptr(b, self.n))))
        return b

    def factor(self) -> None:
        _lib.check("ras_pml_factor", self.lib.ras_pml_factor(self._h))

    def tune(self) -> dict:
        """Time the factor and apply tile shapes, keep the fastest (leaves the handle factored)."""
        rep = _lib.TuneReport()
        _lib.check("ras_pml_tune", self.lib.ras_pml_tune(self._h, byref(rep)))
        return tune_dict(rep)

    def attach_net(self, net) -> None:
        """Use net (a paper_2602_00735_gb300.net.Net, or None) as the learned FGMRES stage."""
        self._net = net
        _lib.check("ras_pml_attach_net", self.lib.ras_pml_attach_net(self._h, net._h if net is not None else None))

    def net_correct(self, net, r: torch.Tensor, z: torch.Tensor) -> torch.Tensor:
        """z += the learned correction of r (in place; returns z)."""
        _lib.check("ras_pml_net_correct", self.lib.ras_pml_net_correct(
            self._h, net._h, c_void_p(_dev_ptr(r, self.n)), c_void_p(_dev_ptr(z, self.n))))
        return z

    def set_shapes(self, factor_threads: int, factor_rank: int, apply_cols: int, wide_cluster: int = 0) -> None:
        """Tile shapes (e.g. another handle's tuning); wide_cluster 0: automatic."""
        _lib.check("ras_pml_set_shapes", self.lib.ras_pml_set_shapes(self._h, int(factor_threads), int(factor_rank),
                                                                     int(apply_cols), int(wide_cluster)))

    # -- operators -------------------------------------------------------------
    def apply(self, r: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        z = self.empty() if out is None else out
        _lib.check("ras_pml_apply", self.lib.ras_pml_apply(self._h, c_void_p(_dev_ptr(r, self.n)),
                                                           c_void_p(_dev_ptr(z, self.n))))
        return z

    def matvec(self, x: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        y = self.empty() if out is None else out
        _lib.check("ras_pml_matvec", self.lib.ras_pml_matvec(self._h, c_void_p(_dev_ptr(x, self.n)),
                                                             c_void_p(_dev_ptr(y, self.n))))
        return y

    # -- solvers ---------------------------------------------------------------
    def solve(self, b: torch.Tensor, rtol: float = 1e-6, maxit: int = 500, restart: int = 0,
              x0: torch.Tensor | None = None):
        """Flexible GMRES; returns (x, iterations, true relative residual, status)."""
        x = torch.zeros_like(b) if x0 is None else x0.clone()
        it, rel = c_int(), c_double()
        st = self.lib.helmholtz_solve(self._h, c_void_p(_dev_ptr(b, self.n)), c_void_p(_dev_ptr(x, self.n)),
                                      float(rtol), int(maxit), int(restart), byref(it), byref(rel))
        _lib.check("helmholtz_solve", st, allow_not_converged=True)
        return x, it.value, rel.value, st

    def solve_host(self, b_host: torch.Tensor, rtol: float = 1e-6, maxit: int = 500, restart: int = 0,
                   x_host: torch.Tensor | None = None):
        """helmholtz_solve_host on CPU tensors (pinned memory recommended)."""
        if b_host.is_cuda or b_host.dtype != torch.complex128 or not b_host.is_contiguous():
            raise ValueError("expected a contiguous CPU complex128 tensor")
        x = torch.zeros_like(b_host) if x_host is None else x_host
        it, rel = c_int(), c_double()
        st = self.lib.helmholtz_solve_host(self._h, c_void_p(b_host.data_ptr()), c_void_p(x.data_ptr()),
                                           float(rtol), int(maxit), int(restart), byref(it), byref(rel))
        _lib.check("helmholtz_solve_host", st, allow_not_converged=True)
        return x, it.value, rel.value, st

    def richardson(self, b: torch.Tensor, rtol: float = 1e-6, maxit: int = 500, x0: torch.Tensor | None = None):
        """Algorithm 1 (discrete form); returns (x, sweeps, relres, status)."""
        x = torch.zeros_like(b) if x0 is None else x0.clone()
        it, rel = c_int(), c_double()
        st = self.lib.ras_pml_richardson(self._h, c_void_p(_dev_ptr(b, self.n)), c_void_p(_dev_ptr(x, self.n)),
                                         float(rtol), int(maxit), byref(it), byref(rel))
        _lib.check("ras_pml_richardson", st, allow_not_converged=True)
        return x, it.value, rel.value, st

    def close(self) -> None:
        if getattr(self, "_h", None) and self._h.value:
            self.lib.ras_pml_destroy(self._h)
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
