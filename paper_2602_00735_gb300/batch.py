"""Python face of the batched form of libraspml: many independent RAS-PML
Helmholtz problems set up, factored, applied and solved in the same kernel
launches. Argument marshalling only; every step runs in the library's CUDA
kernels.

Batch vectors are concatenations: problem q occupies elements
[offsets[q], offsets[q] + sizes[q]) of a complex128 vector of `ntot` elements;
`split` and `join` convert between a batch vector and per-problem views.
"""
from __future__ import annotations

from ctypes import byref, c_void_p

import numpy as np
import torch

from . import _lib
from .solver import _dev_ptr, make_params, tune_dict


class BatchRasPml:
    """Handle on a set of problems (one parameter dict each)."""

    def __init__(self, params_list, factor_prec: int = 1, device=None, stream: torch.cuda.Stream | None = None):
        self.lib = _lib.load()
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   torch.device(device).index or 0)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        arr = (_lib.Params * len(params_list))(*[make_params(p, factor_prec) for p in params_list])
        self._h = c_void_p()
        with torch.cuda.device(self.device):
            _lib.check("ras_pml_batch_setup", self.lib.ras_pml_batch_setup(
                arr, len(params_list), c_void_p(self.stream.cuda_stream), byref(self._h)))
        inf = self.info()
        self.nprob, self.ntot = inf["nprob"], inf["ntot"]
        off = np.zeros(self.nprob, dtype=np.int64)
        siz = np.zeros(self.nprob, dtype=np.int64)
        _lib.check("ras_pml_batch_layout", self.lib.ras_pml_batch_layout(
            self._h, off.ctypes.data_as(c_void_p), siz.ctypes.data_as(c_void_p)))
        self.offsets, self.sizes = off, siz

    def info(self) -> dict:
        inf = _lib.BatchInfo()
        _lib.check("ras_pml_batch_info", self.lib.ras_pml_batch_info(self._h, byref(inf)))
        return {name: getattr(inf, name) for name, _ in _lib.BatchInfo._fields_}

    # -- vectors ---------------------------------------------------------------
    def empty(self) -> torch.Tensor:
        return torch.empty(self.ntot, dtype=torch.complex128, device=self.device)

    def split(self, v: torch.Tensor):
        """Per-problem views of a batch vector."""
        return [v[int(o):int(o) + int(n)] for o, n in zip(self.offsets, self.sizes)]

    def join(self, parts) -> torch.Tensor:
        """A batch vector from per-problem vectors (gaps zero)."""
        v = torch.zeros(self.ntot, dtype=torch.complex128, device=self.device)
        for o, n, p in zip(self.offsets, self.sizes, parts):
            v[int(o):int(o) + int(n)] = torch.as_tensor(p, dtype=torch.complex128).to(self.device)
        return v

    # -- set-up ----------------------------------------------------------------
    def assemble_rhs(self, sources) -> torch.Tensor:
        """sources: per problem (centres (ns, 2), amps (ns,), width)."""
        ns = np.array([len(np.ravel(a)) for _, a, _ in sources], dtype=np.int32)
        cen = np.ascontiguousarray(np.concatenate(
            [np.asarray(c, dtype=np.float64).reshape(-1, 2) for c, _, _ in sources] + [np.zeros((0, 2))]))
        amp = np.ascontiguousarray(np.concatenate(
            [np.asarray(a, dtype=np.float64).ravel() for _, a, _ in sources] + [np.zeros(0)]))
        wid = np.ascontiguousarray(np.array([w for _, _, w in sources], dtype=np.float64))
        b = self.empty()
        _lib.check("ras_pml_batch_assemble_rhs", self.lib.ras_pml_batch_assemble_rhs(
            self._h, ns.ctypes.data_as(c_void_p), cen.ctypes.data_as(c_void_p), amp.ctypes.data_as(c_void_p),
            wid.ctypes.data_as(c_void_p), c_void_p(_dev_ptr(b, self.ntot))))
        return b

    def factor(self) -> None:
        _lib.check("ras_pml_batch_factor", self.lib.ras_pml_batch_factor(self._h))

    def tune(self) -> dict:
        rep = _lib.TuneReport()
        _lib.check("ras_pml_batch_tune", self.lib.ras_pml_batch_tune(self._h, byref(rep)))
        return tune_dict(rep)

    def set_shapes(self, factor_threads: int, factor_rank: int, apply_cols: int, wide_cluster: int = 0) -> None:
        """Tile shapes (e.g. another batch's tuning); wide_cluster 0: automatic."""
        _lib.check("ras_pml_batch_set_shapes",
                   self.lib.ras_pml_batch_set_shapes(self._h, int(factor_threads), int(factor_rank), int(apply_cols),
                                                     int(wide_cluster)))

    # -- operators and solver ----------------------------------------------------
    def apply(self, r: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        z = self.empty() if out is None else out
        _lib.check("ras_pml_batch_apply", self.lib.ras_pml_batch_apply(
            self._h, c_void_p(_dev_ptr(r, self.ntot)), c_void_p(_dev_ptr(z, self.ntot))))
        return z

    def matvec(self, x: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        y = self.empty() if out is None else out
        _lib.check("ras_pml_batch_matvec", self.lib.ras_pml_batch_matvec(
            self._h, c_void_p(_dev_ptr(x, self.ntot)), c_void_p(_dev_ptr(y, self.ntot))))
        return y

    def solve(self, b: torch.Tensor, rtol: float = 1e-6, maxit: int = 500, restart: int = 0,
              out: torch.Tensor | None = None):
        """Lockstep FGMRES of every problem from x0 = 0; returns
        (x, iterations per problem, true relative residual per problem, status)."""
        x = self.empty() if out is None else out
        it = np.zeros(self.nprob, dtype=np.int32)
        rel = np.zeros(self.nprob, dtype=np.float64)
        st = self.lib.ras_pml_batch_solve(self._h, c_void_p(_dev_ptr(b, self.ntot)),
                                          c_void_p(_dev_ptr(x, self.ntot)), float(rtol), int(maxit), int(restart),
                                          it.ctypes.data_as(c_void_p), rel.ctypes.data_as(c_void_p))
        _lib.check("ras_pml_batch_solve", st, allow_not_converged=True)
        return x, it, rel, st

    def close(self) -> None:
        if getattr(self, "_h", None) and self._h.value:
            self.lib.ras_pml_batch_destroy(self._h)
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
