"""Helpers shared by the GPU tests: seeded inputs and oracle results."""
import numpy as np
import torch

import workloads
from oracle import fem, ras


def random_vector(n, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(n) + 1j * rng.standard_normal(n)


def to_dev(v):
    return torch.from_numpy(np.ascontiguousarray(v, dtype=np.complex128)).cuda()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def variant(name, **kw):
    return workloads.get(name).with_(**kw)


_cache = {}


def oracle_problem(w):
    key = repr(w.params())
    if key not in _cache:
        p = w.params()
        grid, A = fem.assemble_global(p)
        R = ras.RAS(p).factor()
        _cache[key] = (grid, A, R)
    return _cache[key]
