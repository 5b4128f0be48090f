"""The oracle's process-pool form of B^-1 (used by the timed CPU baseline)
equals the serial oracle: the same SuperLU local solves and weights, only
the order of the final additions differs, and on these cases the sums come
out identical."""
import numpy as np
import pytest

import workloads
from oracle import pool, ras


@pytest.mark.parametrize("name,nproc", [("tiny3", 3), ("small", 2)])
def test_pool_apply_equals_serial_apply(name, nproc):
    p = workloads.get(name).params()
    R = ras.RAS(p).factor()
    rng = np.random.default_rng(4)
    r = rng.standard_normal(R.n) + 1j * rng.standard_normal(R.n)
    zr = R.apply(r)
    with pool.PoolRAS(p, nproc=nproc) as P:
        assert P.nsub == len(R.subs)
        z = P.apply(r)
        z2 = P.apply(1j * r)       # workers keep their factors between applies
    assert np.linalg.norm(z - zr) <= 1e-15 * np.linalg.norm(zr)
    assert np.linalg.norm(z2 - 1j * zr) <= 1e-15 * np.linalg.norm(zr)
