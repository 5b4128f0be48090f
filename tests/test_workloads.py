"""The seeded workloads hold what their recipes state (no method arithmetic
here: sizes, ranges and the covering's band widths from the oracle)."""
import math

import numpy as np
import pytest

import workloads
from oracle import ras


def _max_band(w):
    grid, rxs, rys = ras.covering(w.params())
    nl = [min(r.ext_hi, grid.Mx - 1) - max(r.ext_lo, 1) + 1 for r in rxs]   # impedance: ext nodes
    return max(nl) + 1


@pytest.mark.parametrize("name", ["c3", "c3small"])
def test_batch_recipe(name):
    probs = workloads.batch(name)
    lo, hi = (20 * math.pi, 120 * math.pi) if name == "c3" else (8 * math.pi, 24 * math.pi)
    assert len(probs) == (64 if name == "c3" else 8)
    for w in probs:
        assert lo <= w.k <= hi
        side = w.x1 - w.x0
        assert 0.5 <= side <= 1.5 and w.y1 - w.y0 == side and w.kappa_g == 0.1
        # about 16 points per wavelength, Omega whole cells
        ppw = 2 * math.pi / (w.k * w.h)
        assert abs(ppw - 16) <= 16 * 0.05
        assert abs(w.cells_x * w.h - (side + 0.2)) < 1e-12
        assert w.ovlp_cells == w.pml_cells == workloads.width_cells(w.k, w.h)
        assert 2 <= w.px <= 12 and 2 <= w.py <= 12
        assert 1 <= len(w.amps) <= 8 and abs(w.width * w.k - 0.4 * math.pi) < 1e-12
        assert w.cells_x // w.px >= 2 * w.ovlp_cells
    assert len({(w.px, w.py) for w in probs}) > 1 and any(w.px != w.py for w in probs)


def test_c3_grids_are_drawn_uniformly_without_a_band_filter():
    """c3: px and py independent and uniform in 2..12. The draws are
    the generator's own: the same integers as rng.integers(2, 13, size=2) at
    that point of the sequence, so nothing narrows them to what a kernel can
    hold; the widest local band follows from them (408 with seed 3)."""
    probs = workloads.batch("c3")
    grids = np.array([(w.px, w.py) for w in probs])
    assert grids.min() == 2 and grids.max() == 12
    assert max(_max_band(w) for w in probs) > 232        # beyond the old window limit
    rng = np.random.default_rng(3)
    for w in probs:                                       # replay the draw order
        k = float(np.exp(rng.uniform(math.log(20 * math.pi), math.log(120 * math.pi))))
        rng.uniform(0.5, 1.5)
        px, py = (int(v) for v in rng.integers(2, 13, size=2))
        ns = int(rng.integers(1, 9))
        rng.uniform(0.0, 1.0, size=(ns, 2))
        assert (w.k, w.px, w.py, len(w.amps)) == (k, px, py, ns)


def test_batch_is_seeded():
    a, b = workloads.batch("c3"), workloads.batch("c3")
    assert all(x.k == y.k and np.array_equal(x.centres, y.centres) for x, y in zip(a, b))
    c3 = workloads.batch("c3")
    assert sum(w.px * w.py for w in c3) == 3335
    assert sum(w.n_unknowns for w in c3) == 19501307


@pytest.mark.parametrize("name,k,ppw", [("c0", 20 * math.pi, 16), ("c2", 160 * math.pi, 16), ("c4", 320 * math.pi, 16)])
def test_single_recipes(name, k, ppw):
    w = workloads.get(name)
    assert w.k == k and abs(2 * math.pi / (w.k * w.h) - ppw) < 1e-9
    assert w.x0 == 0.0 and w.x1 == 1.0 and w.kappa_g == 0.1
