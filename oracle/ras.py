"""Oracle, part 2: the RAS-PML preconditioner (paper Section 2 and Section 3 (ii)).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Cartesian covering (Section 2): the cells of Omega are split into px x py
non-overlapping boxes (the first Mx mod px boxes one cell wider). Omega_j,int
is the box widened by `ovlp` cells on every side that is not on the outer
boundary (the overlap delta, read as a per-side extension). Omega_j is
Omega_j,int widened by `pml` cells (kappa) on the same sides, clamped to Omega.

Local stretching (Section 2): g_j equals the global g_i inside Omega_j,int and
restarts as g(x - b_j) beyond an interior side b_j (resp. -g(a_j - x) below
a_j); on sides that lie on the outer boundary the global stretching is kept.

Local operator A_j (Section 2 and Section 3 (ii)): the form a(.,.) of the
global problem with g replaced by g_j, assembled on the elements of Omega_j.
With local_bc = 0 (RAS-PML-Imp, the paper's default from Section 4.1 on) the
nodes on the artificial boundary of Omega_j are unknowns and the impedance
condition d_nu u - i k u = 0 (eq. impedance) enters as the natural term
-i k int gamma_t u v ds (gamma_t: the local stretch along the edge), each edge
integral by 2-point Gauss. With local_bc = 1 (RAS-PML-Drch) those nodes are
dropped (Dirichlet). Nodes on the outer boundary are always Dirichlet.

With form = 1 (eq. weak as printed, not symmetric) the element terms carry
D = diag(gamma^-2) and the beta term with the local gamma_j and its
derivative, and the impedance condition, read in the stretched normal
coordinate (gamma_n^-1 d_nu u = i k u), enters as -i k int gamma_n^-1 u v ds:
the same local problem as form 0's, tested with v/(gamma_1 gamma_2).

Partition of unity (Section 2, Section 4): chi_j is the tensor product of 1D
weights that are 1 on the box away from the overlaps and vary linearly across
every overlap strip (2*ovlp cells centred on the box edge), reaching 0 on the
boundary of Omega_j,int; zero in the local PML.

Preconditioner (Section 2, the equation defining B^-1):
    B^-1 r = sum_j R_j^T ( chi_j * A_j^-1 (R_j r) ),
R_j the 0/1 restriction of global unknowns to Omega_j's unknowns. Local
factors are SciPy's SuperLU (with pivoting); the CUDA path factors without
pivoting, which agrees up to rounding.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fem


def box_edges(M: int, P: int):
    """Cell indices c_0 = 0 < c_1 < ... < c_P = M of the non-overlapping boxes."""
    base, extra = divmod(M, P)
    sizes = [base + (1 if q < extra else 0) for q in range(P)]
    return np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)


@dataclass
class Range1D:
    """One direction of one subdomain, in cell indices."""
    box_lo: int
    box_hi: int
    int_lo: int      # Omega_j,int
    int_hi: int
    ext_lo: int      # Omega_j
    ext_hi: int
    lo_interior: bool   # side a_j is not on the outer boundary
    hi_interior: bool


def ranges_1d(M: int, P: int, ovlp: int, pml: int):
    """Per-box cell ranges in one direction (Section 2, Cartesian covering)."""
    c = box_edges(M, P)
    out = []
    for q in range(P):
        lo_int = q > 0
        hi_int = q < P - 1
        if (c[q + 1] - c[q]) < 2 * ovlp:
            raise ValueError("overlap strips wider than a box")
        ilo = c[q] - (ovlp if lo_int else 0)
        ihi = c[q + 1] + (ovlp if hi_int else 0)
        elo = max(0, ilo - (pml if lo_int else 0))
        ehi = min(M, ihi + (pml if hi_int else 0))
        out.append(Range1D(int(c[q]), int(c[q + 1]), int(ilo), int(ihi),
                           int(elo), int(ehi), lo_int, hi_int))
    return out


def pou_1d(r: Range1D, ovlp: int, M: int):
    """1D partition-of-unity weight at every node 0..M (Section 4: linear across overlaps)."""
    i = np.arange(M + 1, dtype=np.float64)
    w = np.zeros(M + 1)
    inside = (i >= r.int_lo) & (i <= r.int_hi)
    w[inside] = 1.0
    if r.lo_interior:
        a, b = r.box_lo - ovlp, r.box_lo + ovlp
        s = (i >= a) & (i <= b)
        w[s] = (i[s] - a) / (2.0 * ovlp)
    if r.hi_interior:
        a, b = r.box_hi - ovlp, r.box_hi + ovlp
        s = (i >= a) & (i <= b)
        w[s] = (b - i[s]) / (2.0 * ovlp)
    return w


def local_gamma_fn(grid: fem.Grid, r: Range1D, axis: int, amp: float, ramp: float, profile: int = 0):
    """gamma_j along one axis as a function of half-index s (Section 2, g_j).

    Beyond an interior side of Omega_j,int (s >= 2*int_hi, resp. s <= 2*int_lo)
    the stretching restarts from that side; otherwise it is the global one.
    """
    glob = fem.global_gamma_x if axis == 0 else fem.global_gamma_y
    hh = 0.5 * grid.h

    def fn(s):
        s = np.asarray(s, dtype=np.float64)
        val = glob(grid, s, amp, ramp, profile)
        if r.hi_interior:
            d = (s - 2 * r.int_hi) * hh
            val = np.where(s >= 2 * r.int_hi, 1.0 + 1j * fem.gprime(d, amp, ramp, profile), val)
        if r.lo_interior:
            d = (2 * r.int_lo - s) * hh
            val = np.where(s <= 2 * r.int_lo, 1.0 + 1j * fem.gprime(d, amp, ramp, profile), val)
        return val
    return fn


def local_dgamma_fn(grid: fem.Grid, r: Range1D, axis: int, amp: float, ramp: float, profile: int = 0):
    """gamma_j' along one axis (derivative of local_gamma_fn; eq. weak's beta, form 1).

    Beyond an interior side hi of Omega_j,int g_j = g(x - hi), so gamma_j' =
    i g''(x - hi); below an interior side lo g_j = -g(lo - x), so gamma_j' =
    -i g''(lo - x); otherwise the global derivative.
    """
    glob = fem.global_dgamma_x if axis == 0 else fem.global_dgamma_y
    hh = 0.5 * grid.h

    def fn(s):
        s = np.asarray(s, dtype=np.float64)
        val = glob(grid, s, amp, ramp, profile)
        if r.hi_interior:
            d = (s - 2 * r.int_hi) * hh
            val = np.where(s >= 2 * r.int_hi, 1j * fem.gsecond(d, amp, ramp, profile), val)
        if r.lo_interior:
            d = (2 * r.int_lo - s) * hh
            val = np.where(s <= 2 * r.int_lo, -1j * fem.gsecond(d, amp, ramp, profile), val)
        return val
    return fn


_GAUSS2 = (0.5 - 0.5 / math.sqrt(3.0), 0.5 + 0.5 / math.sqrt(3.0))


@dataclass
class Subdomain:
    rx: Range1D
    ry: Range1D
    nodes: np.ndarray    # global node ids of local unknowns, local order (x fastest)
    glob: np.ndarray     # global unknown index of each local unknown (R_j)
    chi: np.ndarray      # chi_j at each local unknown
    A: sp.csr_matrix     # local operator A_j
    nlx: int             # local unknowns per row (x)
    nly: int


def local_operator(p: dict, grid: fem.Grid, rx: Range1D, ry: Range1D):
    """Local matrix A_j, its unknowns, and R_j, chi_j (Section 2 and Section 3 (ii))."""
    amp, ramp, k = p["g_amp"], p["g_ramp"], p["k"]
    prof = p.get("g_profile", 0)
    imp = p.get("local_bc", 0) == 0
    weak = p.get("form", 0) == 1
    gx = local_gamma_fn(grid, rx, 0, amp, ramp, prof)
    gy = local_gamma_fn(grid, ry, 1, amp, ramp, prof)
    cj, ci = np.meshgrid(np.arange(ry.ext_lo, ry.ext_hi),
                         np.arange(rx.ext_lo, rx.ext_hi), indexing="ij")
    if weak:
        dgx = local_dgamma_fn(grid, rx, 0, amp, ramp, prof)
        dgy = local_dgamma_fn(grid, ry, 1, amp, ramp, prof)
        rows, cols, vals = fem.assemble_cells_weak(grid, ci, cj, gx, gy, dgx, dgy, k)
    else:
        rows, cols, vals = fem.assemble_cells(grid, ci, cj, gx, gy, k)

    # which nodes of Omega_j are local unknowns
    def keep_1d(lo, hi, M):
        i = np.arange(lo, hi + 1)
        keep = (i > 0) & (i < M)                       # outer boundary: Dirichlet
        if not imp:
            keep &= (i > lo) & (i < hi)                # artificial boundary: Dirichlet
        return i[keep]
    ix = keep_1d(rx.ext_lo, rx.ext_hi, grid.Mx)
    iy = keep_1d(ry.ext_lo, ry.ext_hi, grid.My)
    JJ, II = np.meshgrid(iy, ix, indexing="ij")
    nodes = (JJ * (grid.Mx + 1) + II).ravel()
    numbering = -np.ones((grid.Mx + 1) * (grid.My + 1), dtype=np.int64)
    numbering[nodes] = np.arange(nodes.size)

    # impedance term on the artificial boundary: -i k int gamma_t phi_a phi_b ds
    # (form 0); with form 1 the weight is 1/gamma_n, the reciprocal of the
    # stretch normal to the edge (constant along it)
    if imp:
        er, ec, ev = [], [], []
        h = grid.h

        def edge_terms(n0, n1, gam):
            # gam: gamma_t at the two Gauss points (parameter q from n0 to n1)
            for a, b in ((0, 0), (0, 1), (1, 0), (1, 1)):
                s = 0.0
                for q, gt in zip(_GAUSS2, gam):
                    phi = (1.0 - q, q)
                    s = s + 0.5 * h * gt * phi[a] * phi[b]
                er.append((n0, n1)[a])
                ec.append((n0, n1)[b])
                ev.append(-1j * k * s)

        # vertical sides x = const (tangential stretch: gamma_2; normal: gamma_1)
        for side_ok, ii in ((rx.lo_interior and rx.ext_lo > 0, rx.ext_lo),
                            (rx.hi_interior and rx.ext_hi < grid.Mx, rx.ext_hi)):
            if not side_ok:
                continue
            for jc in range(ry.ext_lo, ry.ext_hi):
                if weak:
                    gam = [1.0 / gx(2.0 * ii)] * 2
                else:
                    gam = [gy(2.0 * (jc + q)) for q in _GAUSS2]
                edge_terms(jc * (grid.Mx + 1) + ii, (jc + 1) * (grid.Mx + 1) + ii, gam)
        # horizontal sides y = const (tangential stretch: gamma_1; normal: gamma_2)
        for side_ok, jj in ((ry.lo_interior and ry.ext_lo > 0, ry.ext_lo),
                            (ry.hi_interior and ry.ext_hi < grid.My, ry.ext_hi)):
            if not side_ok:
                continue
            for ic in range(rx.ext_lo, rx.ext_hi):
                if weak:
                    gam = [1.0 / gy(2.0 * jj)] * 2
                else:
                    gam = [gx(2.0 * (ic + q)) for q in _GAUSS2]
                edge_terms(jj * (grid.Mx + 1) + ic, jj * (grid.Mx + 1) + ic + 1, gam)
        if er:
            rows = np.concatenate([rows, np.array(er, dtype=np.int64)])
            cols = np.concatenate([cols, np.array(ec, dtype=np.int64)])
            vals = np.concatenate([vals, np.array(ev, dtype=np.complex128)])

    A = fem._to_matrix(rows, cols, vals, numbering, nodes.size)
    gnum = fem.interior_numbering(grid)
    glob = gnum[nodes]
    assert np.all(glob >= 0)
    return A, nodes, glob, ix.size, iy.size


def build_subdomain(p: dict, grid: fem.Grid, rx: Range1D, ry: Range1D) -> Subdomain:
    """One subdomain: local operator, R_j and chi_j."""
    ovlp = p["ovlp_cells"]
    wx = pou_1d(rx, ovlp, grid.Mx)
    wy = pou_1d(ry, ovlp, grid.My)
    A, nodes, glob, nlx, nly = local_operator(p, grid, rx, ry)
    ii = nodes % (grid.Mx + 1)
    jj = nodes // (grid.Mx + 1)
    return Subdomain(rx, ry, nodes, glob, wx[ii] * wy[jj], A, nlx, nly)


def covering(p: dict):
    """Grid and the per-direction ranges of the covering (Section 2)."""
    grid = fem.make_grid(p)
    ovlp, pml = p["ovlp_cells"], p["pml_cells"]
    if ovlp < 1:
        raise ValueError("overlap must be at least one cell")
    return grid, ranges_1d(grid.Mx, p["px"], ovlp, pml), ranges_1d(grid.My, p["py"], ovlp, pml)


def build_subdomains(p: dict):
    """All subdomains of the covering with their local operators and weights."""
    grid, rxs, rys = covering(p)
    subs = [build_subdomain(p, grid, rx, ry) for ry in rys for rx in rxs]
    return grid, subs


def local_apply(s: Subdomain, lu, r, z):
    """z += R_j^T (chi_j * A_j^-1 (R_j r)) for one subdomain."""
    c = lu.solve(r[s.glob])
    np.add.at(z, s.glob, s.chi * c)


class RAS:
    """B^-1 = sum_j R~_j^T A_j^-1 R_j with SuperLU local factors (Section 2)."""

    def __init__(self, p: dict):
        self.grid, self.subs = build_subdomains(p)
        self.n = self.grid.n
        self.lu = None

    def factor(self):
        self.lu = [spla.splu(s.A.tocsc()) for s in self.subs]
        return self

    def apply(self, r):
        if self.lu is None:
            self.factor()
        r = np.asarray(r, dtype=np.complex128)
        z = np.zeros(self.n, dtype=np.complex128)
        for s, lu in zip(self.subs, self.lu):
            local_apply(s, lu, r, z)
        return z

    def chi_sum(self):
        """sum_j R_j^T chi_j over all global unknowns (must be identically 1)."""
        t = np.zeros(self.n)
        for s in self.subs:
            np.add.at(t, s.glob, s.chi)
        return t
