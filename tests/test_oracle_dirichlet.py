"""Exact pins of the oracle's Dirichlet closure of the local problems
(RAS-PML-Drch, local_bc = 1; Section 2: the local forms a_j on H^1_0(Omega_j),
and Section 3 (ii), where the Dirichlet and impedance closures are compared).

What fixes the Dirichlet closure independently of the oracle's own code:
  * without a local PML (pml_cells = 0) the local stretch g_j equals the global
    g on Omega_j, so the Dirichlet local matrix is the principal submatrix of
    the global matrix A at the interior nodes of Omega_j: the classical
    restricted additive Schwarz block;
  * the impedance term lives on the artificial boundary only, so the Dirichlet
    local matrix is the impedance local matrix with the artificial-boundary
    nodes removed, entry by entry;
  * B^-1 assembled densely from its definition with those local matrices.
A closure that keeps the artificial-boundary nodes without a term (Neumann),
or drops them on one side only, fails the first two (planted below, in the
oracle, on the CPU)."""

import numpy as np
import pytest

import workloads
from oracle import fem, ras


def _p(name="tiny3", **kw):
    return workloads.get(name).with_(**kw).params()


def _artificial_boundary(grid, rx, ry, nodes):
    """Mask of the local unknowns on the artificial boundary of Omega_j
    (sides of Omega_j that are interior to Omega), decided from node
    coordinates alone."""
    i = nodes % (grid.Mx + 1)
    j = nodes // (grid.Mx + 1)
    m = np.zeros(nodes.size, dtype=bool)
    if rx.lo_interior and rx.ext_lo > 0:
        m |= i == rx.ext_lo
    if rx.hi_interior and rx.ext_hi < grid.Mx:
        m |= i == rx.ext_hi
    if ry.lo_interior and ry.ext_lo > 0:
        m |= j == ry.ext_lo
    if ry.hi_interior and ry.ext_hi < grid.My:
        m |= j == ry.ext_hi
    return m


def _drch_is_imp_without_boundary(p):
    """True when, for every subdomain, A_j(Drch) equals A_j(Imp) restricted
    to the unknowns off the artificial boundary, with the same unknowns in
    the same order."""
    grid, rxs, rys = ras.covering(p)
    pi = dict(p, local_bc=0)
    pd = dict(p, local_bc=1)
    for ry in rys:
        for rx in rxs:
            Ai, nodes_i, _, _, _ = ras.local_operator(pi, grid, rx, ry)
            Ad, nodes_d, _, _, _ = ras.local_operator(pd, grid, rx, ry)
            keep = ~_artificial_boundary(grid, rx, ry, nodes_i)
            if nodes_d.size != keep.sum() or not np.array_equal(nodes_d, nodes_i[keep]):
                return False
            sub = Ai.tocsr()[keep][:, keep].toarray()
            ref = Ad.toarray()
            if np.max(np.abs(sub - ref)) > 1e-14 * np.max(np.abs(ref)):
                return False
    return True


def _drch_is_principal_submatrix(p):
    """True when, with no local PML, every A_j(Drch) equals A[glob, glob] of
    the global matrix (classical RAS with Dirichlet local problems)."""
    assert p["pml_cells"] == 0
    grid, A = fem.assemble_global(p)
    A = A.tocsr()
    grid, subs = ras.build_subdomains(dict(p, local_bc=1))
    for s in subs:
        ref = A[s.glob][:, s.glob].toarray()
        loc = s.A.toarray()
        if loc.shape != ref.shape or np.max(np.abs(loc - ref)) > 1e-13 * np.max(np.abs(ref)):
            return False
    return True


@pytest.mark.parametrize("name,px,py", [("tiny3", 3, 3), ("small", 4, 3), ("tiny", 2, 2)])
def test_dirichlet_without_local_pml_is_the_classical_ras_block(name, px, py):
    """pml_cells = 0: g_j = g on Omega_j, so A_j(Drch) = R_j A R_j^T exactly."""
    assert _drch_is_principal_submatrix(_p(name, px=px, py=py, pml_cells=0))


@pytest.mark.parametrize("name,px,py", [("tiny3", 3, 3), ("small", 4, 3), ("tiny3", 2, 3)])
def test_dirichlet_is_the_impedance_operator_without_its_boundary_nodes(name, px, py):
    """The impedance term -ik int gamma_t u v ds touches only artificial-boundary
    nodes, so removing those nodes from A_j(Imp) gives A_j(Drch)."""
    assert _drch_is_imp_without_boundary(_p(name, px=px, py=py))


def test_dirichlet_local_problem_drops_exactly_the_artificial_boundary():
    """Unknown counts: Drch keeps nlx - (interior x-sides) by nly - (interior
    y-sides) nodes of the impedance problem's nlx by nly."""
    p = _p("tiny3")
    grid, rxs, rys = ras.covering(p)
    for ry in rys:
        for rx in rxs:
            _, _, _, nlx, nly = ras.local_operator(dict(p, local_bc=0), grid, rx, ry)
            _, _, _, dlx, dly = ras.local_operator(dict(p, local_bc=1), grid, rx, ry)
            assert dlx == nlx - int(rx.lo_interior) - int(rx.hi_interior)
            assert dly == nly - int(ry.lo_interior) - int(ry.hi_interior)


def test_planted_neumann_closure_fails_both_pins(monkeypatch):
    """A Neumann closure (boundary nodes kept, no boundary term), planted in
    the oracle: with the 2-point edge rule emptied, local_bc = 0 assembles
    exactly that, and it is substituted for the Dirichlet operator."""
    orig = ras.local_operator

    def neumann(p, grid, rx, ry):
        if p.get("local_bc", 0) == 1:
            monkeypatch.setattr(ras, "_GAUSS2", ())
            try:
                return orig(dict(p, local_bc=0), grid, rx, ry)
            finally:
                monkeypatch.setattr(ras, "_GAUSS2", _G2)
        return orig(p, grid, rx, ry)

    _G2 = ras._GAUSS2
    monkeypatch.setattr(ras, "local_operator", neumann)
    assert not _drch_is_imp_without_boundary(_p("tiny3"))
    assert not _drch_is_principal_submatrix(_p("tiny3", pml_cells=0))


def test_planted_one_sided_dirichlet_fails_the_pin(monkeypatch):
    """Dirichlet on the upper artificial sides only (the lower ones keep their
    nodes and impedance term), planted in the oracle."""
    orig = ras.local_operator

    def one_sided(p, grid, rx, ry):
        if p.get("local_bc", 0) == 1:
            A, nodes, glob, nlx, nly = orig(dict(p, local_bc=0), grid, rx, ry)
            i = nodes % (grid.Mx + 1)
            j = nodes // (grid.Mx + 1)
            drop = np.zeros(nodes.size, dtype=bool)
            if rx.hi_interior and rx.ext_hi < grid.Mx:
                drop |= i == rx.ext_hi
            if ry.hi_interior and ry.ext_hi < grid.My:
                drop |= j == ry.ext_hi
            keep = ~drop
            return (A.tocsr()[keep][:, keep], nodes[keep], glob[keep],
                    nlx - int(rx.hi_interior), nly - int(ry.hi_interior))
        return orig(p, grid, rx, ry)

    monkeypatch.setattr(ras, "local_operator", one_sided)
    assert not _drch_is_imp_without_boundary(_p("tiny3"))


def test_dirichlet_preconditioner_matches_dense_definition():
    """B^-1 = sum_j R_j^T diag(chi_j) inv(A_j) R_j with the Dirichlet local
    matrices, built densely from explicit R_j, against the SuperLU apply."""
    p = _p("tiny", local_bc=1)
    grid, subs = ras.build_subdomains(p)
    n = grid.n
    B = np.zeros((n, n), dtype=np.complex128)
    for s in subs:
        Rj = np.zeros((s.glob.size, n))
        Rj[np.arange(s.glob.size), s.glob] = 1.0
        B += Rj.T @ np.diag(s.chi) @ np.linalg.inv(s.A.toarray()) @ Rj
    rng = np.random.default_rng(1)
    r = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    z = ras.RAS(p).factor().apply(r)
    assert np.linalg.norm(z - B @ r) <= 1e-11 * np.linalg.norm(B @ r)
    # the closure matters: the impedance preconditioner differs by far more
    # than rounding (about 1% here; the local PML damps most of the difference)
    zi = ras.RAS(dict(p, local_bc=0)).factor().apply(r)
    assert np.linalg.norm(zi - z) > 1e-3 * np.linalg.norm(z)
