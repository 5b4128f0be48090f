"""Pins for the oracle's RAS-PML preconditioner and outer iterations
(paper Section 2, Section 3 (ii), Algorithm 1, Section 4.1)."""
import math

import numpy as np
import pytest

import workloads
from oracle import fem, krylov, ras


def _w(name="tiny3", **kw):
    return workloads.get(name).with_(**kw)


def test_box_edges_cover_cells():
    e = ras.box_edges(50, 4)
    assert list(e) == [0, 13, 26, 38, 50]          # first 50 mod 4 boxes one wider


@pytest.mark.parametrize("name", ["tiny", "tiny3", "small", "c0"])
def test_partition_of_unity(name):
    """Section 2: sum_j chi_j = 1, chi_j >= 0, supp chi_j in Omega_j,int,
    chi_j = 1 on the non-overlapped part of Omega_j."""
    p = _w(name).params()
    grid, subs = ras.build_subdomains(p)
    t = np.zeros(grid.n)
    for s in subs:
        np.add.at(t, s.glob, s.chi)
        assert np.all(s.chi >= 0.0)
        ii = s.nodes % (grid.Mx + 1)
        jj = s.nodes // (grid.Mx + 1)
        outside = ((ii <= s.rx.int_lo) & s.rx.lo_interior) | ((ii >= s.rx.int_hi) & s.rx.hi_interior) \
            | ((jj <= s.ry.int_lo) & s.ry.lo_interior) | ((jj >= s.ry.int_hi) & s.ry.hi_interior)
        assert np.all(s.chi[outside] == 0.0)
        o = p["ovlp_cells"]
        core = ((ii >= s.rx.box_lo + o) | ~np.array(s.rx.lo_interior)) \
            & ((ii <= s.rx.box_hi - o) | ~np.array(s.rx.hi_interior)) \
            & ((jj >= s.ry.box_lo + o) | ~np.array(s.ry.lo_interior)) \
            & ((jj <= s.ry.box_hi - o) | ~np.array(s.ry.hi_interior)) \
            & (ii >= s.rx.box_lo) & (ii <= s.rx.box_hi) & (jj >= s.ry.box_lo) & (jj <= s.ry.box_hi)
        assert np.all(s.chi[core] == 1.0)
    assert np.max(np.abs(t - 1.0)) < 1e-15


def test_local_pml_extension_only_on_interior_sides():
    """Section 2: kappa_j = 0 on sides on the outer boundary, kappa elsewhere."""
    p = _w("tiny3").params()
    grid = fem.make_grid(p)
    rs = ras.ranges_1d(grid.Mx, 3, p["ovlp_cells"], p["pml_cells"])
    o, k = p["ovlp_cells"], p["pml_cells"]
    assert (rs[0].ext_lo, rs[0].int_lo) == (0, 0)
    assert rs[0].ext_hi == rs[0].box_hi + o + k
    assert (rs[1].ext_lo, rs[1].ext_hi) == (rs[1].box_lo - o - k, rs[1].box_hi + o + k)
    assert (rs[2].ext_hi, rs[2].int_hi) == (grid.Mx, grid.Mx)


def test_local_stretching_restarts_beyond_interior_sides():
    """Section 2: g_j = g_i in (a_j, b_j), g(x - b_j) beyond b_j, -g(a_j - x) below a_j."""
    p = _w("tiny3").params()
    grid = fem.make_grid(p)
    r = ras.ranges_1d(grid.Mx, 3, p["ovlp_cells"], p["pml_cells"])[1]
    fn = ras.local_gamma_fn(grid, r, 0, p["g_amp"], p["g_ramp"])
    hh = grid.h / 2
    for ds in (1, 2, 3, 5):
        s = 2 * r.int_hi + ds
        assert fn(s) == 1 + 1j * fem.gprime(ds * hh, p["g_amp"], p["g_ramp"])
        s = 2 * r.int_lo - ds
        assert fn(s) == 1 + 1j * fem.gprime(ds * hh, p["g_amp"], p["g_ramp"])
    mid = np.arange(2 * r.int_lo + 1, 2 * r.int_hi)
    assert np.all(fn(mid) == fem.global_gamma_x(grid, mid, p["g_amp"], p["g_ramp"]))
    # first box: its low side is on the outer boundary, where the global PML stays
    r0 = ras.ranges_1d(grid.Mx, 3, p["ovlp_cells"], p["pml_cells"])[0]
    fn0 = ras.local_gamma_fn(grid, r0, 0, p["g_amp"], p["g_ramp"])
    assert fn0(1) == fem.global_gamma_x(grid, 1, p["g_amp"], p["g_ramp"])


def test_local_rows_equal_global_rows_inside_omega_j_int():
    """Section 2: the local form equals the global one where g_j = g_i, so rows of
    nodes whose six triangles lie inside Omega_j,int agree entry by entry."""
    p = _w("tiny3").params()
    grid, A = fem.assemble_global(p)
    grid, subs = ras.build_subdomains(p)
    s = subs[4]                                      # the middle subdomain
    Al = s.A.tocsr()
    checked = 0
    for l, node in enumerate(s.nodes):
        i, j = node % (grid.Mx + 1), node // (grid.Mx + 1)
        if not (s.rx.int_lo + 1 <= i <= s.rx.int_hi - 1 and s.ry.int_lo + 1 <= j <= s.ry.int_hi - 1):
            continue
        lr = Al.getrow(l).tocoo()
        gr = A.getrow(s.glob[l]).tocoo()
        loc = {int(s.glob[c]): v for c, v in zip(lr.col, lr.data)}
        glo = {int(c): v for c, v in zip(gr.col, gr.data)}
        assert loc == glo
        checked += 1
    assert checked > 100


def test_impedance_closed_form_row_sums():
    """Section 3 (ii): with the impedance closure on every side of an interior
    subdomain, 1^T A_j 1 = -k^2 int_{Omega_j} g1 g2 - i k int_{boundary} gamma_t ds,
    because the constant lies in the local space and has no gradient. The
    right-hand side is evaluated with the closed-form integral of g'. With the
    end of the g' ramp on a grid line, both quadratures are exact here (the two
    triangles of a cell combine into Simpson's rule along each axis)."""
    w = _w("tiny3", h=0.01, ovlp_cells=4, pml_cells=6)
    p = w.params()
    grid, subs = ras.build_subdomains(p)
    s = subs[4]
    k, amp, ramp = p["k"], p["g_amp"], p["g_ramp"]
    one = np.ones(s.A.shape[0])
    lhs = one @ (s.A @ one)

    def side_integral(r):
        # int over [ext_lo, ext_hi] of gamma_j: length + i * (g(beyond hi) + g(beyond lo))
        L = (r.ext_hi - r.ext_lo) * grid.h
        dh = (r.ext_hi - r.int_hi) * grid.h
        dl = (r.int_lo - r.ext_lo) * grid.h
        return L + 1j * (fem.g_integral(dh, amp, ramp) + fem.g_integral(dl, amp, ramp))
    Ix, Iy = side_integral(s.rx), side_integral(s.ry)
    rhs = -k * k * Ix * Iy - 1j * k * (2 * Ix + 2 * Iy)
    assert abs(lhs - rhs) < 1e-12 * abs(rhs)
    # the impedance term alone is about k*perimeter: a dropped or mis-signed term fails
    assert abs(1j * k * (2 * Ix + 2 * Iy)) > 1e-2 * abs(rhs)


def test_one_subdomain_gives_exact_inverse():
    """One subdomain: Omega_1 = Omega, chi = 1, A_1 = A, so B^-1 = A^-1 and
    GMRES stops after a single iteration."""
    w = _w("tiny", px=1, py=1)
    p = w.params()
    grid, A = fem.assemble_global(p)
    b = fem.assemble_rhs(p, w.centres, w.amps, w.width)
    R = ras.RAS(p).factor()
    z = R.apply(b)
    u = fem.dense_solve(A, b)
    assert np.linalg.norm(z - u) <= 1e-12 * np.linalg.norm(u)
    x, it, rel, _ = krylov.fgmres(A.dot, R.apply, b, rtol=1e-10, maxit=10)
    assert it == 1 and rel < 1e-10


def test_preconditioner_matches_dense_definition():
    """B^-1 built densely from its definition (explicit R_j, diag(chi_j), inv(A_j))."""
    w = _w("tiny")
    p = w.params()
    grid, subs = ras.build_subdomains(p)
    n = grid.n
    B = np.zeros((n, n), dtype=np.complex128)
    for s in subs:
        Rj = np.zeros((s.glob.size, n))
        Rj[np.arange(s.glob.size), s.glob] = 1.0
        B += Rj.T @ np.diag(s.chi) @ np.linalg.inv(s.A.toarray()) @ Rj
    rng = np.random.default_rng(0)
    r = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    z = ras.RAS(p).factor().apply(r)
    assert np.linalg.norm(z - B @ r) <= 1e-11 * np.linalg.norm(B @ r)


@pytest.mark.parametrize("name", ["tiny", "small"])
def test_gmres_agrees_with_direct_solve(name):
    w = _w(name)
    p = w.params()
    grid, A = fem.assemble_global(p)
    b = fem.assemble_rhs(p, w.centres, w.amps, w.width)
    R = ras.RAS(p).factor()
    x, it, rel, _ = krylov.fgmres(A.dot, R.apply, b, rtol=1e-12, maxit=300)
    u = fem.direct_solve(A, b)
    assert rel <= 1e-12
    assert np.linalg.norm(x - u) <= 1e-10 * np.linalg.norm(u)


def test_flexible_and_right_gmres_agree_at_fixed_m():
    w = _w("tiny3")
    p = w.params()
    grid, A = fem.assemble_global(p)
    b = fem.assemble_rhs(p, w.centres, w.amps, w.width)
    R = ras.RAS(p).factor()
    x1, i1, _, h1 = krylov.fgmres(A.dot, R.apply, b, rtol=0.0, maxit=8)
    x2, i2, _, h2 = krylov.gmres_right(A.dot, R.apply, b, rtol=0.0, maxit=8)
    assert i1 == i2 == 8
    assert np.linalg.norm(x1 - x2) <= 1e-12 * np.linalg.norm(x1)
    # the Arnoldi estimate is non-increasing and equals the true residual at the end
    e = np.array(h1[1:])
    assert np.all(np.diff(e) <= 1e-14)
    assert abs(np.linalg.norm(b - A @ x1) / np.linalg.norm(b) - e[-1]) < 1e-10


def test_restarted_gmres_converges():
    w = _w("tiny3")
    p = w.params()
    grid, A = fem.assemble_global(p)
    b = fem.assemble_rhs(p, w.centres, w.amps, w.width)
    R = ras.RAS(p).factor()
    x, it, rel, _ = krylov.fgmres(A.dot, R.apply, b, rtol=1e-8, maxit=200, restart=6)
    assert rel <= 1e-8
    assert np.linalg.norm(A @ x - b) <= 1e-8 * np.linalg.norm(b) * 1.0001


def test_richardson_algorithm_1_converges():
    """Algorithm 1 with the impedance closure converges on a small case and
    its residual is then confined to the overlaps (Section 3 (i))."""
    w = _w("tiny")
    p = w.params()
    grid, A = fem.assemble_global(p)
    b = fem.assemble_rhs(p, w.centres, w.amps, w.width)
    R = ras.RAS(p).factor()
    u, it, rel, hist = krylov.richardson(A.dot, R.apply, b, rtol=1e-8, maxit=200)
    assert rel <= 1e-8
    # Section 3 (i): after one RAS step from u = 0, the residual vanishes on
    # nodes whose whole stencil lies where a single chi_j = 1.
    u1 = R.apply(b)
    r1 = b - A @ u1
    grid_, subs = ras.build_subdomains(p)
    single = np.zeros(grid.n, dtype=bool)
    for s in subs:
        ii = s.nodes % (grid.Mx + 1)
        jj = s.nodes // (grid.Mx + 1)
        o = p["ovlp_cells"]
        away = (ii > s.rx.box_lo + o) | ~np.array(s.rx.lo_interior)
        away &= (ii < s.rx.box_hi - o) | ~np.array(s.rx.hi_interior)
        away &= (jj > s.ry.box_lo + o) | ~np.array(s.ry.lo_interior)
        away &= (jj < s.ry.box_hi - o) | ~np.array(s.ry.hi_interior)
        away &= (ii >= s.rx.box_lo) & (ii <= s.rx.box_hi) & (jj >= s.ry.box_lo) & (jj <= s.ry.box_hi)
        single[s.glob[away]] = True
    assert np.max(np.abs(r1[single])) < 1e-10 * np.max(np.abs(r1))
    assert np.max(np.abs(r1[~single])) > 1e-3 * np.max(np.abs(b))


@pytest.mark.slow
def test_iterations_grow_with_k_at_fixed_resolution():
    """Sections 2 and 4: with h ~ 1/k and a fixed number of cells per box, the
    GMRES iteration count grows with k (roughly linearly, Table 2, Table 3)."""
    its = []
    for k_over_pi, p_ in ((10, 2), (20, 4), (40, 8)):
        k = k_over_pi * math.pi
        h = 1.0 / (8 * k_over_pi)          # 16 points per wavelength
        w = workloads.get("small").with_(k=k, h=h, px=p_, py=p_,
                                         ovlp_cells=workloads.width_cells(k, h),
                                         pml_cells=workloads.width_cells(k, h))
        p = w.params()
        grid, A = fem.assemble_global(p)
        b = fem.assemble_rhs(p, w.centres, w.amps, w.width)
        R = ras.RAS(p).factor()
        _, it, rel, _ = krylov.fgmres(A.dot, R.apply, b, rtol=1e-6, maxit=400)
        assert rel <= 1e-6
        its.append(it)
    assert its[0] < its[1] < its[2]
    assert its[2] < 4 * 4 * its[0]                 # far below quadratic growth


def deep_core_mask(p):
    """Unknowns whose whole 7-point stencil lies where exactly one subdomain
    carries the partition of unity (chi_j = 1 away from every overlap strip)."""
    grid, rxs, rys = ras.covering(p)
    o = p["ovlp_cells"]
    ok_x = np.zeros(grid.Mx + 1, bool)
    ok_y = np.zeros(grid.My + 1, bool)
    for r, ok in ((rxs, ok_x), (rys, ok_y)):
        for q in r:
            lo = q.box_lo + o + 1 if q.lo_interior else 1
            hi = q.box_hi - o - 1 if q.hi_interior else len(ok) - 2
            ok[lo:hi + 1] = True
    ii = np.arange(1, grid.Mx)
    jj = np.arange(1, grid.My)
    return (ok_y[jj][:, None] & ok_x[ii][None, :]).ravel()


@pytest.mark.parametrize("name", ["small", "c0"])
def test_residual_after_one_sweep_lives_in_the_overlaps(name):
    """Section 3, practical point (i): after one RAS sweep from u = 0 the
    residual b - A B^-1 b vanishes wherever a single subdomain's local solve
    is exact for the global equations, i.e. away from the overlaps."""
    w = _w(name)
    p = w.params()
    grid, A = fem.assemble_global(p)
    R = ras.RAS(p).factor()
    rng = np.random.default_rng(3)
    b = rng.standard_normal(grid.n) + 1j * rng.standard_normal(grid.n)
    r = b - A @ R.apply(b)
    m = deep_core_mask(p)
    assert m.sum() > 0.3 * grid.n
    assert np.max(np.abs(r[m])) <= 1e-11 * np.max(np.abs(b))
    assert np.linalg.norm(r[~m]) >= 0.1 * np.linalg.norm(b)    # but not in the overlaps
