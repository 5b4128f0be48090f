"""Pins for the oracle's second bilinear form: the paper's eq. weak as printed
(Section 1), int (D grad u).grad v - (beta.grad u) v - k^2 u v with
D_ii = gamma_i^-2 and beta_i = gamma_i'/gamma_i^3, which is not symmetric.

What fixes it independently of its own code: the PML operator it discretises
(consistency with a smooth function at O(h^2)), the closed form for constant
stretching (a scaled copy of the symmetric form), the symmetric form's rows
where gamma = 1, the symmetric form's solution up to discretisation error,
and the impedance closure's integral of a constant."""

import numpy as np
import pytest

import workloads
from oracle import fem, krylov, ras


def _w(name="tiny3", **kw):
    return workloads.get(name).with_(form=1, **kw)


def _p(**kw):
    p = dict(k=5.0, x0=0.0, y0=0.0, x1=1.0, y1=1.0, kappa_g=0.25, h=1 / 40, px=1, py=1, ovlp_cells=2,
             pml_cells=2, g_amp=20.0, g_ramp=0.05, local_bc=0, g_profile=0, form=1)
    p.update(kw)
    return p


@pytest.mark.parametrize("profile,amp,ramp", [(0, 20.0, 0.05), (1, 50.0, 0.05)])
def test_gsecond_is_the_derivative_of_gprime(profile, amp, ramp):
    d = np.linspace(-0.02, 0.12, 57) + 1e-4
    e = 1e-6
    fd = (fem.gprime(d + e, amp, ramp, profile) - fem.gprime(d - e, amp, ramp, profile)) / (2 * e)
    assert np.allclose(fem.gsecond(d, amp, ramp, profile), fd, rtol=1e-6, atol=1e-4 * amp / ramp)
    assert np.all(fem.gsecond(np.array([-1.0, 0.0]), amp, ramp, profile) == 0.0)


def test_dgamma_sign_on_both_sides_of_omega_int():
    """g_i(x) = g(x - b) beyond b and -g(a - x) below a (Section 1): gamma_i'
    = i g''(x - b) above, -i g''(a - x) below, 0 inside."""
    grid = fem.make_grid(_p(h=1 / 100))
    amp, ramp = 20.0, 0.05
    for s, want in ((2 * 10, -1j * fem.gsecond(0.15, amp, ramp)), (2 * 140, 1j * fem.gsecond(0.15, amp, ramp)),
                    (2 * 50, 0.0)):
        got = fem.global_dgamma_x(grid, float(s), amp, ramp)
        assert abs(got - want) < 1e-12 * max(1.0, abs(want))
    # below Omega_int the stretch decreases away from the box: a finite
    # difference of gamma_1 along x agrees with gamma_1'
    s = 2.0 * 22
    fd = (fem.global_gamma_x(grid, s + 0.01, amp, ramp) - fem.global_gamma_x(grid, s - 0.01, amp, ramp)) / (0.01 * grid.h)
    assert abs(fd - fem.global_dgamma_x(grid, s, amp, ramp)) < 1e-3 * abs(fd)


def test_constant_stretch_is_the_symmetric_form_divided_by_gamma1_gamma2():
    """With constant gamma_1 = a, gamma_2 = b (so beta = 0) eq. weak is the
    symmetric form divided by ab, element by element: (b/a)/(ab) = a^-2 on
    u_x v_x, (a/b)/(ab) = b^-2 on u_y v_y, k^2 ab/(ab) = k^2 on u v. A
    swapped D11/D22 fails it (a != b)."""
    a, b = 1 + 0.7j, 1 - 0.4j
    p = _p(h=1 / 8)
    c = lambda v: (lambda s: np.full(np.shape(s), v))  # noqa: E731
    _, A0 = fem.assemble_global(dict(p, form=0), gx_fn=c(a), gy_fn=c(b))
    _, A1 = fem.assemble_global(p, gx_fn=c(a), gy_fn=c(b), dgx_fn=c(0j), dgy_fn=c(0j))
    assert abs(A1 - A0 / (a * b)).max() < 1e-14 * abs(A1).max()


def _consistency(h, form, sign=1.0):
    """max over nodes >= 2.5 cells from the outer boundary of
    |(A I_h u)_i / h^2 - w(x_i) (L u)(x_i)|, L u = -sum_i gamma_i^-1 d_i(gamma_i^-1 d_i u) - k^2 u,
    w = 1 (form 1) or gamma_1 gamma_2 (form 0), for smooth u and smooth
    analytic stretching; sign = -1 plants a flipped gamma' in the oracle."""
    p = _p(h=h, form=form)
    grid = fem.make_grid(p)
    c1, c2 = 0.6, 0.4
    gxf = lambda s: 1 + 1j * c1 * (1 + np.sin(2 * grid.xs(s)))  # noqa: E731
    dgxf = lambda s: sign * 2j * c1 * np.cos(2 * grid.xs(s))  # noqa: E731
    gyf = lambda s: 1 + 1j * c2 * (1 + np.cos(3 * grid.ys(s)))  # noqa: E731
    dgyf = lambda s: -sign * 3j * c2 * np.sin(3 * grid.ys(s))  # noqa: E731
    _, A = fem.assemble_global(p, gxf, gyf, dgxf, dgyf)
    x, y = fem.unknown_coords(grid)
    a, b = 3.0, 2.0
    u = np.sin(a * x) * np.cos(b * y)
    ux, uxx = a * np.cos(a * x) * np.cos(b * y), -a * a * u
    uy, uyy = -b * np.sin(a * x) * np.sin(b * y), -b * b * u
    g1, dg1 = 1 + 1j * c1 * (1 + np.sin(2 * x)), 2j * c1 * np.cos(2 * x)
    g2, dg2 = 1 + 1j * c2 * (1 + np.cos(3 * y)), -3j * c2 * np.sin(3 * y)
    Lu = -(uxx / g1 ** 2 - dg1 / g1 ** 3 * ux) - (uyy / g2 ** 2 - dg2 / g2 ** 3 * uy) - p["k"] ** 2 * u
    wgt = 1.0 if form == 1 else g1 * g2
    X1, Y1 = grid.X0 + grid.Mx * h, grid.Y0 + grid.My * h
    m = (x > grid.X0 + 2.5 * h) & (x < X1 - 2.5 * h) & (y > grid.Y0 + 2.5 * h) & (y < Y1 - 2.5 * h)
    err = np.abs((A @ u) / h ** 2 - wgt * Lu)[m].max()
    beta = np.abs(dg1 / g1 ** 3 * ux + dg2 / g2 ** 3 * uy)[m].max()
    return err, beta


@pytest.mark.parametrize("form", [0, 1])
def test_both_forms_are_consistent_with_the_pml_operator_at_second_order(form):
    """Section 1: eq. weak comes from -Delta_pml u - k^2 u = f by parts, so
    a(I_h u, phi_i) = h^2 (w L u)(x_i) + O(h^4) on this uniform mesh. The
    error falls by ~4 per halving; the beta term is ~70x the error at
    h = 1/40, so dropping it or flipping its sign cannot pass."""
    e1, beta = _consistency(1 / 20, form)
    e2, _ = _consistency(1 / 40, form)
    assert e1 / e2 > 3.5
    assert e2 < 0.05 * beta


def test_flipped_gamma_prime_is_caught():
    """The same check with gamma' negated (a planted mistake) does not converge."""
    e1, beta = _consistency(1 / 20, 1, sign=-1.0)
    e2, _ = _consistency(1 / 40, 1, sign=-1.0)
    assert e2 > 0.5 * beta and e1 / e2 < 1.5


def test_weak_form_is_not_symmetric_but_equals_the_symmetric_form_where_gamma_is_one():
    p = _w("tiny").params()
    grid, A1 = fem.assemble_global(p)
    _, A0 = fem.assemble_global(dict(p, form=0))
    assert abs(A1 - A1.T).max() > 1e-3 * abs(A1).max()
    # rows of nodes whose six triangles lie in Omega_int (gamma = 1 at every midpoint)
    x, y = fem.unknown_coords(grid)
    h = grid.h
    inner = (x >= p["x0"] + h - 1e-12) & (x <= p["x1"] - h + 1e-12) & (y >= p["y0"] + h - 1e-12) & \
        (y <= p["y1"] - h + 1e-12)
    idx = np.flatnonzero(inner)
    assert idx.size > 100
    assert abs(A1[idx] - A0[idx]).max() < 1e-13 * abs(A0).max()
    # no stretching at all: the two forms are the same matrix
    _, B1 = fem.assemble_global(dict(p, g_amp=0.0))
    _, B0 = fem.assemble_global(dict(p, g_amp=0.0, form=0))
    assert abs(B1 - B0).max() < 1e-14 * abs(B0).max()


def test_weak_and_symmetric_solutions_agree_to_discretisation_error():
    """Both forms discretise the same PML problem (form 1 is form 0 tested
    with v/(gamma_1 gamma_2)), so their solutions in Omega_int differ by a
    discretisation error that falls at second order (0.43% at h = 1/40, 0.11%
    at 1/80 with the cubic profile g = 30 d^3)."""
    rng = np.random.default_rng(5)
    centres = rng.uniform(0.2, 0.8, size=(2, 2))
    diffs = []
    for h in (1 / 40, 1 / 80):
        p = _p(k=8.0, h=h, kappa_g=0.25, g_amp=30.0, g_profile=1)
        grid, A1 = fem.assemble_global(p)
        _, A0 = fem.assemble_global(dict(p, form=0))
        b = fem.assemble_rhs(p, centres, np.ones(2), 0.1)
        u1, u0 = fem.direct_solve(A1, b), fem.direct_solve(A0, b)
        x, y = fem.unknown_coords(grid)
        m = (x > 0) & (x < 1) & (y > 0) & (y < 1)
        diffs.append(np.linalg.norm((u1 - u0)[m]) / np.linalg.norm(u0[m]))
    assert diffs[0] < 0.01 and diffs[0] / diffs[1] > 3.5


def test_weak_impedance_closed_form_row_sums():
    """Section 3 (ii) for form 1: the constant lies in the local space of an
    interior subdomain and has no gradient, so 1^T A_j 1 = -k^2 |Omega_j|
    - i k sum_sides |side| / gamma_n(side): gamma_n, the stretch normal to
    the side, is constant along it. Both quadratures are exact here."""
    w = _w("tiny3", h=0.01, ovlp_cells=4, pml_cells=6)
    p = w.params()
    grid, subs = ras.build_subdomains(p)
    s = subs[4]
    k = p["k"]
    one = np.ones(s.A.shape[0])
    lhs = one @ (s.A @ one)
    Lx = (s.rx.ext_hi - s.rx.ext_lo) * grid.h
    Ly = (s.ry.ext_hi - s.ry.ext_lo) * grid.h
    gn = 1 + 1j * fem.gprime(p["pml_cells"] * grid.h, p["g_amp"], p["g_ramp"])   # every side: p cells beyond
    rhs = -k * k * Lx * Ly - 1j * k * (2 * Lx + 2 * Ly) / gn
    assert abs(lhs - rhs) < 1e-12 * abs(rhs)
    assert abs(k * (2 * Lx + 2 * Ly) / gn) > 1e-2 * abs(rhs)
    # the symmetric form's weight (gamma_t, varying along the side) gives another value
    assert abs(gn - 1) > 0.05


def test_weak_local_rows_equal_global_rows_inside_omega_j_int():
    p = _w("tiny3").params()
    grid, A = fem.assemble_global(p)
    grid, subs = ras.build_subdomains(p)
    s = subs[4]
    Al = s.A.tocsr()
    checked = 0
    for l, node in enumerate(s.nodes):
        i, j = node % (grid.Mx + 1), node // (grid.Mx + 1)
        if not (s.rx.int_lo + 1 <= i <= s.rx.int_hi - 1 and s.ry.int_lo + 1 <= j <= s.ry.int_hi - 1):
            continue
        lr = Al.getrow(l).tocoo()
        gr = A.getrow(s.glob[l]).tocoo()
        assert {int(s.glob[c]): v for c, v in zip(lr.col, lr.data)} == {int(c): v for c, v in zip(gr.col, gr.data)}
        checked += 1
    assert checked > 100


def test_weak_one_subdomain_and_gmres():
    """One subdomain: B^-1 = A^-1 and GMRES takes one step; with the covering
    of tiny, FGMRES with RAS-PML reaches the direct solve of the
    non-symmetric system."""
    w = _w("tiny", px=1, py=1)
    p = w.params()
    grid, A = fem.assemble_global(p)
    b = fem.assemble_rhs(p, w.centres, w.amps, w.width)
    R = ras.RAS(p).factor()
    u = fem.dense_solve(A, b)
    assert np.linalg.norm(R.apply(b) - u) <= 1e-12 * np.linalg.norm(u)
    x, it, rel, _ = krylov.fgmres(A.dot, R.apply, b, rtol=1e-10, maxit=10)
    assert it == 1 and rel < 1e-10
    w = _w("tiny")
    p = w.params()
    grid, A = fem.assemble_global(p)
    b = fem.assemble_rhs(p, w.centres, w.amps, w.width)
    x, it, rel, _ = krylov.fgmres(A.dot, ras.RAS(p).factor().apply, b, rtol=1e-12, maxit=300)
    u = fem.direct_solve(A, b)
    assert rel <= 1e-12 and np.linalg.norm(x - u) <= 1e-10 * np.linalg.norm(u)


def _local_solution_gap(h, planted=False):
    """Relative difference on Omega_j,int of the local solutions of the two
    forms for the middle subdomain of a 3 x 3 covering (widths fixed in length
    as h halves), one Gaussian source inside Omega_int. planted = True swaps
    form 1's impedance weight 1/gamma_n for form 0's gamma_t (a mistake planted
    in the oracle)."""
    import scipy.sparse.linalg as spla
    p = _p(k=10.0, h=h, kappa_g=0.1, px=3, py=3, ovlp_cells=round(0.05 / h), pml_cells=round(0.1 / h),
           g_amp=30.0, g_profile=1)
    sols = {}
    for form in (0, 1):
        q = dict(p, form=form)
        grid, rxs, rys = ras.covering(q)
        rx, ry = rxs[1], rys[1]
        A, nodes, _, _, _ = ras.local_operator(q, grid, rx, ry)
        if planted and form == 1:
            A0, _, _, _, _ = ras.local_operator(dict(q, form=0), grid, rx, ry)
            A = A - _impedance_part(q, grid, rx, ry, nodes, A) + _impedance_part(dict(q, form=0), grid, rx, ry,
                                                                                 nodes, A0)
        xs, ys = grid.xs(2 * (nodes % (grid.Mx + 1))), grid.ys(2 * (nodes // (grid.Mx + 1)))
        f = np.exp(-((xs - 0.5) ** 2 + (ys - 0.5) ** 2) / 0.05 ** 2) * h * h
        ii, jj = nodes % (grid.Mx + 1), nodes // (grid.Mx + 1)
        m = (ii >= rx.int_lo) & (ii <= rx.int_hi) & (jj >= ry.int_lo) & (jj <= ry.int_hi)
        sols[form] = (spla.splu(A.tocsc()).solve(f.astype(complex)), m)
    (u0, m), (u1, _) = sols[0], sols[1]
    return np.linalg.norm((u1 - u0)[m]) / np.linalg.norm(u0[m])


def _impedance_part(p, grid, rx, ry, nodes, A):
    """A_j minus its element terms: the impedance closure alone."""
    amp, ramp, prof = p["g_amp"], p["g_ramp"], p["g_profile"]
    gx, gy = ras.local_gamma_fn(grid, rx, 0, amp, ramp, prof), ras.local_gamma_fn(grid, ry, 1, amp, ramp, prof)
    cj, ci = np.meshgrid(np.arange(ry.ext_lo, ry.ext_hi), np.arange(rx.ext_lo, rx.ext_hi), indexing="ij")
    if p["form"] == 1:
        dgx, dgy = ras.local_dgamma_fn(grid, rx, 0, amp, ramp, prof), ras.local_dgamma_fn(grid, ry, 1, amp, ramp, prof)
        r, c, v = fem.assemble_cells_weak(grid, ci, cj, gx, gy, dgx, dgy, p["k"])
    else:
        r, c, v = fem.assemble_cells(grid, ci, cj, gx, gy, p["k"])
    num = -np.ones((grid.Mx + 1) * (grid.My + 1), dtype=np.int64)
    num[nodes] = np.arange(nodes.size)
    return A - fem._to_matrix(r, c, v, num, nodes.size)


def test_both_forms_pose_the_same_local_problem():
    """Section 3 (ii) read in the stretched normal coordinate: form 1's closure
    -i k int gamma_n^-1 u v ds is form 0's -i k int gamma_t u v ds tested with
    v/(gamma_1 gamma_2), so the two local solutions converge to each other
    (0.40% -> 0.10% from h = 1/40 to 1/80, with a weak local PML g = 30 d^3
    whose boundary condition matters). With form 0's weight planted in form 1
    the local problems differ and the gap stays at ~25%."""
    d1, d2 = _local_solution_gap(1 / 40), _local_solution_gap(1 / 80)
    assert d1 < 0.01 and d1 / d2 > 3.5
    p1, p2 = _local_solution_gap(1 / 40, planted=True), _local_solution_gap(1 / 80, planted=True)
    assert p2 > 0.1 and p1 / p2 < 1.2


def test_tables_1_2_ordering_in_the_papers_own_form():
    """Section 4, Tables 1-2, on the paper's set-up (g = 10 k x^3, a
    three-wavelength global PML, h = 1/(2k), the smoothed delta) in eq. weak as
    printed: RAS-PML-Imp needs no more iterations than RAS-PML-Drch, and both
    fewer than RAS-Imp (k = 160, 5 x 5 boxes of 64 cells: 28, 29, 44)."""
    its = {}
    for name, kw in (("imp", dict(local_bc=0)), ("drch", dict(local_bc=1)),
                     ("ras_imp", dict(local_bc=0, pml=False))):
        w = workloads.paper_setup(160, 64, C_delta=1 / 6, C_kappa=3 / 8, **kw).with_(form=1)
        p = w.params()
        grid, A = fem.assemble_global(p)
        b = fem.assemble_rhs(p, w.centres, w.amps, w.width)
        x, its[name], rel, _ = krylov.fgmres(A.dot, ras.RAS(p).factor().apply, b, rtol=1e-10, maxit=300)
        assert rel <= 1e-10
    assert its["imp"] <= its["drch"] < its["ras_imp"], its


@pytest.mark.parametrize("profile,amp", [(0, 20.0), (1, 30.0)])
def test_local_dgamma_is_the_derivative_of_the_local_stretch(profile, amp):
    """Section 2's local stretching restarts beyond an interior side of
    Omega_j,int (g(x - b_j) above, -g(a_j - x) below): a central difference of
    gamma_j along each axis matches gamma_j', below, inside and above."""
    p = _w("tiny3", g_profile=profile, g_amp=amp).params()
    grid, rxs, rys = ras.covering(p)
    rx, ry = rxs[1], rys[1]
    hh, e = 0.5 * grid.h, 1e-4
    for axis, r in ((0, rx), (1, ry)):
        gam = ras.local_gamma_fn(grid, r, axis, p["g_amp"], p["g_ramp"], profile)
        dgam = ras.local_dgamma_fn(grid, r, axis, p["g_amp"], p["g_ramp"], profile)
        pts = [2 * r.int_lo - 1.3, 2 * r.int_lo - 0.4, r.int_lo + r.int_hi + 0.5, 2 * r.int_hi + 0.4,
               2 * r.int_hi + 1.3]
        checked = 0
        for s in pts:
            fd = (gam(s + e) - gam(s - e)) / (2 * e * hh)
            d = dgam(s)
            assert abs(fd - d) <= 1e-5 * max(1.0, abs(d)), (axis, s, fd, d)
            checked += abs(d) > 0
        assert checked >= 4     # the points beyond both sides carry a nonzero derivative
