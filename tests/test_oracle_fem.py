"""Pins for the oracle's discretisation (paper Section 1) against closed forms,
textbook P1 element matrices, brute force and the free-space Green's function."""
import math

import numpy as np
import pytest
from scipy.integrate import quad

import workloads
from oracle import fem

GOLDEN = __file__.replace("test_oracle_fem.py", "golden/p1_stencils.txt")


def _params(**kw):
    w = workloads.get("tiny").with_(**kw)
    return w.params()


def _stencil(A, grid, i, j):
    """Row of node (i, j) as {(di, dj): value}."""
    r = (j - 1) * grid.nx + (i - 1)
    row = A.getrow(r).tocoo()
    out = {}
    for c, v in zip(row.col, row.data):
        out[(c % grid.nx - (i - 1), c // grid.nx - (j - 1))] = v
    return out


def _load_golden():
    st = {}
    name = None
    for line in open(GOLDEN):
        line = line.split("#", 1)[0].strip()
        if not line:
            continue
        if line.startswith("["):
            name = line.strip("[]")
            st[name] = {}
            continue
        di, dj, v = line.split()
        st[name][(int(di), int(dj))] = float(v)
    return st


def test_gprime_meets_paper_conditions():
    # Section 1: g = g' = 0 for x <= 0, g' > 0 for x > 0, g'' = 0 beyond kappa_inf.
    amp, ramp = 20.0, 0.05
    assert np.all(fem.gprime([-1.0, -1e-9, 0.0], amp, ramp) == 0.0)
    d = np.linspace(1e-6, 0.3, 1001)
    assert np.all(fem.gprime(d, amp, ramp) > 0.0)
    beyond = np.linspace(ramp, 0.3, 50)
    assert np.allclose(fem.gprime(beyond, amp, ramp), amp)
    # C^1 at the end of the ramp: one-sided slopes both vanish there
    e = 1e-6
    slope_in = (fem.gprime(ramp, amp, ramp) - fem.gprime(ramp - e, amp, ramp)) / e
    assert abs(slope_in) < 1e-3 * amp / ramp
    # closed-form g equals the numerical integral of g' (independent quadrature)
    for x in (0.01, 0.03, 0.05, 0.08, 0.1):
        val, _ = quad(lambda t: float(fem.gprime(t, amp, ramp)), 0.0, x, points=[ramp])
        assert abs(float(fem.g_integral(x, amp, ramp)) - val) < 1e-12


def test_laplacian_and_mass_stencils_match_p1_closed_forms():
    gold = _load_golden()
    h = 1.0 / 40
    p0 = _params(k=0.0, g_amp=0.0)
    grid, A0 = fem.assemble_global(p0)
    st = _stencil(A0, grid, 20, 20)
    for key in set(st) | set(gold["laplace"]):
        assert abs(st.get(key, 0.0) - gold["laplace"].get(key, 0.0)) < 1e-14, key
    k = 7.0
    _, Ak = fem.assemble_global(_params(k=k, g_amp=0.0))
    M = (Ak - A0) / (-k * k)
    st = _stencil(M, grid, 20, 20)
    for key in set(st) | set(gold["mass"]):
        assert abs(st.get(key, 0.0) - gold["mass"].get(key, 0.0) * h * h / 12) < 1e-16, key


def test_constant_stretch_closed_form():
    """gamma_1 = c1, gamma_2 = c2 constant: A = (c2/c1) Dxx + (c1/c2) Dyy - k^2 c1 c2 M."""
    c1, c2, k = 1.0 + 0.7j, 1.3 - 0.2j, 5.0
    p = _params(k=k)
    grid, A = fem.assemble_global(p, gx_fn=lambda s: c1 + 0 * s, gy_fn=lambda s: c2 + 0 * s)
    h = grid.h
    st = _stencil(A, grid, 10, 13)
    m = h * h / 12
    expect = {(0, 0): 2 * c2 / c1 + 2 * c1 / c2 - k * k * c1 * c2 * 6 * m,
              (1, 0): -c2 / c1 - k * k * c1 * c2 * m, (-1, 0): -c2 / c1 - k * k * c1 * c2 * m,
              (0, 1): -c1 / c2 - k * k * c1 * c2 * m, (0, -1): -c1 / c2 - k * k * c1 * c2 * m,
              (1, 1): -k * k * c1 * c2 * m, (-1, -1): -k * k * c1 * c2 * m}
    for key in set(st) | set(expect):
        assert abs(st.get(key, 0.0) - expect.get(key, 0.0)) < 1e-13, key


def test_matrix_is_complex_symmetric_not_hermitian():
    grid, A = fem.assemble_global(_params())
    assert abs(A - A.T).max() == 0.0
    assert abs(A - A.conj().T).max() > 1.0          # PML and -k^2 make it non-Hermitian
    assert A.nnz <= 7 * grid.n


def test_pml_coefficients_only_outside_omega_int():
    # Inside Omega_int gamma = 1: rows there equal the unstretched rows.
    p = _params()
    grid, A = fem.assemble_global(p)
    _, A0 = fem.assemble_global(dict(p, g_amp=0.0))
    i_in = int(round((0.5 - grid.X0) / grid.h))
    assert _stencil(A, grid, i_in, i_in) == _stencil(A0, grid, i_in, i_in)
    st = _stencil(A, grid, 2, 2)                    # deep in the corner PML
    st0 = _stencil(A0, grid, 2, 2)
    assert abs(st[(0, 0)] - st0[(0, 0)]) > 1.0


def test_load_vector_integrates_gaussian():
    p = _params()
    w = 0.05
    grid = fem.make_grid(p)
    b = fem.assemble_rhs(p, [[0.5, 0.5]], [1.0], w)
    # sum_i F_i = int f (hats sum to one away from the outer boundary)
    assert abs(b.sum() - math.pi * w * w) < 2e-3 * math.pi * w * w
    # centre on the edge x = x0 of Omega_int: the cut keeps half the mass
    b2 = fem.assemble_rhs(p, [[0.0, 0.5]], [1.0], w)
    assert abs(b2.sum() - 0.5 * math.pi * w * w) < 0.05 * math.pi * w * w
    x, y = fem.unknown_coords(grid)
    assert np.all(b2[x < grid.x0 - 0.5 * grid.h] == 0.0)


def test_direct_solve_matches_dense_brute_force():
    w = workloads.get("tiny")
    p = w.with_(h=1.0 / 20).params()
    grid, A = fem.assemble_global(p)
    b = fem.assemble_rhs(p, w.centres, w.amps, 0.1)
    u1 = fem.direct_solve(A, b)
    u2 = fem.dense_solve(A, b)
    assert np.linalg.norm(u1 - u2) <= 1e-12 * np.linalg.norm(u2)
    assert np.linalg.norm(A @ u1 - b) <= 1e-12 * np.linalg.norm(b)


@pytest.mark.slow
def test_point_source_converges_to_hankel_with_pml():
    """u_h -> (i/4) H_0^(1)(k r) away from source and PML, at about O(h^2);
    without the PML (g = 0, Dirichlet box) it does not converge."""
    def err(N, amp):
        p = _params(k=4 * math.pi, h=1.0 / N, g_amp=amp)
        grid, A = fem.assemble_global(p)
        i = int(round((0.5 - grid.X0) / grid.h))
        u = fem.direct_solve(A, fem.point_source_rhs(grid, i, i))
        x, y = fem.unknown_coords(grid)
        r = np.hypot(x - 0.5, y - 0.5)
        m = (r > 0.15) & (r < 0.4)
        ue = fem.hankel_solution(x[m], y[m], 0.5, 0.5, p["k"])
        return np.linalg.norm(u[m] - ue) / np.linalg.norm(ue)
    e40, e80 = err(40, 20.0), err(80, 20.0)
    assert e80 < 0.05
    assert e40 / e80 > 3.0
    assert err(80, 0.0) > 0.5


def test_cubic_profile_of_the_papers_experiments():
    """Section 4: g(x) = 10 k x^3, so g'(d) = 30 k d^2 (profile 1), zero for d <= 0;
    its numerical integral is g."""
    k = 300.0
    amp = 10.0 * k
    d = np.array([-0.01, 0.0, 0.001, 0.01, 0.05])
    gp = fem.gprime(d, amp, 1.0, profile=1)
    assert np.all(gp[:2] == 0.0)
    assert np.allclose(gp[2:], 3.0 * amp * d[2:] ** 2, rtol=1e-15)
    for x in (0.003, 0.02, 0.06):
        val, _ = quad(lambda t: float(fem.gprime(t, amp, 1.0, profile=1)), 0.0, x)
        assert abs(val - amp * x ** 3) < 1e-12 * max(1.0, amp * x ** 3)


def test_paper_setup_geometry():
    """Section 4: Omega = (0,1)^2 with a three-wavelength PML, h = 1/(2k), the
    smoothed-delta source of unit mass, widths from the law of Section 3 (iii)."""
    w = workloads.paper_setup(300, 75, C_delta=1 / 6, C_kappa=3 / 8)
    p = w.params()
    grid = fem.make_grid(p)
    assert grid.Mx == grid.My == 600 and abs(grid.X0) < 1e-15
    assert abs(p["kappa_g"] - 3 * 2 * math.pi / 300) <= 0.5 * grid.h
    # l(300) = 2: delta = lambda/3 -> 4 cells, kappa = 0.75 lambda -> 9 cells
    assert (p["ovlp_cells"], p["pml_cells"]) == (4, 9)
    b = fem.assemble_rhs(p, w.centres, w.amps, w.width)
    assert abs(b.sum().real - 1.0) < 1e-3                    # unit mass (16k^2/pi^3 * pi w^2 = 1)
