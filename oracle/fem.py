"""Oracle, part 1: PML-truncated Helmholtz problem on P1 triangles (paper Section 1).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Continuous problem (Section 1, eq. helmholtz0 with c = 1): -Delta u - k^2 u = f,
truncated to Omega = Omega_int widened by kappa_g on every side, with the
Cartesian PML of Section 1: gamma_i = 1 + i g_i'(x^i), where g_i is the
stretching g shifted to the side of Omega_int that x^i lies beyond and zero
inside Omega_int, and u = 0 on the outer boundary (u in H^1_0(Omega)).

The default weak form (form 0) is the paper's eq. (weak) multiplied through by
gamma_1 gamma_2, which turns it into a complex-symmetric bilinear form with the
same solution (gamma = 1 in Omega_int, where f lives):

    a(u, v) = int (gamma_2/gamma_1) u_x v_x + (gamma_1/gamma_2) u_y v_y
              - k^2 gamma_1 gamma_2 u v,          F(v) = int f v.

Form 1 is eq. (weak) as printed, int (D grad u).grad v - (beta.grad u) v
- k^2 u v with D_ii = gamma_i^-2 and beta_i = gamma_i'/gamma_i^3 (not
symmetric); at the continuous level it is form 0 tested with v/(gamma_1
gamma_2), so both discretise the same problem.

Discretisation: uniform cells of size h, each split along its
(i,j)-(i+1,j+1) diagonal into two right triangles; P1 elements; every element
integral by the three-point edge-midpoint rule (exact for quadratics). Unknowns
are the nodes not on the outer boundary, numbered x-fastest.

Coordinates are handled in half-cell index units s (x = X0 + s*h/2), so that a
quadrature point's position relative to a grid line is an exact integer test.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


# ----------------------------------------------------------------------------
# Stretching function (Section 1: conditions on g; profile fixed by workload)
# ----------------------------------------------------------------------------

def gprime(d, amp: float, ramp: float, profile: int = 0):
    """Derivative of the stretching function g at distance d beyond the box.

    profile 0: g'(d) = amp*(3t^2 - 2t^3), t = min(d/ramp, 1) for d > 0. It
    satisfies the paper's conditions on g (Section 1): g = g' = 0 for d <= 0,
    g' > 0 for d > 0, g'' = 0 beyond kappa_inf = ramp.
    profile 1: g(d) = amp*d^3, so g'(d) = 3 amp d^2 (the function of the
    paper's experiments, Section 4, with amp = 10k).
    Both are 0 for d <= 0.
    """
    d = np.asarray(d, dtype=np.float64)
    if profile == 1:
        return np.where(d > 0.0, 3.0 * amp * d * d, 0.0)
    t = np.clip(d / ramp, 0.0, 1.0)
    return np.where(d > 0.0, amp * (3.0 * t * t - 2.0 * t ** 3), 0.0)


def gsecond(d, amp: float, ramp: float, profile: int = 0):
    """Second derivative g''(d) of the same stretching (enters beta of eq. weak).

    profile 0: amp*6t(1-t)/ramp for 0 < d < ramp, 0 beyond; profile 1: 6 amp d.
    Both are 0 for d <= 0 and continuous.
    """
    d = np.asarray(d, dtype=np.float64)
    if profile == 1:
        return np.where(d > 0.0, 6.0 * amp * d, 0.0)
    t = np.clip(d / ramp, 0.0, 1.0)
    return np.where(d > 0.0, amp * 6.0 * t * (1.0 - t) / ramp, 0.0)


def g_integral(d, amp: float, ramp: float):
    """g(d) = int_0^d g' (closed form; used only by tests as an independent value)."""
    d = np.asarray(d, dtype=np.float64)
    t = np.clip(d / ramp, 0.0, 1.0)
    inside = amp * ramp * (t ** 3 - 0.5 * t ** 4)
    beyond = amp * ramp * 0.5 + amp * np.maximum(d - ramp, 0.0)
    return np.where(d <= 0.0, 0.0, np.where(d <= ramp, inside, beyond))


# ----------------------------------------------------------------------------
# Grid
# ----------------------------------------------------------------------------

@dataclass
class Grid:
    """Uniform grid on Omega = [X0, X0 + Mx h] x [Y0, Y0 + My h]."""
    X0: float
    Y0: float
    h: float
    Mx: int
    My: int
    x0: float  # Omega_int
    x1: float
    y0: float
    y1: float

    @property
    def nx(self) -> int:  # unknowns per grid row
        return self.Mx - 1

    @property
    def ny(self) -> int:
        return self.My - 1

    @property
    def n(self) -> int:
        return self.nx * self.ny

    def xs(self, s):
        """x coordinate of half-index s."""
        return self.X0 + np.asarray(s, dtype=np.float64) * (0.5 * self.h)

    def ys(self, s):
        return self.Y0 + np.asarray(s, dtype=np.float64) * (0.5 * self.h)


def make_grid(p: dict) -> Grid:
    """Grid of Omega = Omega_int widened by kappa_g (Section 1)."""
    X0 = p["x0"] - p["kappa_g"]
    Y0 = p["y0"] - p["kappa_g"]
    lx = p["x1"] - p["x0"] + 2 * p["kappa_g"]
    ly = p["y1"] - p["y0"] + 2 * p["kappa_g"]
    Mx = int(round(lx / p["h"]))
    My = int(round(ly / p["h"]))
    if abs(Mx * p["h"] - lx) > 1e-9 * lx or abs(My * p["h"] - ly) > 1e-9 * ly:
        raise ValueError("Omega is not a whole number of cells")
    return Grid(X0, Y0, p["h"], Mx, My, p["x0"], p["x1"], p["y0"], p["y1"])


def global_gamma_x(grid: Grid, s, amp, ramp, profile: int = 0):
    """gamma_1 = 1 + i g_1'(x): g_1' = g'(distance of x beyond Omega_int in x)."""
    x = grid.xs(s)
    d = np.maximum(np.maximum(grid.x0 - x, x - grid.x1), 0.0)
    return 1.0 + 1j * gprime(d, amp, ramp, profile)


def global_gamma_y(grid: Grid, s, amp, ramp, profile: int = 0):
    y = grid.ys(s)
    d = np.maximum(np.maximum(grid.y0 - y, y - grid.y1), 0.0)
    return 1.0 + 1j * gprime(d, amp, ramp, profile)


def _dgamma(c, lo, hi, amp, ramp, profile):
    """gamma_i' = i g_i'' at coordinate c: g_i(c) = g(c - hi) beyond hi, -g(lo - c)
    below lo (Section 1), so g_i'' = g''(c - hi) there and -g''(lo - c) below."""
    return 1j * (gsecond(c - hi, amp, ramp, profile) - gsecond(lo - c, amp, ramp, profile))


def global_dgamma_x(grid: Grid, s, amp, ramp, profile: int = 0):
    """gamma_1'(x) = i g_1''(x) of the global PML at half-index s."""
    return _dgamma(grid.xs(s), grid.x0, grid.x1, amp, ramp, profile)


def global_dgamma_y(grid: Grid, s, amp, ramp, profile: int = 0):
    return _dgamma(grid.ys(s), grid.y0, grid.y1, amp, ramp, profile)


# ----------------------------------------------------------------------------
# Element assembly
# ----------------------------------------------------------------------------

# Triangles of cell (i, j), vertices as (di, dj) offsets, gradients of the
# hat functions in units of 1/h, and the three edge midpoints in half-index
# offsets from (2i, 2j) with the hat values there.
_TRI = [
    # lower: (i,j), (i+1,j), (i+1,j+1)
    dict(verts=[(0, 0), (1, 0), (1, 1)],
         grads=[(-1.0, 0.0), (1.0, -1.0), (0.0, 1.0)],
         mids=[((1, 0), (0.5, 0.5, 0.0)),
               ((2, 1), (0.0, 0.5, 0.5)),
               ((1, 1), (0.5, 0.0, 0.5))]),
    # upper: (i,j), (i+1,j+1), (i,j+1)
    dict(verts=[(0, 0), (1, 1), (0, 1)],
         grads=[(0.0, -1.0), (1.0, 0.0), (-1.0, 1.0)],
         mids=[((1, 1), (0.5, 0.5, 0.0)),
               ((1, 2), (0.0, 0.5, 0.5)),
               ((0, 1), (0.5, 0.0, 0.5))]),
]


def assemble_cells(grid: Grid, ci, cj, gx_fn, gy_fn, k: float):
    """Element contributions of the symmetric stretched form over cells (ci, cj).

    ci, cj: integer arrays of cell indices (same shape). gx_fn(s), gy_fn(s):
    gamma_1 and gamma_2 at half-index positions. Returns COO triplets over
    global node ids (node (i, j) -> j*(Mx+1) + i).
    Each triangle T (area h^2/2) contributes
        int_T (g2/g1) dxphi_a dxphi_b + (g1/g2) dyphi_a dyphi_b - k^2 g1 g2 phi_a phi_b
    with every integral by the edge-midpoint rule, weight |T|/3 = h^2/6.
    """
    ci = np.asarray(ci).ravel()
    cj = np.asarray(cj).ravel()
    h = grid.h
    rows, cols, vals = [], [], []
    for tri in _TRI:
        sx = [2 * ci + m[0][0] for m in tri["mids"]]
        sy = [2 * cj + m[0][1] for m in tri["mids"]]
        g1 = [gx_fn(s) for s in sx]
        g2 = [gy_fn(s) for s in sy]
        kx = sum(g2[m] / g1[m] for m in range(3)) / 6.0     # (1/h^2) int_T g2/g1
        ky = sum(g1[m] / g2[m] for m in range(3)) / 6.0
        mass_w = [g1[m] * g2[m] * (h * h / 6.0) for m in range(3)]
        nodes = [(cj + dj) * (grid.Mx + 1) + (ci + di) for (di, dj) in tri["verts"]]
        for a in range(3):
            for b in range(3):
                ga, gb = tri["grads"][a], tri["grads"][b]
                stiff = kx * (ga[0] * gb[0]) + ky * (ga[1] * gb[1])
                mass = sum(mass_w[m] * tri["mids"][m][1][a] * tri["mids"][m][1][b]
                           for m in range(3))
                rows.append(nodes[a])
                cols.append(nodes[b])
                vals.append(stiff - k * k * mass)
    return (np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def assemble_cells_weak(grid: Grid, ci, cj, gx_fn, gy_fn, dgx_fn, dgy_fn, k: float):
    """Element contributions of the paper's eq. weak itself over cells (ci, cj).

        a(u, v) = int (D grad u) . grad v - (beta . grad u) v - k^2 u v,
        D = diag(gamma_1^-2, gamma_2^-2), beta_i = gamma_i' / gamma_i^3,

    which is not symmetric (the beta term). Row a is the test function phi_a,
    column b the trial function phi_b; on triangle T
        int_T D11 dxphi_b dxphi_a + D22 dyphi_b dyphi_a
              - (beta_1 dxphi_b + beta_2 dyphi_b) phi_a - k^2 phi_b phi_a,
    every integral by the edge-midpoint rule (weight h^2/6 per midpoint).
    dgx_fn(s), dgy_fn(s): gamma_1' and gamma_2' at half-index positions.
    """
    ci = np.asarray(ci).ravel()
    cj = np.asarray(cj).ravel()
    h = grid.h
    rows, cols, vals = [], [], []
    for tri in _TRI:
        sx = [2 * ci + m[0][0] for m in tri["mids"]]
        sy = [2 * cj + m[0][1] for m in tri["mids"]]
        g1 = [gx_fn(s) for s in sx]
        g2 = [gy_fn(s) for s in sy]
        b1 = [dgx_fn(s) / g ** 3 for s, g in zip(sx, g1)]
        b2 = [dgy_fn(s) / g ** 3 for s, g in zip(sy, g2)]
        dx = sum(1.0 / (g1[m] * g1[m]) for m in range(3)) / 6.0   # (1/h^2) int_T D11
        dy = sum(1.0 / (g2[m] * g2[m]) for m in range(3)) / 6.0
        nodes = [(cj + dj) * (grid.Mx + 1) + (ci + di) for (di, dj) in tri["verts"]]
        for a in range(3):
            for b in range(3):
                ga, gb = tri["grads"][a], tri["grads"][b]
                stiff = dx * (gb[0] * ga[0]) + dy * (gb[1] * ga[1])
                adv = sum((b1[m] * gb[0] + b2[m] * gb[1]) * tri["mids"][m][1][a]
                          for m in range(3)) * (h / 6.0)
                mass = sum(tri["mids"][m][1][a] * tri["mids"][m][1][b] for m in range(3)) * (h * h / 6.0)
                rows.append(nodes[a])
                cols.append(nodes[b])
                vals.append(stiff - adv - k * k * mass)
    return (np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def load_cells(grid: Grid, ci, cj, f_fn):
    """Load contributions int_T f phi_a over cells, by the same edge-midpoint rule."""
    ci = np.asarray(ci).ravel()
    cj = np.asarray(cj).ravel()
    h = grid.h
    rows, vals = [], []
    for tri in _TRI:
        fm = [f_fn(2 * ci + m[0][0], 2 * cj + m[0][1]) for m in tri["mids"]]
        nodes = [(cj + dj) * (grid.Mx + 1) + (ci + di) for (di, dj) in tri["verts"]]
        for a in range(3):
            v = sum(fm[m] * tri["mids"][m][1][a] for m in range(3)) * (h * h / 6.0)
            rows.append(nodes[a])
            vals.append(v)
    return np.concatenate(rows), np.concatenate(vals)


def interior_numbering(grid: Grid):
    """Map global node id -> unknown index (-1 on the outer boundary), x-fastest."""
    num = -np.ones((grid.My + 1, grid.Mx + 1), dtype=np.int64)
    num[1:grid.My, 1:grid.Mx] = np.arange(grid.n).reshape(grid.ny, grid.nx)
    return num.ravel()


def _to_matrix(rows, cols, vals, numbering, n):
    ur = numbering[rows]
    uc = numbering[cols]
    keep = (ur >= 0) & (uc >= 0)
    A = sp.coo_matrix((vals[keep], (ur[keep], uc[keep])), shape=(n, n)).tocsr()
    A.sum_duplicates()
    return A


def assemble_global(p: dict, gx_fn=None, gy_fn=None, dgx_fn=None, dgy_fn=None):
    """Global matrix A of a(.,.) on V_h subset H^1_0(Omega) (Section 1, eq. weak).

    p["form"] (default 0) selects the bilinear form: 0 the gamma_1 gamma_2
    multiplied, complex-symmetric one; 1 eq. weak as printed (not symmetric).
    gx_fn/gy_fn (and dgx_fn/dgy_fn, the derivatives, for form 1) override the
    stretching (tests); default: the global PML.
    Returns (grid, A) with A a CSR complex128 matrix of size n x n.
    """
    grid = make_grid(p)
    amp, ramp, prof = p["g_amp"], p["g_ramp"], p.get("g_profile", 0)
    if gx_fn is None:
        gx_fn = lambda s: global_gamma_x(grid, s, amp, ramp, prof)  # noqa: E731
    if gy_fn is None:
        gy_fn = lambda s: global_gamma_y(grid, s, amp, ramp, prof)  # noqa: E731
    if dgx_fn is None:
        dgx_fn = lambda s: global_dgamma_x(grid, s, amp, ramp, prof)  # noqa: E731
    if dgy_fn is None:
        dgy_fn = lambda s: global_dgamma_y(grid, s, amp, ramp, prof)  # noqa: E731
    cj, ci = np.meshgrid(np.arange(grid.My), np.arange(grid.Mx), indexing="ij")
    if p.get("form", 0) == 1:
        r, c, v = assemble_cells_weak(grid, ci, cj, gx_fn, gy_fn, dgx_fn, dgy_fn, p["k"])
    else:
        r, c, v = assemble_cells(grid, ci, cj, gx_fn, gy_fn, p["k"])
    return grid, _to_matrix(r, c, v, interior_numbering(grid), grid.n)


def source_function(grid: Grid, centres, amps, width):
    """f(x) = sum_s amp_s exp(-|x - c_s|^2 / width^2), cut to Omega_int.

    The cut to Omega_int (f is supported there, Section 1) is taken on the
    closed box [x0,x1] x [y0,y1].
    """
    centres = np.asarray(centres, dtype=np.float64).reshape(-1, 2)
    amps = np.asarray(amps, dtype=np.float64).ravel()

    def f(sx, sy):
        x = grid.xs(sx)
        y = grid.ys(sy)
        val = np.zeros(np.broadcast(x, y).shape)
        for (cx, cy), a in zip(centres, amps):
            val = val + a * np.exp(-((x - cx) ** 2 + (y - cy) ** 2) / (width * width))
        inside = (x >= grid.x0) & (x <= grid.x1) & (y >= grid.y0) & (y <= grid.y1)
        return np.where(inside, val, 0.0)
    return f


def assemble_rhs(p: dict, centres, amps, width):
    """Load vector F_i = int f phi_i over interior unknowns (complex128)."""
    grid = make_grid(p)
    f = source_function(grid, centres, amps, width)
    cj, ci = np.meshgrid(np.arange(grid.My), np.arange(grid.Mx), indexing="ij")
    rows, vals = load_cells(grid, ci, cj, f)
    num = interior_numbering(grid)
    u = num[rows]
    keep = u >= 0
    b = np.zeros(grid.n, dtype=np.complex128)
    np.add.at(b, u[keep], vals[keep])
    return b


def point_source_rhs(grid: Grid, i: int, j: int):
    """b = (phi_l(x_s))_l for a point source at node (i, j): a unit vector."""
    b = np.zeros(grid.n, dtype=np.complex128)
    b[(j - 1) * grid.nx + (i - 1)] = 1.0
    return b


# ----------------------------------------------------------------------------
# Direct solves (the plain definition u_h = A^-1 F)
# ----------------------------------------------------------------------------

def direct_solve(A, b):
    """u = A^-1 b by sparse LU with partial pivoting (SuperLU)."""
    return spla.splu(A.tocsc()).solve(np.asarray(b, dtype=np.complex128))


def dense_solve(A, b):
    """u = A^-1 b by dense LAPACK (brute force, tiny meshes only)."""
    return np.linalg.solve(A.toarray(), np.asarray(b, dtype=np.complex128))


def unknown_coords(grid: Grid):
    """(x, y) of every unknown, in unknown order."""
    jj, ii = np.meshgrid(np.arange(1, grid.My), np.arange(1, grid.Mx), indexing="ij")
    return grid.xs(2 * ii.ravel()), grid.ys(2 * jj.ravel())


def hankel_solution(x, y, xs, ys, k):
    """Outgoing free-space solution of -Delta u - k^2 u = delta: (i/4) H_0^(1)(k r)."""
    from scipy.special import hankel1
    r = np.hypot(x - xs, y - ys)
    return 0.25j * hankel1(0, k * r)


def law_cells(k: float, h: float) -> int:
    """Whole cells in 0.5*ln(k)/k, rounded half up, at least one."""
    return max(1, int(math.floor(0.5 * math.log(k) / k / h + 0.5)))
