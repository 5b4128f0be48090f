"""Seeded synthetic workloads for the RAS-PML Helmholtz solver.

This module is the one piece shared by the CPU oracle and the CUDA path. It
holds problem parameters and seeded random draws only (wavenumber, domain,
mesh size, subdomain grid, widths, Gaussian source centres); it contains none
of the method's arithmetic (no stretching, quadrature, assembly or solve).

Workloads (all with wave speed c = 1 and a Cartesian PML of width 0.1 around
Omega_int, stretching profile g'(x) = 20 (3t^2 - 2t^3), t = min(x/0.05, 1)):

  c0   k = 20*pi,  h = 1/160,  4 x 4 subdomains,    3 Gaussians, width 0.02
  c1   k = 80*pi,  h = 1/640,  16 x 16 subdomains,  8 Gaussians, width 0.005
  c2   k = 160*pi, h = 1/1280, 32 x 32 subdomains, 16 Gaussians, width 0.0025
  c4   k = 320*pi, h = 1/2560, 64 x 64 subdomains, 32 Gaussians, width 0.00125

Omega_int = (0,1)^2 in all four; overlap and local PML width are both
0.5*ln(k)/k rounded half up to whole cells (at least one cell). Source centres
are uniform in Omega_int from numpy's default_rng(seed); amplitudes are 1.
Smaller "tiny*" workloads with the same construction serve the tests.

paper_setup(k, cells_per_box, ...) builds the set-up of the paper's own
experiments (Omega = (0,1)^2 with a three-wavelength PML, h = 1/(2k),
g(x) = 10 k x^3, smoothed-delta source, the paper's width law).

batch(name) returns a list of independent problems for the batched form:
  c3   64 problems; k log-uniform in [20*pi, 120*pi]; Omega_int = (0, s)^2
       with s uniform in [0.5, 1.5] and the same PML of width 0.1; about 16
       points per wavelength (h = (s + 0.2)/M, M = round((s + 0.2) 16 k / 2 pi));
       overlap and local PML width 0.5*ln(k)/k in cells; px and py drawn
       independently and uniformly from 2..12; 1..8 Gaussian sources (width
       0.4*pi/k, amplitude 1) uniform in Omega_int. All draws from numpy's
       default_rng(seed). A drawn grid whose boxes could not hold the two
       overlap strips (fewer than 2*overlap cells) raises instead of being
       redrawn; seed 3 draws none.
  c3small  8 problems of the same construction at k in [8*pi, 24*pi] (test
       size); there px, py are drawn from 2 up to the largest count whose
       boxes hold the two overlap strips.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

__all__ = ["Workload", "get", "batch", "width_cells", "NAMES", "BATCH_NAMES"]


def width_cells(k: float, h: float) -> int:
    """Cells in 0.5*ln(k)/k, rounded half up, at least 1 (workload recipe)."""
    return max(1, int(math.floor(0.5 * math.log(k) / k / h + 0.5)))


@dataclass
class Workload:
    name: str
    k: float
    x0: float
    y0: float
    x1: float
    y1: float
    kappa_g: float
    h: float
    px: int
    py: int
    ovlp_cells: int
    pml_cells: int
    g_amp: float = 20.0
    g_ramp: float = 0.05
    local_bc: int = 0          # 0 impedance (RAS-PML-Imp), 1 Dirichlet
    g_profile: int = 0         # 0 smoothstep ramp; 1 g(d) = g_amp d^3
    form: int = 0              # 0 gamma_1 gamma_2 (symmetric) form; 1 eq. weak as printed
    centres: np.ndarray = field(default_factory=lambda: np.zeros((0, 2)))
    amps: np.ndarray = field(default_factory=lambda: np.zeros(0))
    width: float = 0.02
    seed: int = 0

    @property
    def cells_x(self) -> int:
        return int(round((self.x1 - self.x0 + 2 * self.kappa_g) / self.h))

    @property
    def cells_y(self) -> int:
        return int(round((self.y1 - self.y0 + 2 * self.kappa_g) / self.h))

    @property
    def n_unknowns(self) -> int:
        return (self.cells_x - 1) * (self.cells_y - 1)

    def params(self) -> dict:
        """Scalar parameters, in the field order of the C parameter struct."""
        return dict(k=self.k, x0=self.x0, y0=self.y0, x1=self.x1, y1=self.y1,
                    kappa_g=self.kappa_g, h=self.h, px=self.px, py=self.py,
                    ovlp_cells=self.ovlp_cells, pml_cells=self.pml_cells,
                    g_amp=self.g_amp, g_ramp=self.g_ramp, local_bc=self.local_bc,
                    g_profile=self.g_profile, form=self.form)

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)


def _make(name, k, h, p, ns, width, seed, side=1.0, kappa_g=0.1, ovlp=None, pml=None):
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0.0, side, size=(ns, 2))
    w = width_cells(k, h)
    return Workload(name=name, k=k, x0=0.0, y0=0.0, x1=side, y1=side,
                    kappa_g=kappa_g, h=h, px=p, py=p,
                    ovlp_cells=w if ovlp is None else ovlp,
                    pml_cells=w if pml is None else pml,
                    centres=centres, amps=np.ones(ns), width=width, seed=seed)


def paper_width_cells(k: float, h: float, C: float, k0: float = 150.0) -> int:
    """C * l(k) * 2*pi/k in whole cells (rounded half up, at least 1), with
    l(k) = k/(k - k0) * log2(k/k0): the overlap / PML width law the paper
    proposes for k > k0 (Section 3 (iii))."""
    if not k > k0:
        raise ValueError("the width law needs k > k0")
    ell = k / (k - k0) * math.log2(k / k0)
    return max(1, int(math.floor(C * ell * 2 * math.pi / k / h + 0.5)))


def paper_setup(k: int, cells_per_box: int, C_delta: float = 1.0 / 6, C_kappa: float = 0.5,
                local_bc: int = 0, pml: bool = True) -> Workload:
    """The set-up of the paper's experiments (Section 4) on P1 triangles:
    Omega = (0,1)^2 holds Omega_int and a global PML of three wavelengths
    (kappa_g rounded to whole cells), h = 1/(2k) (12 points per wavelength),
    stretching g(x) = 10 k x^3, the smoothed-delta source
    f = 16k^2/pi^3 exp(-16 k^2 |x - (0.5,0.5)|^2 / pi^2) (a Gaussian of width
    pi/(4k) and unit integral), overlap and local PML widths from the paper's
    law. The number of boxes is chosen so that boxes have about
    `cells_per_box` cells (the paper's boxes have ~300; the GPU kernels here
    take subdomains up to ~110 cells across). pml=False gives RAS-Imp."""
    if int(k) != k:
        raise ValueError("k must be an integer (h = 1/(2k))")
    M = 2 * int(k)
    h = 1.0 / M
    lam = 2 * math.pi / k
    kg_cells = max(1, int(math.floor(3 * lam / h + 0.5)))
    kappa_g = kg_cells * h
    P = max(1, int(round(M / cells_per_box)))
    ovlp = paper_width_cells(k, h, C_delta)
    pml_cells = paper_width_cells(k, h, C_kappa) if pml else 0
    w = math.pi / (4 * k)
    return Workload(name=f"paper-k{k}", k=float(k), x0=kappa_g, y0=kappa_g, x1=1 - kappa_g, y1=1 - kappa_g,
                    kappa_g=kappa_g, h=h, px=P, py=P, ovlp_cells=ovlp, pml_cells=pml_cells,
                    g_amp=10.0 * k, g_ramp=1.0, local_bc=local_bc, g_profile=1,
                    centres=np.array([[0.5, 0.5]]), amps=np.array([16 * k * k / math.pi ** 3]), width=w, seed=0)


def get(name: str) -> Workload:
    """Return the named seeded workload."""
    pi = math.pi
    table = {
        "c0": lambda: _make("c0", 20 * pi, 1 / 160, 4, 3, 0.02, 0),
        "c1": lambda: _make("c1", 80 * pi, 1 / 640, 16, 8, 0.005, 1),
        "c2": lambda: _make("c2", 160 * pi, 1 / 1280, 32, 16, 0.0025, 2),
        "c4": lambda: _make("c4", 320 * pi, 1 / 2560, 64, 32, 0.00125, 4),
        # small cases with the same construction (tests)
        "tiny": lambda: _make("tiny", 4 * pi, 1 / 40, 2, 2, 0.08, 10, ovlp=2, pml=3),
        "tiny3": lambda: _make("tiny3", 8 * pi, 1 / 50, 3, 3, 0.05, 11, ovlp=2, pml=3),
        "small": lambda: _make("small", 10 * pi, 1 / 80, 4, 3, 0.04, 12),
        "mid": lambda: _make("mid", 40 * pi, 1 / 320, 8, 5, 0.01, 13),
    }
    if name not in table:
        raise KeyError(f"unknown workload {name!r}; known: {sorted(table)}")
    return table[name]()


NAMES = ("c0", "c1", "c2", "c4", "tiny", "tiny3", "small", "mid")

def _max_boxes(M: int, w: int, cap: int = 12) -> int:
    """The largest box count P <= cap whose boxes (floor(M/P) cells or more)
    hold the two overlap strips of w cells each: the covering's own
    requirement, independent of any kernel."""
    hi = cap
    while hi >= 2 and M // hi < 2 * w:
        hi -= 1
    if hi < 2:
        raise ValueError(f"no subdomain grid of 2 or more boxes fits M={M}, w={w}")
    return hi


def _batch_c3(count=64, seed=3, name="c3") -> list:
    rng = np.random.default_rng(seed)
    out = []
    for q in range(count):
        k = float(np.exp(rng.uniform(math.log(20 * math.pi), math.log(120 * math.pi))))
        side = float(rng.uniform(0.5, 1.5))
        L = side + 0.2
        M = int(round(L * 16 * k / (2 * math.pi)))
        h = L / M
        w = width_cells(k, h)
        px, py = (int(v) for v in rng.integers(2, 13, size=2))
        if M // max(px, py) < 2 * w:
            raise ValueError(f"{name}-{q}: {px}x{py} boxes of {M} cells cannot hold two overlaps of {w} cells")
        ns = int(rng.integers(1, 9))
        centres = rng.uniform(0.0, side, size=(ns, 2))
        out.append(Workload(name=f"{name}-{q}", k=k, x0=0.0, y0=0.0, x1=side, y1=side, kappa_g=0.1, h=h,
                            px=px, py=py, ovlp_cells=w, pml_cells=w, centres=centres, amps=np.ones(ns),
                            width=0.4 * math.pi / k, seed=seed))
    return out


def batch(name: str) -> list:
    """Return the named seeded list of problems for the batched form:
    c3 (the 64-problem set), c3small (8 problems of the same construction at
    k in [8*pi, 24*pi], for tests)."""
    if name == "c3":
        return _batch_c3()
    if name == "c3small":
        rng = np.random.default_rng(5)
        out = []
        for q in range(8):
            k = float(np.exp(rng.uniform(math.log(8 * math.pi), math.log(24 * math.pi))))
            side = float(rng.uniform(0.5, 1.5))
            L = side + 0.2
            M = int(round(L * 16 * k / (2 * math.pi)))
            h = L / M
            w = width_cells(k, h)
            hi = _max_boxes(M, w)
            px, py = (int(v) for v in rng.integers(2, hi + 1, size=2))
            ns = int(rng.integers(1, 9))
            out.append(Workload(name=f"c3small-{q}", k=k, x0=0.0, y0=0.0, x1=side, y1=side, kappa_g=0.1, h=h,
                                px=px, py=py, ovlp_cells=w, pml_cells=w,
                                centres=rng.uniform(0.0, side, size=(ns, 2)), amps=np.ones(ns),
                                width=0.4 * math.pi / k, seed=5))
        return out
    raise KeyError(f"unknown batch {name!r}; known: {BATCH_NAMES}")


BATCH_NAMES = ("c3", "c3small")
