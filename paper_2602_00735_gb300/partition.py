"""Partition of the RAS-PML hot path over ranks, one GPU per rank: the px x py
grid of subdomains (Section 2, the Cartesian covering) split into an Rx x Ry
grid of rank blocks, and the exchanges that one apply of B^-1 and one global
product A x need. Host logic only (index arithmetic on the covering); the
exchanges it describes run as point-to-point sends into each rank's own
buffers, plus one all-reduce of the Arnoldi inner products per direction.

Ownership. Rank (rx, ry) owns the subdomains of its block of boxes and the
global unknowns of those boxes' cells: node i belongs to the box whose cells
[c_q, c_q+1) contain it (a node on a box edge belongs to the upper box).

One apply z = B^-1 r = sum_j R_j^T (chi_j * A_j^-1 R_j r):
  * restriction: a rank's subdomains read r at every node of their Omega_j
    (the box widened by ovlp + pml cells); the nodes owned by other ranks
    form the restriction halo, received from their owners;
  * prolongation: chi_j is non-zero only inside Omega_j,int (the box widened
    by ovlp), so a subdomain contributes to other ranks' nodes only in the
    overlap strips; each contribution goes to the node's owner, which sums
    the contributions of every subdomain covering the node in increasing
    subdomain order (the order of the one-rank sum).
  This is the paper's observation that the exchanges of the method live on
  the overlaps (Section 3 (i); Section 4 runs one process per subdomain).
One product y = A x needs x one node beyond the owned ones (the 1-cell
halo of the seven-point stencil).

Algorithm 1 (u <- u + B^-1 (F - A u)) after its first sweep: the new
residual vanishes at every node whose stencil lies where a single chi_j is 1
(there A B^-1 r reproduces r exactly), so it lives on the nodes within ovlp
of an interior box edge in either direction (Section 3 (i)). The restriction
halo of those sweeps shrinks to its part in that support
(restrict_recv_sparse): the local PML extension beyond the overlap is no
longer exchanged.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = ["box_edges", "split_blocks", "Plan"]


def box_edges(M: int, P: int) -> np.ndarray:
    """Cell indices c_0 = 0 < ... < c_P = M of P boxes of M cells, the first
    M mod P boxes one cell wider."""
    base, extra = divmod(M, P)
    sizes = [base + (1 if q < extra else 0) for q in range(P)]
    return np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)


def split_blocks(P: int, R: int) -> np.ndarray:
    """Box indices b_0 = 0 < ... < b_R = P of R rank blocks of P boxes."""
    if not 1 <= R <= P:
        raise ValueError(f"{R} ranks along an axis of {P} boxes")
    return box_edges(P, R)


@dataclass
class _Axis:
    """One direction of the covering: per box, its cells, Omega_j,int and
    Omega_j (in cells), and the local unknown nodes."""
    M: int
    edges: np.ndarray
    int_lo: np.ndarray
    int_hi: np.ndarray
    ext_lo: np.ndarray
    ext_hi: np.ndarray
    node_lo: np.ndarray     # first local unknown node
    node_hi: np.ndarray     # last local unknown node


def _axis(M: int, P: int, ovlp: int, pml: int, local_bc: int) -> _Axis:
    c = box_edges(M, P)
    lo_in = np.arange(P) > 0
    hi_in = np.arange(P) < P - 1
    int_lo = c[:-1] - np.where(lo_in, ovlp, 0)
    int_hi = c[1:] + np.where(hi_in, ovlp, 0)
    ext_lo = np.maximum(0, int_lo - np.where(lo_in, pml, 0))
    ext_hi = np.minimum(M, int_hi + np.where(hi_in, pml, 0))
    if local_bc == 0:       # impedance: the artificial-boundary nodes are unknowns
        node_lo, node_hi = ext_lo.copy(), ext_hi.copy()
    else:                   # Dirichlet: they are dropped
        node_lo, node_hi = ext_lo + 1, ext_hi - 1
    node_lo = np.maximum(node_lo, 1)
    node_hi = np.minimum(node_hi, M - 1)
    return _Axis(M, c, int_lo, int_hi, ext_lo, ext_hi, node_lo, node_hi)


@dataclass
class Plan:
    """Ownership and exchange lists of one rank layout. Global unknown (i, j),
    1 <= i < Mx, 1 <= j < My, has index (j - 1)(Mx - 1) + (i - 1).

    For every rank r:
      subdomains[r]          its subdomains (natural index qy px + qx)
      owned[r]               its unknowns, sorted
      restrict_recv[r][s]    unknowns it receives from rank s before an apply
      restrict_recv_sparse[r][s]  the same within the residual's support (the
                             later sweeps of Algorithm 1)
      prolong_send[r][s]     (subdomain, unknown) pairs whose contribution it
                             sends to rank s after its local solves
      spmv_recv[r][s]        unknowns it receives from rank s before a product
    The send lists of restriction and SpMV are the mirrored receive lists:
    restrict_recv[s][r] is what r sends to s."""
    Mx: int
    My: int
    px: int
    py: int
    ovlp: int
    pml: int
    local_bc: int
    Rx: int
    Ry: int
    subdomains: list = field(default_factory=list)
    owned: list = field(default_factory=list)
    restrict_recv: list = field(default_factory=list)
    restrict_recv_sparse: list = field(default_factory=list)
    prolong_send: list = field(default_factory=list)
    spmv_recv: list = field(default_factory=list)

    @property
    def nranks(self) -> int:
        return self.Rx * self.Ry

    @classmethod
    def build(cls, Mx: int, My: int, px: int, py: int, ovlp: int, pml: int, local_bc: int, Rx: int, Ry: int):
        X = _axis(Mx, px, ovlp, pml, local_bc)
        Y = _axis(My, py, ovlp, pml, local_bc)
        bx, by = split_blocks(px, Rx), split_blocks(py, Ry)
        nx = Mx - 1
        # owner rank of every interior node, from the box that holds its cell
        box_x = np.searchsorted(X.edges, np.arange(1, Mx), side="right") - 1
        box_y = np.searchsorted(Y.edges, np.arange(1, My), side="right") - 1
        rank_x = np.searchsorted(bx, box_x, side="right") - 1
        rank_y = np.searchsorted(by, box_y, side="right") - 1
        owner = (rank_y[:, None] * Rx + rank_x[None, :]).ravel()   # index (j-1) nx + (i-1)
        plan = cls(Mx, My, px, py, ovlp, pml, local_bc, Rx, Ry)
        R = Rx * Ry
        support = plan.residual_support()

        def nodes(lo, hi):
            return np.arange(lo, hi + 1)

        for r in range(R):
            rx, ry = r % Rx, r // Rx
            subs = [qy * px + qx for qy in range(by[ry], by[ry + 1]) for qx in range(bx[rx], bx[rx + 1])]
            plan.subdomains.append(subs)
            plan.owned.append(np.nonzero(owner == r)[0])
            need, contrib = set(), {s: [] for s in range(R)}
            for q in subs:
                qx, qy = q % px, q // px
                ii, jj = nodes(X.node_lo[qx], X.node_hi[qx]), nodes(Y.node_lo[qy], Y.node_hi[qy])
                g = ((jj[:, None] - 1) * nx + (ii[None, :] - 1)).ravel()
                need.update(g[owner[g] != r].tolist())
                # chi_j > 0 strictly inside Omega_j,int in each direction
                ci = ii[(ii > X.int_lo[qx]) | (X.int_lo[qx] == 0)]
                ci = ci[(ci < X.int_hi[qx]) | (X.int_hi[qx] == Mx)]
                cj = jj[(jj > Y.int_lo[qy]) | (Y.int_lo[qy] == 0)]
                cj = cj[(cj < Y.int_hi[qy]) | (Y.int_hi[qy] == My)]
                gc = ((cj[:, None] - 1) * nx + (ci[None, :] - 1)).ravel()
                for s in np.unique(owner[gc]):
                    if s != r:
                        contrib[int(s)].extend((q, int(v)) for v in gc[owner[gc] == s])
            need = np.array(sorted(need), dtype=np.int64)
            plan.restrict_recv.append({int(s): need[owner[need] == s] for s in np.unique(owner[need])})
            sparse = need[support[need]]
            plan.restrict_recv_sparse.append({int(s): sparse[owner[sparse] == s] for s in np.unique(owner[sparse])})
            plan.prolong_send.append({s: v for s, v in contrib.items() if v})
            # SpMV halo: the W, E, S, N, SW, NE neighbours of owned nodes
            o = plan.owned[r]
            oi, oj = o % nx, o // nx
            halo = set()
            for di, dj in ((-1, 0), (1, 0), (0, -1), (0, 1), (-1, -1), (1, 1)):
                ni, nj = oi + di, oj + dj
                ok = (ni >= 0) & (ni < nx) & (nj >= 0) & (nj < My - 1)
                g = nj[ok] * nx + ni[ok]
                halo.update(g[owner[g] != r].tolist())
            halo = np.array(sorted(halo), dtype=np.int64)
            plan.spmv_recv.append({int(s): halo[owner[halo] == s] for s in np.unique(owner[halo])})
        return plan

    def residual_support(self) -> np.ndarray:
        """Mask over the unknowns of where a residual b - A u can be non-zero
        after a sweep of Algorithm 1: nodes within ovlp of an interior box
        edge in x or in y (their stencil touches a node covered by two
        subdomains' chi > 0)."""
        def near(M, P):
            c = box_edges(M, P)[1:-1]
            i = np.arange(1, M)
            if c.size == 0:
                return np.zeros(M - 1, dtype=bool)
            return np.min(np.abs(i[:, None] - c[None, :]), axis=1) <= self.ovlp
        sx, sy = near(self.Mx, self.px), near(self.My, self.py)
        return (sy[:, None] | sx[None, :]).ravel()

    def restrict_send_sparse(self, r: int) -> dict:
        """Unknowns rank r sends to each other rank before a later sweep of
        Algorithm 1 (the residual's support only)."""
        return {s: self.restrict_recv_sparse[s][r] for s in range(self.nranks) if r in self.restrict_recv_sparse[s]}

    def restrict_send(self, r: int) -> dict:
        """Unknowns rank r sends to each other rank before an apply."""
        return {s: self.restrict_recv[s][r] for s in range(self.nranks) if r in self.restrict_recv[s]}

    def spmv_send(self, r: int) -> dict:
        """Unknowns rank r sends to each other rank before a product."""
        return {s: self.spmv_recv[s][r] for s in range(self.nranks) if r in self.spmv_recv[s]}

    def prolong_recv(self, r: int) -> dict:
        """(subdomain, unknown) pairs whose contributions rank r receives."""
        return {s: self.prolong_send[s][r] for s in range(self.nranks) if r in self.prolong_send[s]}

    def exchange_bytes(self, r: int, entry_bytes: int = 16) -> dict:
        """Bytes rank r receives per apply and per product (complex128
        entries): restriction halo, prolongation contributions, SpMV halo."""
        return {"restrict": entry_bytes * sum(len(v) for v in self.restrict_recv[r].values()),
                "restrict_sparse": entry_bytes * sum(len(v) for v in self.restrict_recv_sparse[r].values()),
                "prolong": entry_bytes * sum(len(v) for v in self.prolong_recv(r).values()),
                "spmv": entry_bytes * sum(len(v) for v in self.spmv_recv[r].values())}
