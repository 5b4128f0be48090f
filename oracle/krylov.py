"""Oracle, part 3: outer iterations (paper Algorithm 1 and Section 4.1).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

richardson: Algorithm 1 in discrete form (eq. local-ras-discrete and
    eq. update1): u <- u + B^-1 (F - A u).
fgmres:     flexible GMRES with B^-1 as a right preconditioner (Section 4.1
    uses GMRES with the method as preconditioner; flexible GMRES stores the
    preconditioned directions z_j and is identical in exact arithmetic for a
    fixed B^-1). x0 = 0 unless given, modified Gram-Schmidt on the Hermitian
    inner product, complex Givens rotations, no restart unless asked.
    Stops when the Arnoldi estimate of ||b - A x|| / ||b|| is <= rtol, or
    after maxit directions.
gmres_right: the same with x = x0 + B^-1 (V y), for the fixed-preconditioner
    form.
"""
from __future__ import annotations

import numpy as np


def _givens(a, b):
    """(c, s, r) with c real, [c s; -conj(s) c] [a; b] = [r; 0]."""
    aa, bb = abs(a), abs(b)
    if bb == 0.0:
        return 1.0, 0.0 + 0.0j, a
    if aa == 0.0:
        return 0.0, 1.0 + 0.0j, b
    nrm = np.hypot(aa, bb)
    ph = a / aa
    return aa / nrm, ph * np.conj(b) / nrm, ph * nrm


def _arnoldi_solve(matvec, prec, b, x0, rtol, maxit, restart, flexible):
    b = np.asarray(b, dtype=np.complex128)
    n = b.size
    x = np.zeros(n, dtype=np.complex128) if x0 is None else np.array(x0, dtype=np.complex128)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, 0, 0.0, [0.0]
    restart = maxit if restart is None else restart
    total = 0
    hist = []
    while True:
        r = b - matvec(x)
        beta = np.linalg.norm(r)
        hist.append(beta / bnorm)
        if beta / bnorm <= rtol or total >= maxit:
            return x, total, beta / bnorm, hist
        m = min(restart, maxit - total)
        V = np.zeros((m + 1, n), dtype=np.complex128)
        Z = np.zeros((m, n), dtype=np.complex128) if flexible else None
        H = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        g[0] = beta
        V[0] = r / beta
        j_done = 0
        for j in range(m):
            z = prec(V[j])
            if flexible:
                Z[j] = z
            w = matvec(z)
            for i in range(j + 1):               # modified Gram-Schmidt
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            for i in range(j):                   # previous rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            c, s, rr = _givens(H[j, j], H[j + 1, j])
            cs[j], sn[j] = c, s
            H[j, j] = rr
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(s) * g[j]
            g[j] = c * g[j]
            j_done = j + 1
            total += 1
            est = abs(g[j + 1]) / bnorm
            hist.append(est)
            hn = np.linalg.norm(w)
            if est <= rtol or total >= maxit or hn == 0.0:
                break
            V[j + 1] = w / hn
        y = np.zeros(j_done, dtype=np.complex128)
        for i in range(j_done - 1, -1, -1):     # back substitution
            y[i] = (g[i] - H[i, i + 1:j_done] @ y[i + 1:j_done]) / H[i, i]
        if flexible:
            x = x + y @ Z[:j_done]
        else:
            x = x + prec(y @ V[:j_done])
        if total >= maxit or abs(g[j_done]) / bnorm <= rtol:
            r = b - matvec(x)
            return x, total, np.linalg.norm(r) / bnorm, hist


def fgmres(matvec, prec, b, x0=None, rtol=1e-6, maxit=500, restart=None):
    """Flexible GMRES(restart) with right preconditioner `prec`.

    Returns (x, iterations, true relative residual, estimate history).
    """
    return _arnoldi_solve(matvec, prec, b, x0, rtol, maxit, restart, True)


def gmres_right(matvec, prec, b, x0=None, rtol=1e-6, maxit=500, restart=None):
    """Right-preconditioned GMRES(restart): x = x0 + prec(V y)."""
    return _arnoldi_solve(matvec, prec, b, x0, rtol, maxit, restart, False)


def richardson(matvec, prec, b, x0=None, rtol=1e-6, maxit=500):
    """Algorithm 1 (discrete): u <- u + B^-1 (b - A u) until ||b - A u||/||b|| <= rtol."""
    b = np.asarray(b, dtype=np.complex128)
    u = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128)
    bnorm = np.linalg.norm(b)
    hist = []
    for it in range(maxit + 1):
        r = b - matvec(u)
        rel = np.linalg.norm(r) / bnorm
        hist.append(rel)
        if rel <= rtol or it == maxit or not np.isfinite(rel):
            return u, it, rel, hist
        u = u + prec(r)
