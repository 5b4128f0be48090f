"""CPU FP64 oracle of the learned coarse correction -- TEST INFRASTRUCTURE ONLY.

The paper has no learned component; this part of the build adds one as an
extra stage of the flexible GMRES (the preconditioner is B^-1 followed by a
coarse correction of the residual it leaves). Everything here is plain
NumPy in float64, written from the definitions below; no blocking or fusion.

Coarse grid. The fine unknowns form an nx x ny array (x fastest). Coarse
pixel (I, J) of an Nc x Nc grid owns the fine nodes i with
floor(i Nc / nx) = I and j with floor(j Nc / ny) = J.
  restrict(v):  the mean of v over each pixel's nodes (full weighting by
                area in index space), per real channel;
  prolong(c):   bilinear interpolation of pixel values, placed at the pixel
                centres u_I = (I + 1/2) nx / Nc - 1/2 in fine-index units,
                at every fine node, constant beyond the outermost centres.

Network. Six 3x3 convolutions with zero padding, channels
2 -> 32 -> 32 -> 32 -> 32 -> 32 -> 2, a bias per output channel, ReLU after
the first five:  y_l = W_l * a_{l-1} + b_l,  a_l = relu(y_l) (l < 5),
out = y_5, with (W * a)[o, p] = sum_{c, d} W[o, c, d] a[c, p + d - 1]
(cross-correlation; d runs over the 3x3 taps).

Correction. For a fine residual r (complex), x = restrict(r) as two real
channels, s = ||x||_2; the network sees x_hat = x Nc / s and its output
(two channels, re and im) is scaled back by gamma s / Nc, so the correction
is linear in the scale of r: c(r) = prolong(gamma s / Nc * net(x Nc / s)).

Loss for a pair (r, e) (e the error the correction should produce):
t_hat = restrict(e) Nc / (gamma s) and L = mean over pixels and channels of
(net(x_hat) - t_hat)^2 / 2.
"""
from __future__ import annotations

import numpy as np

CHANNELS = (2, 32, 32, 32, 32, 32, 2)
NLAYERS = 6


# ---------------------------------------------------------------- transfer --

def owners(n: int, Nc: int) -> np.ndarray:
    """Coarse index of each of n fine indices: floor(i Nc / n)."""
    return (np.arange(n) * Nc) // n


def restrict(v: np.ndarray, nx: int, ny: int, Nc: int) -> np.ndarray:
    """Complex fine vector (nx*ny, x fastest) -> (2, Nc, Nc) pixel means."""
    f = v.reshape(ny, nx)
    ox, oy = owners(nx, Nc), owners(ny, Nc)
    out = np.zeros((2, Nc, Nc))
    cnt = np.zeros((Nc, Nc))
    np.add.at(cnt, (oy[:, None], ox[None, :]), 1.0)
    for ch, part in enumerate((f.real, f.imag)):
        acc = np.zeros((Nc, Nc))
        np.add.at(acc, (oy[:, None], ox[None, :]), part)
        out[ch] = acc / cnt
    return out


def _weights_1d(n: int, Nc: int):
    """For each fine index: left pixel I0 and weight w of pixel I0 + 1."""
    u = (np.arange(n) + 0.5) * Nc / n - 0.5
    u = np.clip(u, 0.0, Nc - 1.0)
    i0 = np.minimum(np.floor(u).astype(int), Nc - 2)
    return i0, u - i0


def prolong(c: np.ndarray, nx: int, ny: int) -> np.ndarray:
    """(2, Nc, Nc) pixel values -> complex fine vector (bilinear)."""
    Nc = c.shape[1]
    ix, wx = _weights_1d(nx, Nc)
    iy, wy = _weights_1d(ny, Nc)
    out = []
    for ch in range(2):
        g = c[ch]
        a = (1 - wy)[:, None] * ((1 - wx)[None, :] * g[np.ix_(iy, ix)] + wx[None, :] * g[np.ix_(iy, ix + 1)])
        a += wy[:, None] * ((1 - wx)[None, :] * g[np.ix_(iy + 1, ix)] + wx[None, :] * g[np.ix_(iy + 1, ix + 1)])
        out.append(a)
    return (out[0] + 1j * out[1]).ravel()


# ------------------------------------------------------------------ network --

def conv3x3(a: np.ndarray, W: np.ndarray, b: np.ndarray) -> np.ndarray:
    """(C, H, X) input, (O, C, 3, 3) weights, (O,) bias -> (O, H, X)."""
    C, H, X = a.shape
    p = np.zeros((C, H + 2, X + 2))
    p[:, 1:-1, 1:-1] = a
    out = np.zeros((W.shape[0], H, X))
    for dy in range(3):
        for dx in range(3):
            out += np.einsum("oc,chx->ohx", W[:, :, dy, dx], p[:, dy:dy + H, dx:dx + X])
    return out + b[:, None, None]


def conv3x3_backward(a: np.ndarray, W: np.ndarray, gy: np.ndarray):
    """Gradients of sum(gy * conv3x3(a, W, b)) w.r.t. a, W and b."""
    C, H, X = a.shape
    p = np.zeros((C, H + 2, X + 2))
    p[:, 1:-1, 1:-1] = a
    gW = np.zeros_like(W)
    gp = np.zeros_like(p)
    for dy in range(3):
        for dx in range(3):
            gW[:, :, dy, dx] = np.einsum("ohx,chx->oc", gy, p[:, dy:dy + H, dx:dx + X])
            gp[:, dy:dy + H, dx:dx + X] += np.einsum("oc,ohx->chx", W[:, :, dy, dx], gy)
    return gp[:, 1:-1, 1:-1], gW, gy.sum(axis=(1, 2))


def init_params(seed: int, channels=CHANNELS):
    """He-normal weights, zero biases (float64)."""
    rng = np.random.default_rng(seed)
    params = []
    for l in range(len(channels) - 1):
        ci, co = channels[l], channels[l + 1]
        W = rng.standard_normal((co, ci, 3, 3)) * np.sqrt(2.0 / (9 * ci))
        params.append((W, np.zeros(co)))
    return params


def forward(params, x: np.ndarray):
    """Network output and the per-layer inputs (for the backward pass)."""
    acts = [x]
    a = x
    for l, (W, b) in enumerate(params):
        y = conv3x3(a, W, b)
        a = np.maximum(y, 0.0) if l < len(params) - 1 else y
        acts.append(a)
    return a, acts


def backward(params, acts, gout: np.ndarray):
    """Gradients of sum(gout * net(x)) for every (W, b), from forward's acts."""
    grads = [None] * len(params)
    g = gout
    for l in range(len(params) - 1, -1, -1):
        W, _ = params[l]
        if l < len(params) - 1:
            g = g * (acts[l + 1] > 0.0)        # ReLU: y > 0 exactly where a > 0
        ga, gW, gb = conv3x3_backward(acts[l], W, g)
        grads[l] = (gW, gb)
        g = ga
    return grads


def loss(params, x_hat: np.ndarray, t_hat: np.ndarray):
    """L = mean((net(x_hat) - t_hat)^2) / 2, its gradients, and the output."""
    out, acts = forward(params, x_hat)
    d = out - t_hat
    L = 0.5 * np.mean(d * d)
    grads = backward(params, acts, d / d.size)
    return L, grads, out


# --------------------------------------------------------------- correction --

def normalise(r: np.ndarray, nx: int, ny: int, Nc: int):
    """x_hat = restrict(r) Nc / s with s = ||restrict(r)||."""
    x = restrict(r, nx, ny, Nc)
    s = float(np.linalg.norm(x))
    return (x * (Nc / s) if s > 0 else x), s


def correction(params, r: np.ndarray, nx: int, ny: int, Nc: int, gamma: float) -> np.ndarray:
    """c(r) = prolong(gamma s / Nc net(restrict(r) Nc / s))."""
    x_hat, s = normalise(r, nx, ny, Nc)
    if s == 0.0:
        return np.zeros_like(r)
    out, _ = forward(params, x_hat)
    return prolong(out * (gamma * s / Nc), nx, ny)


def target(e: np.ndarray, s: float, nx: int, ny: int, Nc: int, gamma: float) -> np.ndarray:
    """t_hat = restrict(e) Nc / (gamma s)."""
    return restrict(e, nx, ny, Nc) * (Nc / (gamma * s))
