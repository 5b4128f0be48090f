"""Pins for the oracle of the learned coarse correction (oracle/cnn.py):
the convolution against scipy's 2D correlation, the hand-written backward
pass against central finite differences, and the grid transfers against
what averaging and bilinear interpolation must reproduce."""
import numpy as np
from scipy.signal import correlate2d

from oracle import cnn


def test_conv_matches_scipy_correlation():
    rng = np.random.default_rng(0)
    a = rng.standard_normal((3, 9, 7))
    W = rng.standard_normal((2, 3, 3, 3))
    b = rng.standard_normal(2)
    out = cnn.conv3x3(a, W, b)
    for o in range(2):
        ref = sum(correlate2d(a[c], W[o, c], mode="same", boundary="fill") for c in range(3)) + b[o]
        assert np.allclose(out[o], ref, atol=1e-13)


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(1)
    ch = (2, 4, 4, 2)
    params = cnn.init_params(3, ch)
    params = [(W, rng.standard_normal(W.shape[0]) * 0.1) for W, _ in params]
    x = rng.standard_normal((2, 6, 5))
    t = rng.standard_normal((2, 6, 5))
    L, grads, _ = cnn.loss(params, x, t)
    h = 1e-6
    for l in range(len(params)):
        W, b = params[l]
        for idx in [(0, 0, 0, 0), (1, 1, 2, 1), (W.shape[0] - 1, W.shape[1] - 1, 1, 2)]:
            Wp, Wm = W.copy(), W.copy()
            Wp[idx] += h
            Wm[idx] -= h
            pp = list(params); pp[l] = (Wp, b)
            pm = list(params); pm[l] = (Wm, b)
            fd = (cnn.loss(pp, x, t)[0] - cnn.loss(pm, x, t)[0]) / (2 * h)
            assert abs(fd - grads[l][0][idx]) <= 1e-7 * max(1.0, abs(fd)), (l, idx)
        bp, bm = b.copy(), b.copy()
        bp[0] += h
        bm[0] -= h
        pp = list(params); pp[l] = (W, bp)
        pm = list(params); pm[l] = (W, bm)
        fd = (cnn.loss(pp, x, t)[0] - cnn.loss(pm, x, t)[0]) / (2 * h)
        assert abs(fd - grads[l][1][0]) <= 1e-7 * max(1.0, abs(fd))


def test_relu_layers_and_linearity_in_scale():
    params = cnn.init_params(5)
    rng = np.random.default_rng(2)
    nx, ny, Nc = 40, 33, 8
    r = rng.standard_normal(nx * ny) + 1j * rng.standard_normal(nx * ny)
    c1 = cnn.correction(params, r, nx, ny, Nc, 1.0)
    c2 = cnn.correction(params, 7.5 * r, nx, ny, Nc, 1.0)
    assert np.allclose(c2, 7.5 * c1, rtol=1e-12, atol=0)
    assert np.all(cnn.correction(params, 0 * r, nx, ny, Nc, 1.0) == 0)


def test_restrict_averages_and_prolong_interpolates():
    nx, ny, Nc = 37, 29, 6
    # constants are kept by both transfers
    v = np.full(nx * ny, 2.0 - 3.0j)
    c = cnn.restrict(v, nx, ny, Nc)
    assert np.allclose(c[0], 2.0) and np.allclose(c[1], -3.0)
    assert np.allclose(cnn.prolong(c, nx, ny), v)
    # the mean of a pixel: brute force over its nodes
    rng = np.random.default_rng(4)
    v = rng.standard_normal(nx * ny) + 1j * rng.standard_normal(nx * ny)
    c = cnn.restrict(v, nx, ny, Nc)
    f = v.reshape(ny, nx)
    I, J = 3, 2
    nodes = [(j, i) for j in range(ny) for i in range(nx) if (i * Nc) // nx == I and (j * Nc) // ny == J]
    assert abs(c[0, J, I] - np.mean([f[j, i].real for j, i in nodes])) < 1e-14
    # bilinear: a field linear in the pixel-centre coordinates is reproduced
    # exactly between the outermost centres
    uc = (np.arange(Nc) + 0.5) * nx / Nc - 0.5
    vc = (np.arange(Nc) + 0.5) * ny / Nc - 0.5
    g = 0.3 * uc[None, :] - 1.7 * vc[:, None] + 0.25
    cc = np.stack([g, 2 * g])
    p = cnn.prolong(cc, nx, ny).reshape(ny, nx)
    i = np.arange(nx)
    j = np.arange(ny)
    inside = ((i >= uc[0]) & (i <= uc[-1]))[None, :] & ((j >= vc[0]) & (j <= vc[-1]))[:, None]
    exact = 0.3 * i[None, :] - 1.7 * j[:, None] + 0.25
    assert np.allclose(p.real[inside], exact[inside], atol=1e-12)
    assert np.allclose(p.imag[inside], 2 * exact[inside], atol=1e-12)
