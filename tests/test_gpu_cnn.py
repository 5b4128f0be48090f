"""The learned coarse correction's network on the GPU (tensor-core 3x3
convolutions, BF16 weights and activations, FP32 accumulation) against the
CPU FP64 oracle (oracle/cnn.py): the same network with weights and the
activations between layers rounded to BF16 must agree to FP32 summation
order (2e-3 relative); the plain FP64 network to the size of BF16 rounding
through six layers (5e-2)."""
import numpy as np
import pytest
import torch

from oracle import cnn

pytestmark = pytest.mark.gpu


def bf16(a):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def forward_bf16(params, x):
    a = bf16(x)
    for l, (W, b) in enumerate(params):
        y = cnn.conv3x3(a, bf16(W), np.asarray(b, np.float32).astype(np.float64))
        a = bf16(np.maximum(y, 0.0)) if l < len(params) - 1 else y
    return a


@pytest.fixture(scope="module")
def netcls():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2602_00735_gb300.net import Net, pack
    return Net, pack


def _params(seed):
    rng = np.random.default_rng(seed)
    return [(W, rng.standard_normal(W.shape[0]) * 0.1) for W, _ in cnn.init_params(seed)]


@pytest.mark.parametrize("Nc", [16, 40])
def test_forward_matches_oracle(netcls, Nc):
    Net, pack = netcls
    params = _params(7)
    rng = np.random.default_rng(8)
    x = rng.standard_normal((3, 2, Nc, Nc))
    with Net(Nc=Nc, cap=3) as net:
        net.set_params(pack(params))
        assert np.array_equal(net.get_params(), pack(params))
        y = net.forward(torch.from_numpy(x.astype(np.float32)).cuda()).cpu().numpy().astype(np.float64)
    for i in range(3):
        ref_b = forward_bf16(params, x[i])
        ref = cnn.forward(params, x[i])[0]
        assert np.linalg.norm(y[i] - ref_b) <= 2e-3 * np.linalg.norm(ref_b), i
        assert np.linalg.norm(y[i] - ref) <= 5e-2 * np.linalg.norm(ref), i


def backward_bf16(params, x, t):
    """The oracle's loss gradient through the BF16-rounded forward pass
    (weights and layer inputs rounded as on the GPU)."""
    acts = [bf16(x)]
    a = acts[0]
    for l, (W, b) in enumerate(params):
        y = cnn.conv3x3(a, bf16(W), np.asarray(b, np.float32).astype(np.float64))
        a = bf16(np.maximum(y, 0.0)) if l < len(params) - 1 else y
        acts.append(a)
    d = a - t
    rp = [(bf16(W), b) for W, b in params]
    return 0.5 * np.mean(d * d), cnn.backward(rp, acts, d / d.size)


def test_gradients_match_oracle(netcls):
    """Every layer's weight and bias gradient against the FP64 oracle (two
    images, mean loss): within 3e-2 relative L2 per layer (BF16 gradients
    between layers), and the loss to 1e-3."""
    Net, pack = netcls
    from paper_2602_00735_gb300.net import unpack
    Nc = 24
    params = _params(11)
    rng = np.random.default_rng(12)
    x = rng.standard_normal((2, 2, Nc, Nc))
    t = rng.standard_normal((2, 2, Nc, Nc))
    with Net(Nc=Nc, cap=2) as net:
        net.set_params(pack(params))
        L, g = net.loss_grad(torch.from_numpy(x.astype(np.float32)).cuda(),
                             torch.from_numpy(t.astype(np.float32)).cuda())
    gg = unpack(g)
    Lo = 0.0
    go = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
    for i in range(2):
        li, gi = backward_bf16(params, x[i], t[i])
        Lo += li / 2
        go = [(a[0] + b[0] / 2, a[1] + b[1] / 2) for a, b in zip(go, gi)]
    assert abs(L - Lo) <= 1e-3 * Lo
    for l, ((gW, gb), (oW, ob)) in enumerate(zip(gg, go)):
        assert np.linalg.norm(gW - oW) <= 3e-2 * np.linalg.norm(oW), l
        assert np.linalg.norm(gb - ob) <= 3e-2 * np.linalg.norm(ob), l


def test_training_steps_reduce_the_loss(netcls):
    Net, pack = netcls
    Nc = 32
    rng = np.random.default_rng(13)
    x = rng.standard_normal((4, 2, Nc, Nc)).astype(np.float32)
    t = (0.5 * x + 0.1 * np.roll(x, 1, axis=3)).astype(np.float32)   # a learnable linear map
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    with Net(Nc=Nc, cap=4, seed=3) as net:
        L0, _ = net.loss_grad(xd, td, want_grad=False)
        for _ in range(60):
            net.loss_grad(xd, td, want_grad=False)
            net.adam_step(2e-3)
        L1, _ = net.loss_grad(xd, td, want_grad=False)
    assert L1 < 0.2 * L0
