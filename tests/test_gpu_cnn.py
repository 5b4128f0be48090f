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
