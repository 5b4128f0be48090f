"""The learned coarse correction as an FGMRES stage: the correction c(r)
against the oracle (oracle/cnn.py, with BF16 rounding emulated), training on
pairs the method generates, and solves with the stage attached against the
direct solve. The stage is gated (it stops after 4 directions that each
removed less than 5% of their residual's squared norm), so the test checks
the gate against the gain the stage itself records, and that the stage never
costs iterations: the iteration counts with and without it are printed (the
paper has no such stage)."""
import numpy as np
import pytest
import torch

from gpu_util import oracle_problem, rel, random_vector, to_dev, variant
from oracle import cnn, fem
from test_gpu_cnn import forward_bf16

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2602_00735_gb300 as p
    from paper_2602_00735_gb300 import net
    return p, net


def test_correction_matches_oracle(pkg):
    p, netmod = pkg
    w = variant("small")
    grid, A, _ = oracle_problem(w)
    nx, ny, Nc = grid.nx, grid.ny, 32
    rng = np.random.default_rng(21)
    params = [(W, rng.standard_normal(W.shape[0]) * 0.1) for W, _ in cnn.init_params(21)]
    r = random_vector(grid.n, 22)
    with p.RasPml(w.params(), factor_prec=1) as s, netmod.Net(Nc=Nc, cap=1) as net:
        net.set_params(netmod.pack(params))
        net.gamma = 0.7
        z = s.net_correct(net, to_dev(r), torch.zeros(grid.n, dtype=torch.complex128, device="cuda")).cpu().numpy()
    x_hat, sn = cnn.normalise(r, nx, ny, Nc)
    out = forward_bf16(params, x_hat.astype(np.float32))
    ref_b = cnn.prolong(out * (0.7 * sn / Nc), nx, ny)
    ref = cnn.correction(params, r, nx, ny, Nc, 0.7)
    assert rel(z, ref_b) <= 3e-3
    assert rel(z, ref) <= 5e-2


@pytest.mark.parametrize("name,Nc", [("small", 16), ("c0", 64)])
def test_trained_stage_solves_to_the_direct_solution(pkg, name, Nc):
    p, netmod = pkg
    w = variant(name)
    prm = w.params()
    grid, A, _ = oracle_problem(w)
    u = fem.direct_solve(A, fem.assemble_rhs(prm, w.centres, w.amps, w.width))
    with p.RasPml(prm, factor_prec=1, ortho=3) as s, netmod.Net(Nc=Nc, cap=8, seed=1) as net:
        b = s.assemble_rhs(w.centres, w.amps, w.width)
        _, it0, _, st0 = s.solve(b, rtol=1e-8, maxit=400)
        hist, gamma = net.train(s, nrhs=3, m_list=(1, 2, 3, 4, 6, 8), epochs=80, lr=1e-3, seed=5)
        assert np.all(np.isfinite(hist)) and hist[-1] < hist[0] and gamma > 0
        s.attach_net(net)
        x, it1, relres, st1 = s.solve(b, rtol=1e-8, maxit=400)
        tm = s.timing()
        s.attach_net(None)
        assert st0 == 0 and st1 == 0 and relres <= 1e-8
        assert rel(x.cpu().numpy(), u) <= 1e-6
    dirs, gain = tm["learned_dirs"], tm["learned_gain"]
    assert 1 <= dirs <= it1 and 0.0 <= gain <= 1.0
    if gain < 0.05:
        # the gate closes after 4 such directions, seen one batch of four
        # late: at most 8 directions corrected
        assert dirs <= 8 or dirs == it1
    # the stage's minimal-residual step never enlarges a residual, and a
    # closed gate restores the plain method: never more iterations
    assert it1 <= it0 + 1
    print(f"\n{name}: iterations plain {it0}, with the learned stage {it1}; stage on {dirs} directions, "
          f"largest gain {gain:.3g}; loss {hist[0]:.3g} -> {hist[-1]:.3g}")
