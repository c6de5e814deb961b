"""autograd.Function wrappers: gradients equal the FP64 oracle's and central differences."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2510_07674_gb300 import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_traj_cost_autograd_matches_oracle_and_fd():
    from paper_2510_07674_gb300 import autograd as A
    from paper_2510_07674_gb300 import spasm as S
    wl = scenes.make_problem("tower4", seed=1, B=2, O=10, W=8)
    orc = O.Oracle(wl)
    sol, _, _ = orc.place_solve()
    rng = np.random.default_rng(0)
    qs = []
    for p in range(4):
        q = orc.lift(sol[p % len(sol)], p)
        q[1:] += rng.normal(0, 0.1, q[1:].shape)
        qs.append(np.clip(q, wl.robot.qlim[:, 0], wl.robot.qlim[:, 1]))
    pr = S.Problem(wl)
    q = torch.tensor(np.stack(qs), dtype=torch.float32, device="cuda", requires_grad=True)
    weights = torch.tensor([1.0, -0.5, 2.0, 0.25], device="cuda")
    L = A.traj_cost(pr, q)
    (L * weights).sum().backward()
    g = q.grad.detach().cpu().double().numpy()
    for p in range(4):
        _, go, *_ = orc.traj_cost(q[p].detach().cpu().double().numpy())
        go = go * float(weights[p])
        assert np.linalg.norm(g[p] - go) <= 1e-4 * max(np.linalg.norm(go), 1e-2)
    # directional central difference of the autograd function itself (FP32, h = 1e-3)
    gen = torch.Generator(device="cuda").manual_seed(7)   # fixed direction: the check is reproducible
    d = torch.randn(q.shape, generator=gen, device="cuda") * 0.1
    d[:, 0] = 0
    h = 1e-3
    with torch.no_grad():
        fd = ((A.traj_cost(pr, q + h * d) - A.traj_cost(pr, q - h * d)) / (2 * h)).cpu().double().numpy()
    an = (q.grad.detach() / weights[:, None, None] * d).sum((1, 2)).cpu().double().numpy()
    np.testing.assert_allclose(an, fd, rtol=2e-2, atol=1e-3)


def test_place_cost_autograd_matches_oracle():
    from paper_2510_07674_gb300 import autograd as A
    from paper_2510_07674_gb300 import spasm as S
    wl = scenes.make_problem("tower4", seed=2)
    orc = O.Oracle(wl)
    pr = S.Problem(wl)
    n, B = 37, pr.B
    xo = orc.place_sample(n)
    xo[:, :, :2] = 0.5 * xo[:, :, :2] + 0.5 * xo[:, :, :2].mean(1, keepdims=True)
    x = torch.tensor(xo.reshape(n, 4 * B).T.copy(), dtype=torch.float32, device="cuda", requires_grad=True)
    for quad in (False, True):
        x.grad = None
        A.place_cost(pr, x, quad).sum().backward()
        g = x.grad.detach().cpu().double().numpy().T.reshape(n, B, 4)
        xs = x.detach().cpu().double().numpy().T.reshape(n, B, 4)
        for p in range(n):
            _, go, _ = orc.place_cost(xs[p], quad=quad)
            assert np.linalg.norm(g[p] - go) <= 1e-4 * max(np.linalg.norm(go), 1e-2)
