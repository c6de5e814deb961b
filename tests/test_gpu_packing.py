"""Packing goal (the appendix's Tetris problem), stage 1: CUDA path vs the FP64 oracle on
identical inputs (1e-4 relative for costs, norm-wise relative for gradients), and the end
to end stage-1 solve returning packings that pass the oracle's check."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2510_07674_gb300 import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

RTOL = 1e-4


def _S():
    from paper_2510_07674_gb300 import spasm as S
    return S


def _soa(x, B):
    return x.detach().cpu().double().numpy().T.reshape(-1, B, 4)


def _dev(xp):
    n, B = xp.shape[0], xp.shape[1]
    return torch.from_numpy(xp.reshape(n, 4 * B).T.copy()).float().cuda().contiguous()


@pytest.mark.parametrize("name,n", [("tetris5", 77), ("tetris8", 141)])
def test_sample_and_cost_match_oracle(name, n):
    S = _S()
    wl = scenes.make_packing(name, seed=1)
    orc = O.Oracle(wl)
    pr = S.Problem(wl)
    x = torch.empty(4 * pr.B, n, device="cuda")
    cost = torch.empty(n, device="cuda")
    S.spasm_place_sample(pr, n, 2, x, cost)
    torch.cuda.synchronize()
    xs = _soa(x, pr.B)
    np.testing.assert_allclose(xs, orc.place_sample(n, attempt=2), rtol=0, atol=2e-6)
    for p in range(n):
        c = orc.place_cost(xs[p], grad=False)[0]
        assert abs(cost[p].item() - c) <= RTOL * max(abs(c), 1e-2), (p, cost[p].item(), c)


@pytest.mark.parametrize("quad", [0, 1])
@pytest.mark.parametrize("name,zspan", [("tetris5", 0.0), ("tetris8", 0.0), ("tetris5", 0.03)])
def test_eval_cost_grad_terms_metrics_match_oracle(name, zspan, quad):
    S = _S()
    wl = scenes.make_packing(name, seed=2, zspan=zspan, w_height=3.0)
    orc = O.Oracle(wl)
    pr = S.Problem(wl)
    B = pr.B
    rng = np.random.default_rng(0)
    # near the planted tiling (many light contacts) and uniform samples (deep overlaps)
    near = np.repeat(wl.packing.planted[None], 96, 0)
    near[:, :, :2] += rng.normal(0, 0.004, (96, B, 2))
    near[:, :, 2] += rng.uniform(0, zspan, (96, B))
    near[:, :, 3] += rng.normal(0, 0.04, (96, B))
    xp = np.concatenate([near, orc.place_sample(64)])
    n = len(xp)
    x = _dev(xp)
    cost, grad = torch.empty(n, device="cuda"), torch.empty_like(x)
    metrics, terms = torch.empty(n, 3, device="cuda"), torch.empty(n, 3, device="cuda")
    S.spasm_place_eval(pr, n, x, quad, cost, grad, metrics, terms)
    torch.cuda.synchronize()
    xs, gs = _soa(x, B), _soa(grad, B)
    worst = 0.0
    for p in range(n):
        c, g, t = orc.place_cost(xs[p], quad=bool(quad))
        ok, m = orc.place_check(xs[p])
        assert abs(cost[p].item() - c) <= RTOL * max(abs(c), 1e-2), (p, cost[p].item(), c)
        # at |z - z*| = 0 (the one-layer box) the sign of the height term is decided by the
        # representation of z* (float32 on the GPU, double in the oracle): compare the
        # remaining components there
        keep = np.ones_like(g, dtype=bool)
        keep[np.abs(xs[p][:, 2] - wl.packing.z_star) < 1e-6, 2] = False
        worst = max(worst, np.linalg.norm((gs[p] - g)[keep]) / max(np.linalg.norm(g[keep]), 1e-2))
        np.testing.assert_allclose(terms[p].cpu().double().numpy(), t, rtol=RTOL, atol=1e-7)
        if not quad:
            np.testing.assert_allclose(metrics[p].cpu().double().numpy(), m, rtol=RTOL, atol=1e-6)
    assert worst <= RTOL, worst


def test_planted_tiling_is_satisfying_on_the_gpu():
    S = _S()
    for name in ("tetris5", "tetris8"):
        wl = scenes.make_packing(name, seed=3)
        pr = S.Problem(wl)
        x = _dev(wl.packing.planted[None])
        cost, metrics = torch.empty(1, device="cuda"), torch.empty(1, 3, device="cuda")
        S.spasm_place_eval(pr, 1, x, 0, cost, None, metrics, None)
        torch.cuda.synchronize()
        assert cost.item() < 1e-5 and metrics.max().item() < 1e-6


def test_descend_few_steps_matches_oracle():
    S = _S()
    wl = scenes.make_packing("tetris5", seed=5)
    orc = O.Oracle(wl)
    pr = S.Problem(wl)
    n, B = 64, pr.B
    x = _dev(orc.place_sample(n))
    x0 = _soa(x, B)
    S.spasm_place_descend(pr, n, x, 3, 2)
    torch.cuda.synchronize()
    err = np.abs(_soa(x, B) - orc.place_descend(x0, 3, 2)).max(axis=(1, 2))
    # identical float32 states: differences stay at rounding level except where a contact
    # switches on or off between the two precisions (rare)
    assert np.mean(err < 1e-4) >= 0.9, np.sort(err)[-10:]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_stage1_solve_returns_packings_that_pass_the_oracle_check(seed):
    """Alg. 1 end to end on the 5-block packing: a solution is found and every returned
    packing satisfies the FP64 check (every penetration and height error within eps)."""
    S = _S()
    wl = scenes.make_packing("tetris5", seed=seed)
    pr = S.Problem(wl)
    S.spasm_place(pr)
    r = S.spasm_placements(pr)
    assert r["n_place"] >= 1
    relaxed = O.Oracle(wl, eps=wl.params.eps * 1.01)
    for x in r["placements"]:
        ok, m = relaxed.place_check(x)
        assert ok, m
    with pytest.raises(S.SpasmError):
        S.spasm_optimize(pr)   # stage 2 is built for the tower goal
