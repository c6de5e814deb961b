"""Point-to-point trajectory optimisation (one transit segment to a tool target): CUDA path
vs the FP64 oracle on identical inputs, and the end-to-end solve."""
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


def _to_dev(qs, C):
    q = torch.zeros(len(qs), C, 8, device="cuda")
    q[:, :, :7] = torch.from_numpy(np.asarray(qs)).float()
    return q


@pytest.mark.parametrize("seed,W,sigma", [(0, 32, 0.0), (1, 16, 0.08), (2, 32, 0.15)])
def test_traj_eval_matches_oracle(seed, W, sigma):
    S = _S()
    wl = scenes.make_p2p("p2p", seed=seed, W=W)
    orc = O.Oracle(wl)
    pr = S.Problem(wl)
    assert pr.C == W
    rng = np.random.default_rng(seed)
    n = 7
    qs = []
    for p in range(n):
        q = orc.lift(np.zeros((1, 4)), p)
        q[1:] += rng.normal(0, sigma, q[1:].shape)
        qs.append(np.clip(q, wl.robot.qlim[:, 0], wl.robot.qlim[:, 1]))
    q = _to_dev(qs, pr.C)
    lam_np = rng.uniform(0, 2, (n, pr.NR)).astype(np.float32)
    mu_np = rng.uniform(0.5, 4, n).astype(np.float32)
    lam, mu = torch.from_numpy(lam_np).cuda(), torch.from_numpy(mu_np).cuda()
    L, grad = torch.empty(n, device="cuda"), torch.empty(n, pr.C, 8, device="cuda")
    groups, h = torch.empty(n, 6, device="cuda"), torch.empty(n, pr.NR, device="cuda")
    S.spasm_traj_eval(pr, n, q, lam, mu, L, grad, groups, h)
    torch.cuda.synchronize()
    active = 0
    for p in range(n):
        qp = q[p, :, :7].cpu().double().numpy()
        Lo, go, cgo, path, jl, ho = orc.traj_cost(qp, lam_np[p].astype(np.float64), float(mu_np[p]))
        active += cgo[1] > 0
        assert abs(L[p].item() - Lo) <= RTOL * max(abs(Lo), 1e-2), (p, L[p].item(), Lo)
        np.testing.assert_allclose(groups[p].cpu().double().numpy(), cgo, rtol=1e-3, atol=1e-6)
        np.testing.assert_allclose(h[p].cpu().double().numpy(), ho, rtol=1e-3, atol=1e-5)
        gd = grad[p, :, :7].cpu().double().numpy()
        assert np.linalg.norm(gd - go) / max(np.linalg.norm(go), 1e-2) <= RTOL
    assert active > 0


def test_lift_and_descent_match_oracle():
    S = _S()
    wl = scenes.make_p2p("p2p", seed=3, W=16)
    orc = O.Oracle(wl)
    pr = S.Problem(wl)
    n = 12
    place = torch.zeros(1, 4, device="cuda")
    q = torch.zeros(n, pr.C, 8, device="cuda")
    S.spasm_lift(pr, n, place, 1, 0, q)
    torch.cuda.synchronize()
    matched = converged = 0
    for p in range(n):
        qo = orc.lift(np.zeros((1, 4)), p)
        qg = q[p, :, :7].cpu().double().numpy()
        np.testing.assert_array_equal(qg[0], np.float32(wl.robot.q_home))
        _, T = orc.fk(qo[-1])
        if np.linalg.norm(T[:3, 3] - wl.scene.init[0][:3]) < 1e-6:
            converged += 1
            matched += np.abs(qg[-1] - qo[-1]).max() < 2e-3
    assert converged >= n // 3 and matched >= 0.9 * converged, (matched, converged)
    # a few descent steps from the GPU's lifted state
    q0 = np.stack([q[p, :, :7].cpu().double().numpy() for p in range(n)])
    lam = torch.zeros(n, pr.NR, device="cuda")
    mu = torch.full((n,), float(wl.params.mu0), device="cuda")
    S.spasm_traj_descend(pr, n, q, lam, mu, 4, 1)
    torch.cuda.synchronize()
    qr, _, _ = orc.traj_descend(q0, k_steps=4)
    err = np.array([np.abs(q[p, :, :7].cpu().double().numpy() - qr[p]).max() for p in range(n)])
    assert np.mean(err < 1e-4) >= 0.9, np.sort(err)[-4:]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_optimize_end_to_end_returns_collision_free_paths(seed):
    """The lifted paths collide (half the clutter sits between robot and target); every
    returned trajectory passes the FP64 oracle check (no penetration above eps, target
    aligned within eps_start, limits respected)."""
    S = _S()
    wl = scenes.make_p2p("p2p", seed=seed)
    orc = O.Oracle(wl, eps=wl.params.eps * 1.05, eps_start=wl.params.eps_start * 1.05)
    pr = S.Problem(wl)
    with pytest.raises(S.SpasmError):
        S.spasm_place(pr)   # no stage 1
    S.spasm_optimize(pr)
    res = S.spasm_result(pr)
    assert res["n_found"] >= 1 and res["traj"].shape[1] == wl.params.W
    for q in res["traj"]:
        ok, m = orc.traj_check(q)
        assert ok, m


def test_batched_form_equals_single_for_p2p():
    S = _S()
    wls = [scenes.make_p2p("p2p", seed=s, Q=300 + 77 * s, W=16 + 8 * s) for s in range(3)]
    alone = []
    for wl in wls:
        pr = S.Problem(wl)
        S.spasm_optimize(pr)
        alone.append(S.spasm_result(pr, allow_empty=True))
        pr.close()
    stream = torch.cuda.Stream()
    prs = [S.Problem(wl) for wl in wls]
    S.spasm_optimize_batch(prs, stream=stream.cuda_stream)
    for a, p in zip(alone, prs):
        b = S.spasm_result(p, allow_empty=True)
        assert a["n_found"] == b["n_found"]
        np.testing.assert_array_equal(a["traj"], b["traj"])
        np.testing.assert_array_equal(a["cost"], b["cost"])
        p.close()
