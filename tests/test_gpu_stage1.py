"""Stage-1 parity: CUDA path vs the FP64 oracle on identical inputs (tolerance 1e-4
relative for costs, norm-wise relative for gradients; bit-exact for selection)."""
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


def _soa_to_particles(x, B):
    return x.detach().cpu().double().numpy().T.reshape(-1, B, 4)


# the last case is the largest problem the kernels take (16 blocks, 256 cuboids, 64 spheres)
MAXIMA = {"B": 16, "O": 255, "n_obstacle_spheres": 64}


@pytest.mark.parametrize("name,n,kw", [("tower1", 77, {}), ("tower4", 333, {}), ("tower10", 141, {}),
                                       ("tower10", 65, MAXIMA)])
def test_sample_and_cost_match_oracle(name, n, kw):
    S = _S()
    wl = scenes.make_problem(name, seed=1, **kw)
    orc = O.Oracle(wl)
    pr = S.Problem(wl)
    x = torch.empty(4 * pr.B, n, device="cuda")
    cost = torch.empty(n, device="cuda")
    S.spasm_place_sample(pr, n, 3, x, cost)
    torch.cuda.synchronize()
    xs = _soa_to_particles(x, pr.B)
    xo = orc.place_sample(n, attempt=3)
    np.testing.assert_allclose(xs, xo, rtol=0, atol=2e-6)
    for p in range(n):
        c = orc.place_cost(xs[p], grad=False)[0]
        assert abs(cost[p].item() - c) <= RTOL * max(abs(c), 1e-2), (p, cost[p].item(), c)


@pytest.mark.parametrize("quad", [0, 1])
@pytest.mark.parametrize("name,kw", [("tower4", {}), ("tower10", {}), ("tower10", MAXIMA)])
def test_eval_cost_grad_terms_match_oracle(name, kw, quad):
    S = _S()
    wl = scenes.make_problem(name, seed=2, **kw)
    orc = O.Oracle(wl)
    pr = S.Problem(wl)
    n, B = 203, pr.B
    rng = np.random.default_rng(0)
    xp = orc.place_sample(n)
    # pull the blocks together so that stability and block-block terms are active
    xp[:, :, :2] = 0.4 * xp[:, :, :2] + 0.6 * xp[:, :, :2].mean(1, keepdims=True) + rng.normal(0, 0.01, (n, B, 2))
    x = torch.from_numpy(xp.reshape(n, 4 * B).T.copy()).float().cuda().contiguous()
    cost, grad = torch.empty(n, device="cuda"), torch.empty_like(x)
    metrics, terms = torch.empty(n, 3, device="cuda"), torch.empty(n, 3, device="cuda")
    S.spasm_place_eval(pr, n, x, quad, cost, grad, metrics, terms)
    torch.cuda.synchronize()
    xs = _soa_to_particles(x, B)
    gs = _soa_to_particles(grad, B)
    worst = 0.0
    for p in range(n):
        c, g, t = orc.place_cost(xs[p], quad=bool(quad))
        ok, m = orc.place_check(xs[p])
        assert abs(cost[p].item() - c) <= RTOL * max(abs(c), 1e-2)
        err = np.linalg.norm(gs[p] - g) / max(np.linalg.norm(g), 1e-2)
        worst = max(worst, err)
        np.testing.assert_allclose(terms[p].cpu().double().numpy(), t, rtol=RTOL, atol=1e-7)
        if not quad:
            np.testing.assert_allclose(metrics[p].cpu().double().numpy(), m, rtol=RTOL, atol=1e-6)
    assert worst <= RTOL, worst


def test_topk_bit_exact_vs_stable_argsort():
    S = _S()
    wl = scenes.make_problem("tower1", seed=0)
    pr = S.Problem(wl)
    rng = np.random.default_rng(3)
    for n, k in [(1, 1), (100, 7), (4096, 1024), (16384, 4096), (20000, 8192), (5000, 5000)]:
        c = rng.integers(0, 50, n).astype(np.float32) * 0.25   # many ties
        c[rng.integers(0, n, n // 50)] = np.nan
        c[rng.integers(0, n, n // 50)] = -0.0
        cost = torch.from_numpy(c).cuda()
        idx = torch.empty(k, dtype=torch.int32, device="cuda")
        S.spasm_select_topk(pr, n, cost, k, idx)
        torch.cuda.synchronize()
        ref = O.argsort(c.astype(np.float64))[:k]
        np.testing.assert_array_equal(idx.cpu().numpy(), ref)


@pytest.mark.parametrize("name,k_lin,k_quad", [("tower4", 2, 0), ("tower4", 1, 1), ("tower10", 2, 0)])
def test_descend_one_step_matches_oracle_on_every_particle(name, k_lin, k_quad):
    """One step of Alg. 1 from identical states, element-wise on every particle: K_lin = 2
    gives the linear-form steps eta_init (1 - 1/2) and 0; K_lin = 1, K_quad = 1 gives a zero
    linear step (only the box projection) and one quadratic-form step with alpha.  The step
    agrees with the oracle's to 1e-4 of its size (the gradient's FP32 rounding) plus the
    float32 rounding of the pose values."""
    S = _S()
    wl = scenes.make_problem(name, seed=5)
    orc = O.Oracle(wl, n_threads=8)
    pr = S.Problem(wl)
    n, B = 256, pr.B
    xo = orc.place_sample(n)
    x = torch.from_numpy(xo.reshape(n, 4 * B).T.copy()).float().cuda().contiguous()
    x0 = _soa_to_particles(x, B)
    S.spasm_place_descend(pr, n, x, k_lin, k_quad)
    torch.cuda.synchronize()
    xg = _soa_to_particles(x, B)
    xr = orc.place_descend(x0, k_lin, k_quad)
    moved = 0
    for p in range(n):
        step_g, step_o = xg[p] - x0[p], xr[p] - x0[p]
        err = np.abs(step_g - step_o).max()
        assert err <= RTOL * np.abs(step_o).max() + 1e-6, (p, err, np.abs(step_o).max())
        moved += np.abs(step_o).max() > 1e-4
    assert moved > n // 2


@pytest.mark.parametrize("name", ["tower1", "tower4"])
def test_full_descent_satisfying_rate_matches_oracle(name):
    """End to end Alg. 1 descent from the same samples: the satisfying fraction of the GPU
    and of the oracle agree within a binomial tolerance, and every GPU particle flagged
    satisfying passes the FP64 check."""
    S = _S()
    wl = scenes.make_problem(name, seed=7)
    orc = O.Oracle(wl, n_threads=8)
    pr = S.Problem(wl)
    n, B = 512, pr.B
    xo = orc.place_sample(n)
    x = torch.from_numpy(xo.reshape(n, 4 * B).T.copy()).float().cuda().contiguous()
    x0 = _soa_to_particles(x, B)
    sat = torch.empty(n, dtype=torch.int32, device="cuda")
    S.spasm_place_descend(pr, n, x, wl.params.K_lin, wl.params.K_quad, None, sat)
    torch.cuda.synchronize()
    xg = _soa_to_particles(x, B)
    xr = orc.place_descend(x0)
    s_gpu = sat.cpu().numpy().astype(bool)
    s_orc = np.array([orc.place_check(v)[0] for v in xr])
    f1, f2 = s_gpu.mean(), s_orc.mean()
    tol = 4 * np.sqrt(max(f2 * (1 - f2), 1.0 / n) / n) + 0.02
    assert abs(f1 - f2) <= tol, (f1, f2)
    relaxed = O.Oracle(wl, eps=wl.params.eps * 1.01)
    assert all(relaxed.place_check(v)[0] for v in xg[s_gpu])


def test_place_end_to_end_returns_satisfying():
    S = _S()
    wl = scenes.make_problem("tower4", seed=0)
    pr = S.Problem(wl)
    S.spasm_place(pr)
    res = S.spasm_result(pr, allow_empty=True)
    place = res["placements"]
    relaxed = O.Oracle(wl, eps=wl.params.eps * 1.01)
    assert all(relaxed.place_check(p)[0] for p in place)


def test_full_size_tower10_sampled_rows():
    """At the full 10-block size (N = 16384) compare sampled particles one by one."""
    S = _S()
    wl = scenes.make_problem("tower10", seed=0)
    orc = O.Oracle(wl)
    pr = S.Problem(wl)
    N, B = wl.params.N, pr.B
    x = torch.empty(4 * B, N, device="cuda")
    cost = torch.empty(N, device="cuda")
    S.spasm_place_sample(pr, N, 0, x, cost)
    torch.cuda.synchronize()
    rows = np.random.default_rng(0).choice(N, 64, replace=False)
    xs = _soa_to_particles(x, B)
    xo = orc.place_sample(N)
    for p in rows:
        np.testing.assert_allclose(xs[p], xo[p], atol=2e-6)
        c = orc.place_cost(xs[p], grad=False)[0]
        assert abs(cost[p].item() - c) <= RTOL * max(abs(c), 1e-2)
