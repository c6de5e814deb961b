"""Launch shapes of the trajectory kernels that the autotuner searches: the sphere tiling
(strided or blocked assignment of a configuration's spheres to lanes) and the particles per
CTA (one, or two on separate warp groups and shared-memory regions).  Every shape passes the
per-evaluation parity with the FP64 oracle at 1e-4 and the one-step descent parity on every
particle; two particles per CTA give the same bits as one; the batched form under each shape
gives the same bits as single solves with that shape; the autotuner returns a valid shape."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2510_07674_gb300 import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

RTOL, ATOL = 1e-4, 2e-6
SHAPES = [(0, 1), (1, 1), (0, 2), (1, 2)]


def _S():
    from paper_2510_07674_gb300 import spasm as S
    return S


def _case(seed=1, n=6, sigma=0.15, **kw):
    wl = scenes.make_problem("tower4", seed=seed, B=3, O=12, W=8, **kw)
    orc = O.Oracle(wl, n_threads=8)
    sol, _, _ = orc.place_solve()
    rng = np.random.default_rng(seed)
    qs = []
    for p in range(n):
        q = orc.lift(sol[p % len(sol)], p)
        q[1:] += rng.normal(0, sigma, q[1:].shape)
        qs.append(np.clip(q, wl.robot.qlim[:, 0], wl.robot.qlim[:, 1]))
    return wl, orc, qs


def _eval(S, pr, qs, lam_np, mu_np):
    n, C, NR = len(qs), pr.C, pr.NR
    q = torch.zeros(n, C, 8, device="cuda")
    q[:, :, :7] = torch.from_numpy(np.asarray(qs)).float()
    lam, mu = torch.from_numpy(lam_np).cuda(), torch.from_numpy(mu_np).cuda()
    L, grad = torch.empty(n, device="cuda"), torch.empty(n, C, 8, device="cuda")
    groups, h = torch.empty(n, 6, device="cuda"), torch.empty(n, NR, device="cuda")
    S.spasm_traj_eval(pr, n, q, lam, mu, L, grad, groups, h)
    torch.cuda.synchronize()
    return q, L.cpu().numpy(), grad.cpu().numpy(), groups.cpu().numpy(), h.cpu().numpy()


@pytest.mark.parametrize("tiling,ppc", SHAPES)
def test_shape_eval_and_one_step_match_oracle(tiling, ppc):
    S = _S()
    wl, orc, qs = _case()
    pr = S.Problem(wl)
    try:
        S.spasm_set_kernel_config(pr, tiling, ppc)
        n, NR = len(qs), pr.NR
        rng = np.random.default_rng(9)
        lam_np = rng.uniform(0, 2, (n, NR)).astype(np.float32)
        mu_np = rng.uniform(0.5, 4, n).astype(np.float32)
        q, L, g, groups, h = _eval(S, pr, qs, lam_np, mu_np)
        for p in range(n):
            qp = q[p, :, :7].cpu().double().numpy()
            Lo, go, cgo, _, _, ho = orc.traj_cost(qp, lam_np[p].astype(np.float64), float(mu_np[p]))
            assert abs(L[p] - Lo) <= RTOL * max(abs(Lo), 1e-2), (p, L[p], Lo)
            np.testing.assert_allclose(groups[p], cgo, rtol=RTOL, atol=ATOL)
            np.testing.assert_allclose(h[p], ho, rtol=RTOL, atol=ATOL)
            assert np.linalg.norm(g[p, :, :7] - go) / max(np.linalg.norm(go), 1e-2) <= RTOL
        # one descent step (K = 2: eta/2, then 0) on every particle
        q0 = np.stack([q[p, :, :7].cpu().double().numpy() for p in range(n)])
        lam0, mu0 = torch.zeros(n, NR, device="cuda"), torch.full((n,), float(wl.params.mu0), device="cuda")
        S.spasm_traj_descend(pr, n, q, lam0, mu0, 2, 1)
        torch.cuda.synchronize()
        qr, _, _ = orc.traj_descend(q0, k_steps=2)
        for p in range(n):
            step_g, step_o = q[p, :, :7].cpu().double().numpy() - q0[p], qr[p] - q0[p]
            assert np.abs(step_g - step_o).max() <= RTOL * np.abs(step_o).max() + 1e-6, p
    finally:
        pr.close()


@pytest.mark.parametrize("tiling", [0, 1])
def test_two_particles_per_cta_give_the_same_bits(tiling):
    S = _S()
    wl, _, qs = _case(seed=2, n=7)   # odd: the last CTA's second group has no particle
    n, out = len(qs), []
    for ppc in (1, 2):
        pr = S.Problem(wl)
        try:
            S.spasm_set_kernel_config(pr, tiling, ppc)
            rng = np.random.default_rng(3)
            lam_np = rng.uniform(0, 2, (n, pr.NR)).astype(np.float32)
            mu_np = rng.uniform(0.5, 4, n).astype(np.float32)
            _, L, g, groups, h = _eval(S, pr, qs, lam_np, mu_np)
            S.spasm_optimize(pr)
            r = S.spasm_result(pr)
            out.append((L, g, groups, h, r["traj"], r["cost"]))
        finally:
            pr.close()
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("tiling,ppc", SHAPES)
def test_batched_shape_equals_single_solves_with_that_shape(tiling, ppc):
    S = _S()
    wls = [scenes.make_problem("tower4", seed=s, B=b, O=o, W=8, Q=q, N=1024, M=256)
           for s, (b, o, q) in enumerate([(2, 6, 300), (3, 12, 517), (4, 20, 256)])]
    alone = []
    for wl in wls:
        pr = S.Problem(wl)
        S.spasm_set_kernel_config(pr, tiling, ppc)
        S.spasm_optimize(pr)
        alone.append(S.spasm_result(pr, allow_empty=True))
        pr.close()
    stream = torch.cuda.Stream()
    prs = [S.Problem(wl, stream=stream.cuda_stream) for wl in wls]
    try:
        S.spasm_optimize_batch(prs, stream=stream.cuda_stream,
                               config={"per_fetch": 2, "sphere_tiling": tiling, "particles_per_cta": ppc})
        for a, p in zip(alone, prs):
            r = S.spasm_result(p, allow_empty=True)
            assert r["n_found"] == a["n_found"]
            for key in ("traj", "cost", "success"):
                assert np.array_equal(np.asarray(r[key]), np.asarray(a[key])), key
    finally:
        for p in prs:
            p.close()


def test_autotuner_returns_a_valid_shape_and_two_particles_fit_tower10():
    S = _S()
    stream = torch.cuda.Stream()
    wls = [scenes.make_problem("tower4", seed=s, B=3, O=12, W=8, Q=512, N=1024, M=256) for s in range(3)]
    prs = [S.Problem(wl, stream=stream.cuda_stream) for wl in wls]
    try:
        best = S.spasm_batch_autotune(prs, stream=stream.cuda_stream)
        assert best["sphere_tiling"] in (0, 1) and best["particles_per_cta"] in (1, 2) and best["ms"] > 0
    finally:
        for p in prs:
            p.close()
    # the 10-block workload: two particles per CTA still fit one SM's shared memory
    wl = scenes.make_problem("tower10", seed=0, Q=64)
    pr = S.Problem(wl)
    try:
        S.spasm_set_kernel_config(pr, 0, 2)
        S.spasm_optimize(pr)
        assert S.spasm_result(pr, allow_empty=True)["n_found"] > 0
    finally:
        pr.close()


def test_the_largest_workload_keeps_two_ctas_per_sm():
    """The shared-memory budget: the 10-block workload (the largest of the benchmark's mixes)
    runs two CTAs per SM in the per-problem and in the batched kernel (one particle per CTA),
    and two particles per CTA still fit one SM."""
    S = _S()
    wl = scenes.make_problem("tower10", seed=0, Q=64)
    pr = S.Problem(wl)
    try:
        assert S.spasm_traj_residency(pr) == {"single": 2, "batched": 2}
        S.spasm_set_kernel_config(pr, 0, 2)
        r = S.spasm_traj_residency(pr)
        assert r["single"] >= 1 and r["batched"] >= 1, r
    finally:
        pr.close()
