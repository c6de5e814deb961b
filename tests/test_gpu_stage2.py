"""Stage-2 parity: lift, trajectory objective/gradient/residuals and descent of the CUDA
path vs the FP64 oracle on identical inputs."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2510_07674_gb300 import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

RTOL = 1e-4
# absolute floor for residuals and group sums that are zero on one side: float32 kinematics
# place a point to ~1e-7 m, and the residuals are differences of such positions and angles
ATOL = 2e-6


def _S():
    from paper_2510_07674_gb300 import spasm as S
    return S


def _to_dev(qs, C):
    n = len(qs)
    q = torch.zeros(n, C, 8, device="cuda")
    q[:, :, :7] = torch.from_numpy(np.asarray(qs)).float()
    return q


def _cases(name, seed, n, sigma, **kw):
    wl = scenes.make_problem(name, seed=seed, **kw)
    orc = O.Oracle(wl, n_threads=8)
    sol, _, _ = orc.place_solve()
    rng = np.random.default_rng(seed)
    qs = []
    for p in range(n):
        q = orc.lift(sol[p % len(sol)], p)
        q[1:] += rng.normal(0, sigma, q[1:].shape)
        q = np.clip(q, wl.robot.qlim[:, 0], wl.robot.qlim[:, 1])
        qs.append(q)
    return wl, orc, sol, qs


@pytest.mark.parametrize("name,seed,n,sigma,kw", [
    ("tower1", 0, 9, 0.05, {}),
    ("tower4", 1, 5, 0.15, {"B": 3, "O": 12, "W": 8}),
    ("tower4", 2, 3, 0.2, {}),
])
def test_traj_eval_matches_oracle(name, seed, n, sigma, kw):
    S = _S()
    wl, orc, _, qs = _cases(name, seed, n, sigma, **kw)
    pr = S.Problem(wl)
    C, NR = pr.C, pr.NR
    q = _to_dev(qs, C)
    rng = np.random.default_rng(9)
    lam_np = rng.uniform(0, 2, (n, NR)).astype(np.float32)
    mu_np = rng.uniform(0.5, 4, n).astype(np.float32)
    lam, mu = torch.from_numpy(lam_np).cuda(), torch.from_numpy(mu_np).cuda()
    L, grad = torch.empty(n, device="cuda"), torch.empty(n, C, 8, device="cuda")
    groups, h = torch.empty(n, 6, device="cuda"), torch.empty(n, NR, device="cuda")
    S.spasm_traj_eval(pr, n, q, lam, mu, L, grad, groups, h)
    torch.cuda.synchronize()
    active = 0
    for p in range(n):
        qp = q[p, :, :7].cpu().double().numpy()
        Lo, go, cgo, path, jl, ho = orc.traj_cost(qp, lam_np[p].astype(np.float64), float(mu_np[p]))
        active += cgo[1] > 0 or cgo[2] > 0
        assert abs(L[p].item() - Lo) <= RTOL * max(abs(Lo), 1e-2), (p, L[p].item(), Lo)
        np.testing.assert_allclose(groups[p].cpu().double().numpy(), cgo, rtol=RTOL, atol=ATOL)
        np.testing.assert_allclose(h[p].cpu().double().numpy(), ho, rtol=RTOL, atol=ATOL)
        gd = grad[p, :, :7].cpu().double().numpy()
        err = np.linalg.norm(gd - go) / max(np.linalg.norm(go), 1e-2)
        assert err <= RTOL, (p, err)
        assert np.all(grad[p, :, 7].cpu().numpy() == 0)
    assert active > 0


def test_traj_eval_and_descent_at_the_compiled_maxima():
    """The largest problem the kernels take: 16 blocks, 256 cuboids (255 + table), 64
    obstacle spheres, 993 configurations (W = 32), NR = 147 residuals, so 8 cuboid mask words,
    2 sphere mask words, 16-bit block masks and one CTA per SM.  Objective, groups, residuals
    and gradient against the oracle, then a few descent steps."""
    S = _S()
    wl = scenes.make_problem("tower10", seed=0, B=16, O=255, W=32, n_obstacle_spheres=64, Q=4)
    orc = O.Oracle(wl, n_threads=8)
    pr = S.Problem(wl)
    C, NR = pr.C, pr.NR
    assert (C, NR, len(wl.scene.cuboid), len(wl.scene.sphere)) == (993, 147, 256, 64)
    rng = np.random.default_rng(3)
    qs = []
    for p, sigma in enumerate((0.1, 0.3, 0.6)):
        qp = np.tile(wl.robot.q_home, (C, 1)) + rng.normal(0, sigma, (C, 7))
        qp = np.clip(qp, wl.robot.qlim[:, 0], wl.robot.qlim[:, 1])
        qp[0] = wl.robot.q_home
        qs.append(qp)
    n = len(qs)
    q = _to_dev(qs, C)
    lam_np = rng.uniform(0, 2, (n, NR)).astype(np.float32)
    mu_np = rng.uniform(0.5, 4, n).astype(np.float32)
    lam, mu = torch.from_numpy(lam_np).cuda(), torch.from_numpy(mu_np).cuda()
    L, grad = torch.empty(n, device="cuda"), torch.empty(n, C, 8, device="cuda")
    groups, h = torch.empty(n, 6, device="cuda"), torch.empty(n, NR, device="cuda")
    S.spasm_traj_eval(pr, n, q, lam, mu, L, grad, groups, h)
    torch.cuda.synchronize()
    for p in range(n):
        qp = q[p, :, :7].cpu().double().numpy()
        Lo, go, cgo, path, jl, ho = orc.traj_cost(qp, lam_np[p].astype(np.float64), float(mu_np[p]))
        assert cgo[1] > 0   # the arm collides: every mask word and candidate path is exercised
        assert abs(L[p].item() - Lo) <= RTOL * max(abs(Lo), 1e-2), (p, L[p].item(), Lo)
        np.testing.assert_allclose(groups[p].cpu().double().numpy(), cgo, rtol=RTOL, atol=ATOL)
        np.testing.assert_allclose(h[p].cpu().double().numpy(), ho, rtol=RTOL, atol=ATOL)
        gd = grad[p, :, :7].cpu().double().numpy()
        assert np.linalg.norm(gd - go) / max(np.linalg.norm(go), 1e-2) <= RTOL, p
    q0 = np.stack([q[p, :, :7].cpu().double().numpy() for p in range(n)])
    lam0, mu0 = torch.zeros(n, NR, device="cuda"), torch.full((n,), float(wl.params.mu0), device="cuda")
    S.spasm_traj_descend(pr, n, q, lam0, mu0, 3, 1)
    torch.cuda.synchronize()
    qr, _, _ = orc.traj_descend(q0, k_steps=3)
    # these states collide hard (objective ~1e4), so a step moves joints by up to the limits and
    # FP32 rounding of the gradient (~1e-5 relative) shows at the 1e-3 level on a few entries,
    # more where a contact switches between the two precisions
    err = np.abs(np.stack([q[p, :, :7].cpu().double().numpy() for p in range(n)]) - qr)
    assert np.quantile(err, 0.99) < 1e-3 and err.max() < 2e-2, (np.quantile(err, 0.99), err.max())


def test_empty_calls_do_nothing():
    """n = 0 at every kernel-level entry point: success, no work, outputs untouched."""
    S = _S()
    wl = scenes.make_problem("tower1", seed=0)
    pr = S.Problem(wl)
    try:
        x = torch.full((4 * pr.B, 1), 7.0, device="cuda")
        cost = torch.full((1,), 7.0, device="cuda")
        S.spasm_place_sample(pr, 0, 0, x, cost)
        S.spasm_place_eval(pr, 0, x, 0, cost, None, None, None)
        S.spasm_place_descend(pr, 0, x, 2, 1)
        q = torch.full((1, pr.C, 8), 7.0, device="cuda")
        place = torch.zeros(1, 4 * pr.B, device="cuda")
        S.spasm_lift(pr, 0, place, 1, 0, q)
        L = torch.full((1,), 7.0, device="cuda")
        S.spasm_traj_eval(pr, 0, q, None, None, L, None, None, None)
        S.spasm_traj_descend(pr, 0, q, None, None, 2, 1)
        torch.cuda.synchronize()
        assert torch.all(x == 7.0) and torch.all(cost == 7.0) and torch.all(q == 7.0) and torch.all(L == 7.0)
    finally:
        pr.close()


def test_lift_matches_oracle():
    """ik_mode 0 (damped least squares).  Interpolated waypoints are exact functions of the endpoints and via points; every IK
    endpoint that converges in the oracle (tool pose within 1e-6 of its target) lands on
    the same joint solution on the GPU.  Endpoints where damped least squares stalls (a
    joint limit, a singular direction) may stop at different points in FP32 and FP64."""
    S = _S()
    wl = scenes.make_problem("tower4", seed=3, B=3, O=8, W=10, ik_mode=0)
    orc = O.Oracle(wl)
    sol, _, _ = orc.place_solve()
    pr = S.Problem(wl)
    n, S_ = 24, wl.params.W - 1
    place = torch.from_numpy(sol.reshape(len(sol), -1)).float().cuda().contiguous()
    q = torch.zeros(n, pr.C, 8, device="cuda")
    S.spasm_lift(pr, n, place, len(sol), 2, q)
    torch.cuda.synchronize()
    ps = place.cpu().double().numpy().reshape(len(sol), pr.B, 4)
    converged = matched = 0
    for p in range(n):
        qo = orc.lift(ps[p % len(sol)], p, attempt=2)
        qg = q[p, :, :7].cpu().double().numpy()
        np.testing.assert_array_equal(qg[0], np.float32(wl.robot.q_home))
        for b in range(pr.B):
            for t, pose in (((2 * b + 1) * S_, wl.scene.init[b]), ((2 * b + 2) * S_, ps[p % len(sol)][b])):
                _, T = orc.fk(qo[t])
                target = np.array(pose[:3]) + [0, 0, wl.scene.half[b, 2] + wl.scene.grasp_off]
                if np.linalg.norm(T[:3, 3] - target) < 1e-6 and T[2, 2] < -1 + 1e-9:
                    converged += 1
                    matched += np.abs(qg[t] - qo[t]).max() < 2e-3
                    # a different IK branch is still a solution: the GPU tool reaches the target
                    _, Tg = orc.fk(qg[t])
                    assert np.linalg.norm(Tg[:3, 3] - target) < 1e-3 and Tg[2, 2] < -0.999
    # FP32 and FP64 iterates can part ways near a singular direction and converge to
    # different branches; the same branch is reached almost everywhere
    assert converged >= n and matched >= 0.95 * converged, (matched, converged)

@pytest.mark.parametrize("name,n,sample", [("tower4", 64, 64), ("tower10", 4096, 24)])
def test_analytic_lift_matches_oracle(name, n, sample):
    """ik_mode 1: every IK endpoint the oracle solves in closed form is the same branch on
    the GPU to FP32 rounding, except where two branches lie nearly equally far from the
    seed (the GPU's endpoint is then another exact solution) or where FP32 loses the last
    in-limit solution at a limit or at the edge of reach (the GPU then falls back to damped
    least squares, as the oracle does where it finds none).  tower10 runs the full
    4096-particle lift of the benchmark and checks a sample of particles."""
    S = _S()
    wl = scenes.make_problem(name, seed=4, ik_mode=1)
    orc = O.Oracle(wl)
    pr = S.Problem(wl)
    S_ = wl.params.W - 1
    lo, hi = wl.robot.qlim[:, 0], wl.robot.qlim[:, 1]
    place_h = wl.scene.init.copy()
    place_h[:, 0] += 0.04
    place_h[:, 3] += 0.25
    place = torch.from_numpy(place_h.reshape(1, -1)).float().cuda().contiguous()
    q = torch.zeros(n, pr.C, 8, device="cuda")
    S.spasm_lift(pr, n, place, 1, 1, q)
    torch.cuda.synchronize()
    ps = place.cpu().double().numpy().reshape(pr.B, 4)
    analytic = matched = other_branch = 0
    for p in np.linspace(0, n - 1, sample).astype(int):
        qo, how = orc.lift_methods(ps, int(p), attempt=1)
        qg = q[p, :, :7].cpu().double().numpy()
        for b in range(pr.B):
            for which, t in enumerate(((2 * b + 1) * S_, (2 * b + 2) * S_)):
                if not how[b, which]:
                    continue
                analytic += 1
                if np.abs(qg[t] - qo[t]).max() < 2e-3:
                    matched += 1
                    continue
                _, T = orc.fk(qo[t])
                _, Tg = orc.fk(qg[t])
                if np.abs(Tg - T).max() < 1e-4 and np.all(qg[t] >= lo - 1e-6) and np.all(qg[t] <= hi + 1e-6):
                    other_branch += 1
    assert analytic >= 0.95 * sample * 2 * pr.B, analytic
    assert matched >= 0.98 * analytic and matched + other_branch >= 0.99 * analytic, (matched, other_branch, analytic)


def test_analytic_lift_rejects_other_joint_layouts():
    S = _S()
    wl = scenes.make_problem("tower1", seed=0, ik_mode=1)
    wl.robot.dh[2, 0] = 0.02          # an elbow offset the closed form does not cover
    with pytest.raises(S.SpasmError, match="ik_mode 1"):
        S.Problem(wl)
    wl.params.ik_mode = 0             # damped least squares takes any layout
    S.Problem(wl).close()


@pytest.mark.parametrize("name,seed,n,sigma,kw", [
    ("tower1", 4, 16, 0.05, {}),
    ("tower4", 1, 8, 0.15, {"B": 3, "O": 12, "W": 8}),
])
def test_descend_one_step_matches_oracle_on_every_particle(name, seed, n, sigma, kw):
    """One descent step from identical states, element-wise on every particle: K = 2 gives
    the steps eta_traj (1 - 1/2) and 0 (the schedule of Sec. III-B), so q moves once along the
    gradient at the start.  The step agrees with the oracle's to 1e-4 of its norm (the
    gradient's FP32 rounding) plus the float32 rounding of the joint values."""
    S = _S()
    wl, orc, _, qs = _cases(name, seed, n, sigma, **kw)
    pr = S.Problem(wl)
    q = _to_dev(qs, pr.C)
    q0 = np.stack([q[p, :, :7].cpu().double().numpy() for p in range(n)])
    lam = torch.zeros(n, pr.NR, device="cuda")
    mu = torch.full((n,), float(wl.params.mu0), device="cuda")
    S.spasm_traj_descend(pr, n, q, lam, mu, 2, 1)
    torch.cuda.synchronize()
    qr, _, _ = orc.traj_descend(q0, k_steps=2)
    for p in range(n):
        step_g = q[p, :, :7].cpu().double().numpy() - q0[p]
        step_o = qr[p] - q0[p]
        err = np.abs(step_g - step_o).max()
        assert err <= RTOL * np.abs(step_o).max() + 1e-6, (p, err, np.abs(step_o).max())


def test_descend_matches_oracle_few_steps():
    S = _S()
    wl, orc, _, qs = _cases("tower1", 4, 6, 0.05)
    pr = S.Problem(wl)
    q = _to_dev(qs, pr.C)
    q0 = [q[p, :, :7].cpu().double().numpy() for p in range(len(qs))]
    lam = torch.zeros(len(qs), pr.NR, device="cuda")
    mu = torch.full((len(qs),), float(wl.params.mu0), device="cuda")
    S.spasm_traj_descend(pr, len(qs), q, lam, mu, 4, 1)
    torch.cuda.synchronize()
    qr, lr, mr = orc.traj_descend(np.stack(q0), k_steps=4)
    for p in range(len(qs)):
        err = np.abs(q[p, :, :7].cpu().double().numpy() - qr[p]).max()
        assert err < 1e-4, (p, err)


def test_descend_full_schedule_matches_oracle():
    """All K_traj = 50 steps in one launch, over which the cached cull skips and re-culls
    chunks: the trajectories stay with the FP64 oracle's (FP32 rounding accumulates over
    the steps, and a contact switching on or off in one precision only can move a particle)."""
    S = _S()
    wl, orc, _, qs = _cases("tower4", 2, 8, 0.05)
    pr = S.Problem(wl)
    n = len(qs)
    q = _to_dev(qs, pr.C)
    q0 = np.stack([q[p, :, :7].cpu().double().numpy() for p in range(n)])
    lam = torch.zeros(n, pr.NR, device="cuda")
    mu = torch.full((n,), float(wl.params.mu0), device="cuda")
    K = wl.params.K_traj
    S.spasm_traj_descend(pr, n, q, lam, mu, K, 1)
    torch.cuda.synchronize()
    qr, _, _ = orc.traj_descend(q0, k_steps=K)
    err = np.array([np.abs(q[p, :, :7].cpu().double().numpy() - qr[p]).max() for p in range(n)])
    assert np.median(err) < 1e-3 and np.mean(err < 1e-2) >= 0.75, np.sort(err)


def test_cached_cull_engages_and_counts():
    """The trajectory kernel's counters: some configurations keep their cull between
    iterations (fewer culled than evaluated), and only culled configurations can have a
    candidate."""
    S = _S()
    wl = scenes.make_problem("tower4", seed=1)
    pr = S.Problem(wl)
    try:
        S.spasm_optimize(pr)
        st = S.spasm_get_stats(pr)
    finally:
        pr.close()
    evals = wl.params.Q * (wl.params.K_traj + 1) * st["traj_launches"]
    assert 0 < st["cand_configs"] <= st["cull_configs"] < evals * (pr.C - 1), st
    assert st["tests_executed"] > 0


def test_optimize_end_to_end_tower1():
    """Both stages on the device; every returned trajectory passes the FP64 oracle check."""
    S = _S()
    wl = scenes.make_problem("tower1", seed=0)
    orc = O.Oracle(wl, eps=wl.params.eps * 1.05, eps_start=wl.params.eps_start * 1.05)
    pr = S.Problem(wl)
    S.spasm_optimize(pr)
    res = S.spasm_result(pr)
    assert res["n_found"] >= 1
    for q in res["traj"]:
        ok, m = orc.traj_check(q)
        assert ok, m


def test_descent_is_bitwise_repeatable_and_independent_of_the_launch():
    """The warps of a particle take the evaluation's work items (chunks, residual jobs, tower
    slices) from a shared counter, so which warp runs which item varies from run to run and
    with what else runs on the SM.  The sums are fixed point and the per-slice sums are added
    in a fixed order, so all 50 descent steps give the same bits twice in a row and for a
    particle descended alone or among others."""
    S = _S()
    wl, _, _, qs = _cases("tower4", 2, 8, 0.05)
    pr = S.Problem(wl)
    n, K = len(qs), wl.params.K_traj

    def descend(sub):
        q = _to_dev([qs[p] for p in sub], pr.C)
        lam = torch.zeros(len(sub), pr.NR, device="cuda")
        mu = torch.full((len(sub),), float(wl.params.mu0), device="cuda")
        S.spasm_traj_descend(pr, len(sub), q, lam, mu, K, 1)
        torch.cuda.synchronize()
        return q.cpu(), lam.cpu(), mu.cpu()

    everyone = list(range(n))
    a, b = descend(everyone), descend(everyone)
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    for p in (0, 3, n - 1):
        alone = descend([p])
        for x, y in zip(alone, a):
            assert torch.equal(x[0], y[p]), p
