"""Element-wise parity of the FP64 final check (GetSatisfyingParticles of Alg. 1 applied to
the returned solutions, Sec. III) against the oracle's or_traj_check.

The GPU check reads the float32 joint values the optimiser returns and holds the joint
limits as float32 (a joint clamped to its limit in FP32 sits on the float nearest the
limit); the oracle is given exactly those joint values and those limits, so both evaluate
the same trajectories in double precision and the metrics agree to rounding (1e-9
relative), the verdicts exactly.  Planted cases put each acceptance criterion 2% of its
threshold inside or outside (far beyond the float32 rounding of the joints), so a check that
accepts everything, or tests a criterion against the wrong threshold, fails.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2510_07674_gb300 import scenes
from probe_scenes import H, CheckScene, Rz, T4

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

MET_RTOL, MET_ATOL = 1e-9, 1e-13


def _S():
    from paper_2510_07674_gb300 import spasm as S
    return S


def _float_limits(wl):
    """The workload with its joint limits rounded to float32 (what the GPU check holds)."""
    r = wl.robot
    robot = scenes.Robot(dh=r.dh, qlim=r.qlim.astype(np.float32).astype(np.float64), sphere_link=r.sphere_link,
                         sphere=r.sphere, ee=r.ee, q_home=r.q_home)
    return scenes.Problem(name=wl.name, robot=robot, scene=wl.scene, params=wl.params, packing=wl.packing,
                          p2p=wl.p2p)


def _gpu_check(pr, qs):
    S = _S()
    n, C = len(qs), pr.C
    q = torch.zeros(n, C, 8, device="cuda")
    q[:, :, :7] = torch.from_numpy(np.asarray(qs, dtype=np.float32))
    m = torch.full((n, 6), -1.0, dtype=torch.float64, device="cuda")
    ok = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    S.spasm_traj_check(pr, n, q, m, ok)
    torch.cuda.synchronize()
    return q[:, :, :7].cpu().double().numpy(), m.cpu().numpy(), ok.cpu().numpy()


def _compare(orc, q32, m, ok):
    for p in range(len(q32)):
        ok_o, m_o = orc.traj_check(q32[p])
        np.testing.assert_allclose(m[p], m_o, rtol=MET_RTOL, atol=MET_ATOL, err_msg=f"particle {p}")
        assert bool(ok[p]) == ok_o, (p, m[p], m_o)
    return [orc.traj_check(q)[0] for q in q32]


def test_check64_matches_oracle_on_solutions_and_perturbations():
    """Solutions of a 3-block scene (from the GPU solve) and copies perturbed at growing scales
    (a mix of accepted and refused trajectories), with more rows than P so the check runs in
    several chunks."""
    S = _S()
    wl = scenes.make_problem("tower4", seed=3, B=3, O=12, W=8, N=2048, M=512, P=8, Q=256)
    pr = S.Problem(wl)
    try:
        S.spasm_optimize(pr)
        r = S.spasm_result(pr)
        assert r["n_found"] > 0
        rng = np.random.default_rng(1)
        qs = []
        for sigma in (0.0, 1e-4, 1e-3, 1e-2, 5e-2):
            for t in r["traj"]:
                q = t.copy()
                q[1:] += rng.normal(0, sigma, q[1:].shape)
                qs.append(q)
        orc = O.Oracle(_float_limits(wl))
        q32, m, ok = _gpu_check(pr, qs)
        verdicts = _compare(orc, q32, m, ok)
        assert 0 < sum(verdicts) < len(verdicts), sum(verdicts)   # both outcomes occur
        # the returned solutions themselves: the success flags spasm_result reported
        np.testing.assert_array_equal(ok[: r["n_found"]], r["success"])
    finally:
        pr.close()


def _planted(**kw):
    cs = CheckScene(**kw)
    return cs, O.Oracle(_float_limits(cs.pr))


EPS = scenes.Params().eps
EPS_START = scenes.Params().eps_start


@pytest.mark.parametrize("criterion", ["arm", "start", "tilt", "place_pen", "com", "height", "limit"])
@pytest.mark.parametrize("side", [-1, 1])
def test_check64_planted_thresholds(criterion, side):
    """Each criterion 2% inside (side -1, accepted) or outside (side +1, refused) its threshold."""
    S = _S()
    f = 1.0 + 0.02 * side
    if criterion == "arm":
        cs, orc = _planted(arm_pen=EPS * f)
    elif criterion == "start":
        cs, orc = _planted(start_off=(0.0, np.sqrt(EPS_START * f), 0.0))
    elif criterion == "tilt":
        cs, orc = _planted(tilt=np.sqrt(EPS_START * f))
    elif criterion == "place_pen":
        cs, orc = _planted(box_gap=EPS * f)
    elif criterion == "height":
        cs, orc = _planted(dz=EPS * f)
    else:
        cs, orc = _planted()
    q = cs.q.copy()
    if criterion == "com":   # block 1 on block 0, shifted along block 0's x axis by h + eps f
        cs.place[1] = T4(Rz(0.4), cs.place[0][:3, 3] + Rz(0.4) @ np.array([H + EPS * f, 0.0, 2 * H]))
        q = cs._configs()
    if criterion == "limit":   # a transit waypoint's joint 2 just inside / outside its limit
        hi = float(np.float32(cs.robot.qlim[2, 1]))
        q[1, 2] = hi + side * 1e-5
    pr = S.Problem(cs.pr)
    try:
        q32, m, ok = _gpu_check(pr, [q])
        verdict = _compare(orc, q32, m, ok)[0]
        assert verdict == (side < 0), (criterion, side, m)
    finally:
        pr.close()


def test_check64_at_full_tower10_size():
    """The 4096 lifted trajectories of the 10-block workload, checked in one call (several
    chunks of P rows); a sample compared with the oracle element by element."""
    S = _S()
    wl = scenes.make_problem("tower10", seed=0)
    pr = S.Problem(wl)
    try:
        S.spasm_place(pr)
        pl = S.spasm_placements(pr)
        place = torch.from_numpy(pl["placements"].reshape(len(pl["placements"]), -1).astype(np.float32)).cuda()
        Q, C = int(wl.params.Q), pr.C
        q = torch.zeros(Q, C, 8, device="cuda")
        S.spasm_lift(pr, Q, place, len(pl["placements"]), 0, q)
        m = torch.full((Q, 6), -1.0, dtype=torch.float64, device="cuda")
        ok = torch.full((Q,), -1, dtype=torch.int32, device="cuda")
        S.spasm_traj_check(pr, Q, q, m, ok)
        torch.cuda.synchronize()
        mm, oo = m.cpu().numpy(), ok.cpu().numpy()
        assert np.all(mm >= 0.0) and np.all((oo == 0) | (oo == 1))
        orc = O.Oracle(_float_limits(wl))
        qh = q[:, :, :7].cpu().double().numpy()
        for p in np.random.default_rng(0).choice(Q, 6, replace=False):
            ok_o, m_o = orc.traj_check(qh[p])
            np.testing.assert_allclose(mm[p], m_o, rtol=MET_RTOL, atol=MET_ATOL, err_msg=f"particle {p}")
            assert bool(oo[p]) == ok_o
    finally:
        pr.close()
