"""Closed-form pins of the oracle's stage-2 arithmetic (appendix trajectory cost, Sec. III-B
augmented Lagrangian, final check, ranking cost) and of the stage-1 sampling map.

Central differences (test_oracle_costs.py) only show that the gradients match the values;
the tests here fix the values themselves on scenes built so that every term has a
hand-computed result:

* a *probe arm* whose seven joints all turn about the world z axis through the origin
  (every DH row zero except an optional offset a along joint 2), with a chosen flange ->
  tool transform, so link frames are Rz(q_1 + ... + q_k) (after the offset, a translation
  by a along the first joint's x axis) and the tool pose is known by hand;
* the real synthetic arm, with its sphere set replaced by one fixed sphere on the base, and
  configurations from its forward and analytic inverse kinematics (both pinned on their own
  in test_oracle_pins.py and test_oracle_ik.py), for the threshold tests of the check.

Which oracle function each test pins:
  C_arm value, obstacle membership   -> config_collisions via or_traj_cost (h[9B+1])
  C_block range and held block       -> config_collisions via or_traj_cost (h[9B+2])
  C_start, tilt residuals            -> traj_evaluate start terms, roll_pitch, held_block_frame
  placement on fk-derived poses      -> pose4_of + place_residuals via or_traj_cost (h[7B..9B])
  residual weights, L's form         -> residual_weight, or_traj_cost
  multiplier and penalty updates     -> or_traj_descend (eta_traj = 0)
  learning-rate schedule             -> or_traj_descend (K_al beyond the step count)
  acceptance thresholds and metrics  -> or_traj_check
  ranking cost                       -> or_traj_rank_cost
  sampling map                       -> or_place_sample
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2510_07674_gb300 import scenes
from probe_scenes import GO, H, CheckScene, Rx, Ry, Rz, T4, cuboid, held_block, probe_ee, probe_problem, probe_tool

def residuals(orc, q):
    L, g, cg, path, jl, h = orc.traj_cost(q, grad=False)
    return h, cg, path, jl


# --------------------------------------------------------------------------------------------
# C_arm: value, moving links, obstacle membership
# --------------------------------------------------------------------------------------------

def test_c_arm_fixed_and_moving_spheres_closed_form():
    """One base sphere sunk delta0 into a box counts delta0 at each of the C - 1 optimised
    configurations; a sphere on link 3 at radius rho from the axis meets the -x face of a
    second box at x = X, so it penetrates rho cos(q1 + q2 + q3) + r - X wherever positive."""
    d0, rho, r1, X = 0.004, 0.6, 0.04, 0.6
    spheres = [(0, (-0.5, -0.5, 0.2), 0.05), (3, (rho, 0.0, 0.1), r1)]
    boxes = [cuboid((-0.5 + 0.05 - d0 + 0.2, -0.5, 0.2), (0.2, 0.2, 0.2)),
             cuboid((X + 0.3, 0.0, 0.1), (0.3, 0.5, 0.3))]
    W = 5
    pr = probe_problem(1, W, probe_ee(), spheres, boxes, w_arm=1.0)
    orc = O.Oracle(pr)
    C = orc.C
    rng = np.random.default_rng(3)
    q = np.zeros((C, 7))
    q[1:, :3] = rng.uniform(-0.1, 0.1, (C - 1, 3))
    q[1:, 3:] = rng.uniform(-1.0, 1.0, (C - 1, 4))
    theta = q[1:, :3].sum(1)
    assert np.all(np.abs(theta) > 1e-3)
    expect = np.sum(d0 + np.maximum(0.0, rho * np.cos(theta) + r1 - X))
    h, cg, _, _ = residuals(orc, q)
    B = 1
    assert h[9 * B + 1] == pytest.approx(expect, rel=1e-12)
    assert cg[O.G_ARM] == pytest.approx(expect, rel=1e-12)
    assert h[9 * B + 2] == 0.0          # the held block stays clear of both boxes


def _membership_scene(d1, d2, d3):
    """Two blocks; every configuration is q = 0, so the tool holds the block at cb and block
    0's placed pose (from fk at its place configuration) is cb.  A base sphere of radius rs
    sits at cb + (h + rs - d1) x, penetrating block 0 *placed* by d1; block 0's initial
    pose is placed so that the sphere would penetrate it by d2, block 1's so that it
    penetrates it by d3."""
    rs = 0.05
    ee = probe_ee()
    cb = held_block(probe_tool(np.zeros(7), ee), H)[:3, 3]
    cs = cb + np.array([H + rs - d1, 0.0, 0.0])
    init = np.array([[*(cs - np.array([0.0, H + rs - d2, 0.0])), 0.0],
                     [*(cs + np.array([0.0, H + rs - d3, 0.0])), 0.0]])
    return probe_problem(2, 3, ee, [(0, tuple(cs), rs)], (), init=init)


def test_obstacle_membership_placed_and_unmoved_blocks():
    """Reading 9: in block b's two segments the obstacles are the blocks placed before b (at
    their fk-derived placed pose) and the blocks not yet moved (initial pose); block b itself
    is excluded.  With d1, d2, d3 distinct, C_arm = 2S d3 (block 1 unmoved, during block 0's
    segments) + 2S d1 (block 0 placed, during block 1's); d2 (block 0 at its initial pose)
    must not appear.  Block 1 held on its transfer interior sits exactly on block 0's placed
    pose: each of its 8 spheres (radius h/2, h/2 inside every face) penetrates by h."""
    d1, d2, d3 = 0.003, 0.005, 0.007
    pr = _membership_scene(d1, d2, d3)
    orc = O.Oracle(pr)
    S, B = pr.params.W - 1, 2
    q = np.zeros((orc.C, 7))
    h, cg, _, _ = residuals(orc, q)
    assert h[9 * B + 1] == pytest.approx(2 * S * (d1 + d3), rel=1e-12)
    # W = 3: one transfer-interior configuration per block; block 0's meets nothing
    assert h[9 * B + 2] == pytest.approx(8 * H, rel=1e-12)


def test_c_block_transfer_interior_only():
    """The held block counts only on the transfer interior (t = 1 .. T-1 of the transfer
    segment, appendix C_block): with every configuration at q = 0 and a box whose bottom face
    is delta below the top of the held block's upper spheres, each of the W - 2 interior
    configurations adds 4 delta; the grasp, the place and the transit configurations, where
    the tool is at the same spot, add nothing."""
    delta, W = 0.002, 5
    ee = probe_ee()
    cb = held_block(probe_tool(np.zeros(7), ee), H)[:3, 3]
    zf = cb[2] + H / 2 + H / 2 - delta
    box = cuboid((cb[0], cb[1], zf + 0.1), (0.2, 0.2, 0.1))
    pr = probe_problem(1, W, ee, [(0, (-0.8, -0.8, 0.1), 0.05)], [box], init=[[-0.5, 0.5, H, 0.0]])
    orc = O.Oracle(pr)
    h, cg, _, _ = residuals(orc, np.zeros((orc.C, 7)))
    assert h[9 * 1 + 2] == pytest.approx((W - 2) * 4 * delta, rel=1e-12)
    assert h[9 * 1 + 1] == 0.0
    # the block placed by the place configuration (q = 0, same spot) meets the box too
    assert h[9 * 1] == pytest.approx(4 * delta, rel=1e-12)


# --------------------------------------------------------------------------------------------
# C_start and the upright-placement residuals
# --------------------------------------------------------------------------------------------

@pytest.mark.parametrize("beta,gamma,dvec", [(0.0, 0.0, (0.0, 0.0, 0.0)), (0.0, 0.0, (0.004, 0.0, 0.0)),
                                             (-0.03, 0.05, (0.001, -0.002, 0.003)), (0.2, -0.1, (0.0, 0.0, 0.0))])
def test_c_start_closed_form(beta, gamma, dvec):
    """With the held block's orientation Rz(yaw) Ry(beta) Rx(gamma) (ZYX: pitch beta, roll
    gamma) and the initial block position offset by -dvec from the block the grasp
    configuration holds, the grasp residuals are (dvec, gamma, beta) and the place
    configuration's tilt residuals (gamma, beta): C_start = |dvec|^2 + 2 (gamma^2 + beta^2)."""
    ee = probe_ee(Ry(beta) @ Rx(gamma))
    W = 3
    S = W - 1
    q = np.zeros((2 * S + 1, 7))
    q[2 * S, 0] = 0.2           # the place configuration turns the yaw only
    blk = held_block(probe_tool(q[S], ee), H)
    init = [[*(blk[:3, 3] - np.array(dvec)), 0.7]]
    pr = probe_problem(1, W, ee, [(0, (-0.8, -0.8, 0.1), 0.05)], (), init=init)
    orc = O.Oracle(pr)
    h, cg, _, _ = residuals(orc, q)
    np.testing.assert_allclose(h[0:3], dvec, atol=1e-15)
    assert h[3] == pytest.approx(gamma, abs=1e-15)
    assert h[4] == pytest.approx(beta, abs=1e-15)
    assert h[5] == pytest.approx(gamma, abs=1e-15) and h[6] == pytest.approx(beta, abs=1e-15)
    expect = float(np.dot(dvec, dvec)) + 2 * (gamma ** 2 + beta ** 2)
    assert cg[O.G_START] == pytest.approx(expect, rel=1e-12, abs=1e-28)


def test_placement_residuals_on_fk_derived_poses():
    """The placement terms of C_trajopt are evaluated on the poses fk gives at the place
    configurations (appendix: C_placement({p_{b,T}})).  Probe arm with an offset a = 0.5 on
    joint 2: the tool is at (0.5 cos q1, 0.5 sin q1, 0.5) with yaw q1 + ... + q7.  Block 0
    (a 0.08 x 0.04 footprint) is placed at yaw pi/3, block 1 beside it: the CoM distance is
    the excess of Rz(-pi/3)(p1 - p0) over the footprint, the heights are 0.5 - hz - standoff
    against the stack targets."""
    a2, W = 0.5, 3
    S = W - 1
    ee = T4(Rx(math.pi), (0.0, 0.0, 0.5))
    half = np.array([[0.04, 0.02, H], [H, H, H]])
    q = np.zeros((4 * S + 1, 7))
    q[2 * S, 1] = math.pi / 3                  # place of block 0: position (0.5, 0), yaw pi/3
    q[4 * S, 0], q[4 * S, 1] = 0.2, 0.1        # place of block 1: position 0.5 (cos .2, sin .2)
    z_table = 0.3
    pr = probe_problem(2, W, ee, [(0, (-0.8, -0.8, 0.1), 0.05)], (), half=half,
                       init=[[-0.5, 0.5, H, 0.0], [-0.5, 0.7, H, 0.0]], z_table=z_table, a2=a2)
    orc = O.Oracle(pr)
    h, cg, _, _ = residuals(orc, q)
    B = 2
    p0 = held_block(probe_tool(q[2 * S], ee, a2), H)[:3, 3]
    p1 = held_block(probe_tool(q[4 * S], ee, a2), H)[:3, 3]
    np.testing.assert_allclose(p0[:2], [0.5, 0.0], atol=1e-15)
    u = Rz(-math.pi / 3)[:2, :2] @ (p1[:2] - p0[:2])
    D0 = float(np.linalg.norm(np.maximum(np.abs(u) - half[0, :2], 0.0)))
    # the yaw matters: the footprint axes in the world frame give another distance
    D_world = float(np.linalg.norm(np.maximum(np.abs(p1[:2] - p0[:2]) - half[0, :2], 0.0)))
    assert abs(D0 - D_world) > 1e-3
    assert h[8 * B + 0] == pytest.approx(D0, rel=1e-12)
    assert h[8 * B + 1] == 0.0
    assert h[7 * B + 0] == pytest.approx(0.5 - H - GO - (z_table + H), abs=1e-15)
    assert h[7 * B + 1] == pytest.approx(0.5 - H - GO - (z_table + 3 * H), abs=1e-15)
    assert cg[O.G_STABLE] == pytest.approx(D0, rel=1e-12)
    assert cg[O.G_HEIGHT] == pytest.approx(h[7 * B] ** 2 + h[7 * B + 1] ** 2, rel=1e-12)
    assert h[9 * B] == 0.0     # the two placed blocks are apart and nothing else is near


# --------------------------------------------------------------------------------------------
# augmented Lagrangian: residual weights, multiplier and penalty updates, step schedule
# --------------------------------------------------------------------------------------------

WEIGHTS = dict(w_start=2.0, w_height=3.0, w_stable=5.0, w_coll=7.0, w_arm=11.0, w_block=13.0)


def _layout_weight(B, r):
    """Residual layout of the stage-2 augmented Lagrangian: 7B start/tilt entries, B heights,
    B CoM distances, then the placement collision sum, C_arm and C_block."""
    if r < 7 * B:
        return WEIGHTS["w_start"]
    if r < 8 * B:
        return WEIGHTS["w_height"]
    if r < 9 * B:
        return WEIGHTS["w_stable"]
    return [WEIGHTS["w_coll"], WEIGHTS["w_arm"], WEIGHTS["w_block"]][r - 9 * B]


def _two_block_case(sigma=0.12, seed=2, **prm):
    pr = scenes.make_problem("tower4", seed=seed, B=2, O=6, W=6, N=512, M=128, **prm)
    orc = O.Oracle(pr, n_threads=4)
    sol, _, _ = orc.place_solve()
    assert len(sol) > 0
    rng = np.random.default_rng(seed)
    qs = []
    for p in range(8):
        q = orc.lift(sol[p % len(sol)], p)
        q[1:] += rng.normal(0, sigma, q[1:].shape)
        q[1:] = np.clip(q[1:], pr.robot.qlim[:, 0] + 1e-3, pr.robot.qlim[:, 1] - 1e-3)
        qs.append(q)
    return pr, orc, qs


def test_lagrangian_form_and_residual_weights():
    """L = w_path path + w_jl jl + sum_r lambda_r sqrt(w_r) h_r + mu/2 w_r h_r^2 with w_r from
    the residual layout: with lambda = e_r, L - L(lambda = 0) = sqrt(w_r) h_r for every r, and
    L(lambda = 0) - w_path path - w_jl jl = mu/2 sum_r w_r h_r^2.  Distinct weights per group,
    so a residual given another group's weight fails."""
    pr, orc, qs = _two_block_case(sigma=0.25, **WEIGHTS)
    B, NR = 2, orc.NR
    mu = 1.7
    nonzero = np.zeros(NR, bool)
    for q in qs:
        L0, _, _, path, jl, h = orc.traj_cost(q, np.zeros(NR), mu, grad=False)
        w = np.array([_layout_weight(B, r) for r in range(NR)])
        quad = L0 - pr.params.w_path * path - pr.params.w_jl * jl
        assert quad == pytest.approx(0.5 * mu * np.sum(w * h * h), rel=1e-12)
        for r in range(NR):
            lam = np.zeros(NR)
            lam[r] = 1.0
            L1 = orc.traj_cost(q, lam, mu, grad=False)[0]
            assert L1 - L0 == pytest.approx(math.sqrt(w[r]) * h[r], rel=1e-9, abs=1e-12 * max(1.0, abs(L0)))
        nonzero |= np.abs(h) > 1e-9
    # every group took part: start, tilt, heights, CoM (block 0), collisions sum, arm, block
    groups = [range(0, 5 * B), range(5 * B, 7 * B), range(7 * B, 8 * B), [8 * B], [9 * B + 1], [9 * B + 2]]
    for g in groups:
        assert nonzero[list(g)].any(), list(g)


def test_multiplier_and_penalty_updates_with_zero_step():
    """eta_traj = 0 leaves q unchanged, so h is constant and the updates follow the closed
    form: every K_al steps lambda += mu sqrt(w) h, then mu = min(2 mu, mu_max).  25 steps with
    K_al = 10, mu0 = 1, mu_max = 3: updates at steps 10 and 20 with mu = 1 and 2, so
    lambda = lambda0 + 3 sqrt(w) h, final mu = min(4, 3) = 3."""
    pr, orc, qs = _two_block_case(eta_traj=0.0, K_al=10, mu0=1.0, mu_max=3.0, **WEIGHTS)
    B, NR = 2, orc.NR
    rng = np.random.default_rng(5)
    q0 = np.stack(qs[:3])
    lam0 = rng.uniform(0.0, 1.0, (3, NR))
    q1, lam1, mu1 = orc.traj_descend(q0, lam0, np.ones(3), 25)
    np.testing.assert_array_equal(q1, q0)
    np.testing.assert_array_equal(mu1, [3.0, 3.0, 3.0])
    w = np.array([_layout_weight(B, r) for r in range(NR)])
    for p in range(3):
        h = orc.traj_cost(q0[p], lam0[p], 1.0, grad=False)[5]
        np.testing.assert_allclose(lam1[p], lam0[p] + 3.0 * np.sqrt(w) * h, rtol=1e-12, atol=1e-15)
    # mu_max above the doublings: 1 -> 2 -> 4
    _, _, mu2 = orc.__class__(pr, eta_traj=0.0, K_al=10, mu0=1.0, mu_max=100.0).traj_descend(q0, lam0, None, 25)
    np.testing.assert_array_equal(mu2, [4.0, 4.0, 4.0])


def test_step_schedule():
    """eta_k = eta_traj (1 - k/K): with K = 3 the steps are 2/3 eta and 1/3 eta along the
    gradient at the current point, and the last step is zero (no multiplier update: K_al
    beyond the step count)."""
    pr, orc, qs = _two_block_case(eta_traj=0.004, K_al=100, **WEIGHTS)
    NR = orc.NR
    eta = 0.004
    q0 = qs[0]
    lam = np.zeros(NR)
    mu = pr.params.mu0
    g0 = orc.traj_cost(q0, lam, mu)[1]
    qa = q0 - (2.0 / 3.0) * eta * g0
    g1 = orc.traj_cost(qa, lam, mu)[1]
    qb = qa - (1.0 / 3.0) * eta * g1
    lo, hi = pr.robot.qlim[:, 0], pr.robot.qlim[:, 1]
    assert np.all((qa[1:] > lo) & (qa[1:] < hi)) and np.all((qb[1:] > lo) & (qb[1:] < hi))
    q3, _, _ = orc.traj_descend(q0[None], None, None, 3)
    np.testing.assert_allclose(q3[0], qb, rtol=0, atol=1e-13)
    q1, _, _ = orc.traj_descend(q0[None], None, None, 1)      # K = 1: eta (1 - 1) = 0
    np.testing.assert_array_equal(q1[0], q0)


# --------------------------------------------------------------------------------------------
# final check: each criterion at its threshold, and the metrics' values
# --------------------------------------------------------------------------------------------

EPS = scenes.Params().eps
EPS_START = scenes.Params().eps_start


def test_check_accepts_the_designed_solution():
    cs = CheckScene()
    ok, m = cs.orc.traj_check(cs.q)
    assert ok, m
    assert m.max() < 1e-12


@pytest.mark.parametrize("side", [-1, 1])
def test_check_arm_penetration_threshold(side):
    d = EPS + side * 1e-9
    cs = CheckScene(arm_pen=d)
    ok, m = cs.orc.traj_check(cs.q)
    assert m[0] == pytest.approx(d, abs=1e-13)
    assert ok == (side < 0)


@pytest.mark.parametrize("side", [-1, 1])
def test_check_grasp_alignment_threshold(side):
    """max grasp alignment = the squared position error when the orientation is exact."""
    d = math.sqrt(EPS_START * (1.0 + side * 1e-6))
    cs = CheckScene(start_off=(0.0, d, 0.0))
    ok, m = cs.orc.traj_check(cs.q)
    assert m[1] == pytest.approx(d * d, rel=1e-8)
    assert ok == (side < 0)


@pytest.mark.parametrize("side", [-1, 1])
def test_check_tilt_threshold(side):
    """Block 0 placed with a roll gamma: the tilt metric is gamma^2 (grasps stay exact)."""
    g = math.sqrt(EPS_START * (1.0 + side * 1e-6))
    cs = CheckScene(tilt=g)
    ok, m = cs.orc.traj_check(cs.q)
    assert m[2] == pytest.approx(g * g, rel=1e-8)
    assert m[1] < 1e-20
    assert ok == (side < 0)


@pytest.mark.parametrize("side", [-1, 1])
def test_check_placement_penetration_threshold(side):
    """A box pressing eps -+ 1e-9 into the side of placed block 0: its two-by-two spheres on
    that side penetrate by that much (placement collision metric)."""
    d = EPS + side * 1e-9
    cs = CheckScene(box_gap=d)
    ok, m = cs.orc.traj_check(cs.q)
    assert m[3] == pytest.approx(d, abs=1e-13)
    assert m[0] < 1e-13         # no arm or held-block contact
    assert ok == (side < 0)


@pytest.mark.parametrize("side", [-1, 1])
def test_check_com_threshold(side):
    """Block 1 on block 0 shifted by h + d along block 0's axis direction (yaw 0.4 for both,
    so the shift is taken along the rotated x axis): CoM distance d."""
    d = EPS + side * 1e-9
    cs = CheckScene()
    # rebuild with the shift along block 0's x axis
    R = Rz(0.4)
    cs.place[1] = T4(Rz(0.4), cs.place[0][:3, 3] + R @ np.array([H + d, 0.0, 2 * H]))
    cs.q = cs._configs()
    ok, m = cs.orc.traj_check(cs.q)
    assert m[4] == pytest.approx(d, abs=1e-12)
    assert ok == (side < 0)


@pytest.mark.parametrize("side", [-1, 1])
def test_check_height_threshold(side):
    d = EPS + side * 1e-9
    cs = CheckScene(dz=d)
    ok, m = cs.orc.traj_check(cs.q)
    assert m[5] == pytest.approx(d, abs=1e-12)
    assert ok == (side < 0)


@pytest.mark.parametrize("side", [-1, 1])
def test_check_joint_limit(side):
    """A transit waypoint with one joint 1e-9 inside / outside its upper limit."""
    cs = CheckScene()
    q = cs.q.copy()
    j = 2
    q[1, j] = cs.robot.qlim[j, 1] + side * 1e-9
    ok, m = cs.orc.traj_check(q)
    assert ok == (side < 0)


# --------------------------------------------------------------------------------------------
# ranking cost of a returned solution
# --------------------------------------------------------------------------------------------

def test_rank_cost_hand_case():
    """Probe arm with the tool on the joint axis (position fixed, yaw = sum q): joint 7 ramps
    by kappa per configuration, so path = (C-1) kappa^2; the grasp holds the block delta from
    its initial position (C_start = delta^2); the placed block is e above its target (C_height
    = e^2); a base sphere sunk da into a box (C_arm = (C-1) da).  Ranking cost = C_trajopt +
    w_path path with the given weights."""
    kappa, delta, e, da, W = 0.1, 0.003, 0.002, 0.004, 3
    ee = probe_ee(t=(0.0, 0.0, 0.5))
    cb = held_block(probe_tool(np.zeros(7), ee), H)[:3, 3]
    z_table = cb[2] - H - e
    sph = (0.9, 0.9, 0.2)
    box = cuboid((sph[0] + 0.05 - da + 0.1, sph[1], sph[2]), (0.1, 0.1, 0.1))
    w = dict(w_path=0.37, w_height=3.0, w_start=2.0, w_arm=11.0, w_block=13.0, w_stable=5.0, w_coll=7.0)
    pr = probe_problem(1, W, ee, [(0, sph, 0.05)], [box], init=[[cb[0] + delta, cb[1], cb[2], 0.0]],
                       z_table=z_table, **w)
    orc = O.Oracle(pr)
    C = orc.C
    q = np.zeros((C, 7))
    q[:, 6] = kappa * np.arange(C)
    expect = w["w_path"] * (C - 1) * kappa ** 2 + w["w_start"] * delta ** 2 + w["w_height"] * e ** 2 \
        + w["w_arm"] * (C - 1) * da
    assert orc.traj_rank_cost(q) == pytest.approx(expect, rel=1e-10)


# --------------------------------------------------------------------------------------------
# stage-1 sampling map (Alg. 1 SampleUniform)
# --------------------------------------------------------------------------------------------

def test_place_sample_map():
    """Draw (block i, particle p) uses Philox counter (i, p, 0, attempt) with the problem seed;
    its four uniforms map affinely onto x, y in the goal box, z between max(box z_lo, table +
    hz) and the box top, and yaw in [-pi, pi).  The draws over many particles are uniform on
    those ranges (Kolmogorov-Smirnov)."""
    stats = pytest.importorskip("scipy.stats")
    pr = scenes.make_problem("tower4", seed=9, B=3)
    orc = O.Oracle(pr)
    n, attempt = 4000, 2
    x = orc.place_sample(n, attempt)
    box = pr.scene.box
    for i in range(3):
        zlo = max(box[2], pr.scene.z_table + pr.scene.half[i, 2])
        lo = np.array([box[0], box[1], zlo, -math.pi])
        hi = np.array([box[3], box[4], box[5], math.pi])
        u = (x[:, i, :] - lo) / (hi - lo)
        assert np.all(u >= 0.0) and np.all(u < 1.0)
        for k in range(4):
            assert stats.kstest(u[:, k], "uniform").pvalue > 1e-3
        for p in (0, 1, 1234, n - 1):
            bits = O.philox4x32_10([i, p, 0, attempt], pr.params.seed)
            uu = np.array([O.u01(int(b)) for b in bits])
            np.testing.assert_allclose(x[p, i], lo + uu * (hi - lo), rtol=0, atol=1e-15)
