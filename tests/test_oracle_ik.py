"""Pins of the oracle's analytic IK (the lift of Sec. III-B with the analytic IK of the
Franka joint layout) against forward kinematics, which is pinned on its own: round trips
from random in-limit configurations, exactness of every returned solution, reach and
structure limits, the nearest-to-seed selection, and the lift rows it produces; no GPU."""
import math

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2510_07674_gb300 import scenes


def _oracle(robot_seed=7, **kw):
    pb = scenes.make_problem("tower4", seed=0, robot_seed=robot_seed)
    return Oracle(pb, **kw), pb.robot.qlim[:, 0], pb.robot.qlim[:, 1]


@pytest.mark.parametrize("robot_seed", [7, 11, 23])
def test_round_trip_recovers_every_in_limit_configuration(robot_seed):
    # any configuration within the limits is a solution of its own tool pose for its own
    # last joint, so the solver must return it; a dropped term, a wrong sign or a swapped
    # branch in any of the steps loses it for most configurations
    o, lo, hi = _oracle(robot_seed)
    assert o.ik_analytic_supported()
    rng = np.random.default_rng(robot_seed)
    counts = []
    for _ in range(300):
        q = rng.uniform(lo, hi)
        _, T = o.fk(q)
        sols = o.ik_analytic(T, q[6])
        counts.append(len(sols))
        assert len(sols) >= 1
        assert np.abs(sols - q).max(axis=1).min() < 1e-9
        # every returned solution reaches the pose exactly and respects the limits
        for s in sols:
            _, T2 = o.fk(s)
            assert np.abs(T2 - T).max() < 1e-10
            assert np.all(s >= lo) and np.all(s <= hi)
            assert s[6] == q[6]
        # solutions are distinct
        for i in range(len(sols)):
            for j in range(i):
                assert np.abs(sols[i] - sols[j]).max() > 1e-9
    assert max(counts) >= 4     # several branches are in limits for some poses


def test_out_of_reach_and_unsupported_layouts():
    o, _, _ = _oracle()
    T = np.eye(4)
    T[:3, 3] = (2.5, 0.0, 0.4)              # beyond the arm's reach
    assert all(len(o.ik_analytic(T, c)) == 0 for c in np.linspace(-2.5, 2.5, 11))
    pb = scenes.make_problem("tower4", seed=0)
    pb.robot.dh[2, 0] = 0.01                # an offset the layout does not have
    assert not Oracle(pb).ik_analytic_supported()
    pb = scenes.make_problem("tower4", seed=0)
    pb.robot.dh[5, 1] = -math.pi / 2        # a flipped twist
    assert not Oracle(pb).ik_analytic_supported()


def test_solutions_of_a_top_down_grasp_over_the_last_joint():
    # a top-down tool pose over the table is reachable for a range of last-joint values,
    # and the elbow-up/down and shoulder branches give distinct configurations
    o, _, _ = _oracle()
    T = np.eye(4)
    T[:3, :3] = np.diag([1.0, -1.0, -1.0])  # Rx(pi): tool z down
    T[:3, 3] = (0.5, 0.1, 0.15)
    found, most = 0, 0
    for c in np.linspace(-2.5, 2.5, 21):
        sols = o.ik_analytic(T, c)
        found += len(sols) > 0
        most = max(most, len(sols))
        for s in sols:
            _, T2 = o.fk(s)
            assert np.abs(T2 - T).max() < 1e-10
    assert found >= 5 and most >= 2


def test_selection_is_the_nearest_solution_over_all_candidates():
    o, lo, hi = _oracle()
    rng = np.random.default_rng(5)
    for _ in range(50):
        q = rng.uniform(lo, hi)
        _, T = o.fk(q)
        seed = np.clip(q + rng.normal(0, 0.4, 7), lo, hi)
        q6s = np.concatenate([[seed[6]], rng.uniform(lo[6], hi[6], 7)])
        found, got = o.ik_select(T, seed, q6s)
        every = [s for c in q6s for s in o.ik_analytic(T, c)]
        if not every:
            assert not found
            continue
        assert found
        d = [float(np.sum((s - seed) ** 2)) for s in every]
        np.testing.assert_allclose(got, every[int(np.argmin(d))], atol=0)


def test_analytic_lift_reaches_the_grasp_targets_exactly():
    # the lift's grasp and place rows are top-down tool poses at the block's top face, with
    # the tool yaw equal to the block yaw modulo pi/2 (the grasp draw); the rows the analytic
    # IK produced reach them to rounding, and with the stratified last-joint values nearly
    # every target has one; damped least squares reaches them only approximately
    pb = scenes.make_problem("tower4", seed=3)
    o1, o0 = Oracle(pb, ik_mode=1), Oracle(pb, ik_mode=0)
    S = pb.params.W - 1
    sc = pb.scene
    place = sc.init.copy()
    place[:, 0] += 0.05
    place[:, 3] += 0.3
    analytic, total, worst_dls = 0, 0, 0.0
    for particle in range(24):
        q1, how = o1.lift_methods(place, particle)
        q0, how0 = o0.lift_methods(place, particle)
        assert not how0.any()
        for b in range(pb.scene.half.shape[0]):
            for which, (t, pose) in enumerate((((2 * b + 1) * S, sc.init[b]), ((2 * b + 2) * S, place[b]))):
                for q, mode in ((q1[t], 1), (q0[t], 0)):
                    _, T = o1.fk(q)
                    top = np.array([pose[0], pose[1], pose[2] + sc.half[b, 2] + sc.grasp_off])
                    yaw = math.atan2(T[1, 0], T[0, 0])
                    dyaw = (yaw - pose[3]) % (math.pi / 2)
                    err = max(np.abs(T[:3, 3] - top).max(), np.abs(T[:3, 2] - (0, 0, -1)).max(),
                              min(dyaw, math.pi / 2 - dyaw))
                    if mode == 1:
                        total += 1
                        if how[b, which]:
                            analytic += 1
                            assert err < 1e-9, (particle, b, which, err)
                    else:
                        worst_dls = max(worst_dls, err)
        np.testing.assert_array_equal(q1[0], pb.robot.q_home)
    assert analytic >= 0.95 * total, (analytic, total)
    assert worst_dls > 1e-9   # the iterative IK stops short of exact: the modes differ
