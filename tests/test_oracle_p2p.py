"""Pins of the oracle's point-to-point stage 2 (one transit segment to a tool target, Sec.
IV's motion-planning use) against its structure, the IK target and central differences."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2510_07674_gb300 import scenes


@pytest.fixture(scope="module")
def case():
    wl = scenes.make_p2p("p2p", seed=1, W=12)
    return wl, Oracle(wl)


def test_layout_and_residual_structure(case):
    wl, o = case
    assert o.C == wl.params.W and o.NR == 12   # one segment; residual vector of one target
    q = o.lift(np.zeros((1, 4)), 3)
    np.testing.assert_array_equal(q[0], wl.robot.q_home)
    L, g, cg, path, jl, h = o.traj_cost(q)
    # only the target alignment (0..4) and the arm group (10) can be nonzero: no placement
    # tilt (5, 6), height (7), support (8), placement collision (9) or held block (11)
    assert np.all(h[[5, 6, 7, 8, 9, 11]] == 0.0)
    assert cg[1] > 0 and cg[2] == 0 and cg[3] == cg[4] == cg[5] == 0
    np.testing.assert_array_equal(g[0], 0.0)   # q_home is not a variable


def test_lift_endpoint_reaches_the_target(case):
    wl, o = case
    tgt = wl.scene.init[0]
    hits = 0
    for p in range(8):
        q = o.lift(np.zeros((1, 4)), p)
        _, T = o.fk(q[-1])
        if np.linalg.norm(T[:3, 3] - tgt[:3]) < 1e-6 and T[2, 2] < -1 + 1e-9:
            hits += 1
            L, g, cg, path, jl, h = o.traj_cost(q)
            assert np.abs(h[:5]).max() < 1e-6   # aligned: position and tilt residuals vanish
    assert hits >= 4   # a target without an in-limit closed-form solution falls back to damped least squares


def test_gradient_matches_central_differences(case):
    wl, o = case
    rng = np.random.default_rng(0)
    q = o.lift(np.zeros((1, 4)), 1)
    q[1:] += rng.normal(0, 0.05, q[1:].shape)
    lam = rng.uniform(0, 1, o.NR)
    L, g, cg, path, jl, h = o.traj_cost(q, lam=lam, mu=2.0)
    assert cg[1] > 0
    h_ = 1e-6
    for t in (1, o.C // 2, o.C - 1):
        for j in range(7):
            qp, qm = q.copy(), q.copy()
            qp[t, j] += h_
            qm[t, j] -= h_
            fd = (o.traj_cost(qp, lam=lam, mu=2.0, grad=False)[0] - o.traj_cost(qm, lam=lam, mu=2.0, grad=False)[0]) / (2 * h_)
            assert abs(fd - g[t, j]) <= 1e-6 * max(1.0, abs(fd)), (t, j, fd, g[t, j])
