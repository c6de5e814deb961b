"""Pins of the oracle's cost terms, gradients, IK, lift and Alg. 1 control flow.

Closed-form special cases of the appendix's tower cost, central differences for every
analytic gradient, FK round trips for IK, and invariants of the lift and the optimiser.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2510_07674_gb300 import scenes

H = scenes.BLOCK_HALF


def _problem(B, O_=0, **kw):
    return scenes.make_problem("tower4", seed=11, B=B, O=O_, **kw)


def _stack(pr, dx=0.0):
    B = len(pr.scene.half)
    cx, cy = pr.scene.box[[0, 3]].mean(), pr.scene.box[[1, 4]].mean()
    x = np.zeros((B, 4))
    for i in range(B):
        x[i] = (cx + (dx if i == B - 1 else 0.0), cy, pr.scene.z_table + (2 * i + 1) * H, 0.3)
    return x


@pytest.mark.parametrize("B", [1, 2, 5])
def test_perfect_stack_costs_zero(B):
    """A centred stack resting face to face: C_stable = C_height = C_coll = 0."""
    pr = _problem(B)
    orc = O.Oracle(pr)
    x = _stack(pr)
    for quad in (False, True):
        c, g, terms = orc.place_cost(x, quad=quad)
        # zero up to the rounding of the stacked heights (a few ulp of 0.25 m)
        assert terms[0] == 0.0 and terms[1] < 1e-30 and terms[2] < 1e-15
        assert c < 1e-13
    ok, m = orc.place_check(x)
    assert ok and m.max() < 1e-15


def test_stable_offset_closed_form():
    """Top block offset by half + delta along x (yaw 0): C_stable = delta."""
    pr = _problem(2)
    orc = O.Oracle(pr)
    for delta in (0.001, 0.01, 0.04):
        x = _stack(pr)
        x[:, 3] = 0.0
        x[1, 0] += H + delta
        _, _, terms = orc.place_cost(x)
        assert terms[0] == pytest.approx(delta, rel=1e-12)
    # com of the two blocks above the bottom one: offsets average (B = 3)
    pr3 = _problem(3)
    orc3 = O.Oracle(pr3)
    x = _stack(pr3)
    x[:, 3] = 0.0
    x[1, 1] += 0.05
    x[2, 1] += 0.05 + 0.04
    _, _, terms = orc3.place_cost(x)
    # block 0: CoM offset 0.07 -> 0.045 outside;  block 1: CoM offset 0.04 -> 0.015 outside
    assert terms[0] == pytest.approx(0.045 + 0.015, rel=1e-9)


def test_height_closed_form():
    pr = _problem(1)
    orc = O.Oracle(pr)
    for delta in (-0.003, 0.02):
        x = _stack(pr)
        x[0, 2] += delta
        _, g, terms = orc.place_cost(x)
        assert terms[1] == pytest.approx(delta * delta, rel=1e-12)
        # sunk into the table: the 4 bottom spheres also penetrate by -delta (linear form)
        n_pen = 4 if delta < 0 else 0
        assert terms[2] == pytest.approx(n_pen * -delta, abs=1e-15)
        expect = 2 * pr.params.w_height * delta - n_pen * pr.params.w_coll
        assert g[0, 2] == pytest.approx(expect, rel=1e-10)


def test_block_penetration_closed_form():
    """Upper block sunk by delta into the one below: its 4 bottom spheres penetrate by delta;
    the quadratic form gives 4 delta^2."""
    pr = _problem(2)
    orc = O.Oracle(pr)
    x = _stack(pr)
    x[:, 3] = 0.0
    delta = 0.004
    x[1, 2] -= delta
    _, _, t_lin = orc.place_cost(x)
    _, _, t_quad = orc.place_cost(x, quad=True)
    assert t_lin[2] == pytest.approx(4 * delta, rel=1e-12)
    assert t_quad[2] == pytest.approx(4 * delta * delta, rel=1e-12)


def _fd(f, x, h=1e-6):
    g = np.zeros_like(x)
    for idx in np.ndindex(x.shape):
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        g[idx] = (f(xp) - f(xm)) / (2 * h)
    return g


@pytest.mark.parametrize("quad", [False, True])
def test_place_gradient_central_difference(quad):
    pr = scenes.make_problem("tower4", seed=3)
    orc = O.Oracle(pr)
    xs = orc.place_sample(40)
    rng = np.random.default_rng(0)
    n_active = 0
    for x in xs:
        # pull blocks together so collisions and stability terms are active
        x[:, :2] = x[:, :2] * 0.3 + 0.7 * x[:, :2].mean(0) + rng.normal(0, 0.01, (len(x), 2))
        c, g, terms = orc.place_cost(x, quad=quad)
        n_active += terms[2] > 0 and terms[0] > 0
        fd = _fd(lambda z: orc.place_cost(z, quad=quad, grad=False)[0], x)
        assert np.linalg.norm(fd - g) <= 1e-6 * max(np.linalg.norm(fd), 1e-6), (fd, g)
    assert n_active > 5


def _traj_case(name, seed, n=3, sigma=0.05):
    pr = scenes.make_problem(name, seed=seed)
    orc = O.Oracle(pr)
    sol, _, _ = orc.place_solve()
    rng = np.random.default_rng(seed)
    qs = []
    for p in range(n):
        q = orc.lift(sol[p % len(sol)], p)
        q[1:] += rng.normal(0, sigma, q[1:].shape)
        qs.append(q)
    return orc, qs


@pytest.mark.parametrize("name,seed", [("tower1", 0), ("tower1", 5)])
def test_traj_gradient_central_difference(name, seed):
    orc, qs = _traj_case(name, seed)
    rng = np.random.default_rng(1)
    for q in qs:
        lam = rng.uniform(0.0, 2.0, orc.NR)
        mu = 3.0
        L, g, cg, path, jl, h = orc.traj_cost(q, lam, mu)
        fd = _fd(lambda z: orc.traj_cost(z, lam, mu, grad=False)[0], q)
        fd[0] = 0.0
        assert np.linalg.norm(fd - g) <= 1e-6 * max(np.linalg.norm(fd), 1e-6)


def test_traj_gradient_central_difference_multiblock():
    """Two blocks: placed-block obstacles and held-block spheres couple configurations."""
    pr = scenes.make_problem("tower4", seed=2, B=2, O=6, W=6)
    orc = O.Oracle(pr)
    sol, _, _ = orc.place_solve()
    rng = np.random.default_rng(2)
    n_coupled = 0
    for p in range(3):
        q = orc.lift(sol[p % len(sol)], p)
        q[1:] += rng.normal(0, 0.15, q[1:].shape)
        lam = rng.uniform(0.0, 2.0, orc.NR)
        L, g, cg, path, jl, h = orc.traj_cost(q, lam, 2.0)
        n_coupled += (cg[O.G_ARM] > 0) + (cg[O.G_BLOCK] > 0)
        fd = _fd(lambda z: orc.traj_cost(z, lam, 2.0, grad=False)[0], q)
        fd[0] = 0.0
        assert np.linalg.norm(fd - g) <= 1e-6 * max(np.linalg.norm(fd), 1e-6)
    assert n_coupled > 0


def test_ik_round_trip():
    """IK of a pose produced by FK from a reachable configuration reaches that pose."""
    pr = scenes.make_problem("tower1", seed=0)
    orc = O.Oracle(pr)
    rng = np.random.default_rng(7)
    qlim = pr.robot.qlim
    for _ in range(20):
        q_true = pr.robot.q_home + rng.uniform(-0.4, 0.4, 7)
        q_true = np.clip(q_true, qlim[:, 0], qlim[:, 1])
        _, T = orc.fk(q_true)
        q0 = np.clip(pr.robot.q_home + rng.uniform(-0.2, 0.2, 7), qlim[:, 0], qlim[:, 1])
        q = orc.ik(T, q0)
        _, T2 = orc.fk(q)
        assert np.abs(T2[:3, 3] - T[:3, 3]).max() < 1e-8
        assert np.abs(T2[:3, :3] - T[:3, :3]).max() < 1e-8
        assert np.all(q >= qlim[:, 0]) and np.all(q <= qlim[:, 1])


def test_lift_structure():
    """q[0] = q_home; interior waypoints of a segment lie on the two legs of a polyline;
    grasp configurations put the tool over the block's top face, pointing down."""
    pr = scenes.make_problem("tower4", seed=1, B=2, W=9)
    orc = O.Oracle(pr)
    sol, _, _ = orc.place_solve()
    q = orc.lift(sol[0], 0)
    S = pr.params.W - 1
    assert q.shape == (2 * 2 * S + 1, 7)
    np.testing.assert_array_equal(q[0], pr.robot.q_home)
    m = S // 2
    for s in range(4):
        qa, qv, qb = q[s * S], q[s * S + m], q[(s + 1) * S]
        for j in range(1, m):
            np.testing.assert_allclose(q[s * S + j], qa + (j / m) * (qv - qa), atol=1e-12)
        for j in range(m + 1, S):
            np.testing.assert_allclose(q[s * S + j], qv + ((j - m) / (S - m)) * (qb - qv), atol=1e-12)
    for b in range(2):
        _, T = orc.fk(q[(2 * b + 1) * S])
        top = pr.scene.init[b, :3] + np.array([0, 0, H])
        assert np.linalg.norm(T[:3, 3] - top) < 5e-3
        assert T[2, 2] < -0.99


def test_descend_schedule_endpoints():
    """eta = eta_init (1 - k/K_lin): with K_lin = 1 the only step has eta = 0, so only the
    clamp acts; with alpha = 0 the quadratic steps do nothing."""
    pr = scenes.make_problem("tower4", seed=4)
    orc = O.Oracle(pr, alpha=0.0)
    x = orc.place_sample(8)
    x[:, :, 3] = np.clip(x[:, :, 3], -3.0, 3.0)
    y = orc.place_descend(x, 1, 3)
    np.testing.assert_array_equal(y, x)


def test_place_solve_returns_satisfying_ranked():
    pr = scenes.make_problem("tower4", seed=0, N=1024, M=256)
    orc = O.Oracle(pr, n_threads=4)
    sol, attempts, steps = orc.place_solve()
    assert len(sol) == pr.params.P and attempts >= 1
    costs = [orc.place_cost(x, quad=True, grad=False)[0] for x in sol]
    assert all(orc.place_check(x)[0] for x in sol)
    assert costs == sorted(costs)
