"""Pins of the oracle's packing cost (the appendix's Tetris problem) against closed forms,
special cases and central differences; no GPU."""
import math

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2510_07674_gb300 import scenes

U = scenes.CELL


def one_cell(**kw):
    return scenes.packing_problem([[(0, 0)]], 1, 1, **kw)


def domino(**kw):
    return scenes.packing_problem([[(0, 0)], [(1, 0)]], 2, 1, **kw)


@pytest.mark.parametrize("name", ["tetris5", "tetris8"])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_planted_tiling_has_zero_cost_and_satisfies(name, seed):
    pb = scenes.make_packing(name, seed=seed)
    o = Oracle(pb)
    x = pb.packing.planted
    c, g, t = o.place_cost(x)
    assert c < 1e-12 and t[2] < 1e-12
    ok, m = o.place_check(x)
    assert ok and m[0] < 1e-12 and m[2] == 0.0


@pytest.mark.parametrize("name", ["tetris5", "tetris8"])
def test_generator_tiles_the_region_exactly(name):
    pb = scenes.make_packing(name, seed=4)
    pk = pb.packing
    x_lo, y_lo, x_hi, y_hi = pk.region
    gx, gy = round((x_hi - x_lo) / U), round((y_hi - y_lo) / U)
    seen = np.zeros((gx, gy), int)
    start = np.concatenate([[0], np.cumsum(pk.n_cells)])
    for b, (px, py, _, yaw) in enumerate(pk.planted):
        c, s = math.cos(yaw), math.sin(yaw)
        for ox, oy in pk.cell[start[b]:start[b + 1]]:
            wx, wy = px + c * ox - s * oy, py + s * ox + c * oy
            ix, iy = (wx - x_lo) / U - 0.5, (wy - y_lo) / U - 0.5
            assert abs(ix - round(ix)) < 1e-9 and abs(iy - round(iy)) < 1e-9
            seen[round(ix), round(iy)] += 1
    assert (seen == 1).all()


@pytest.mark.parametrize("delta", [5e-4, 4e-3])
def test_cube_pushed_into_a_wall(delta):
    # the 4 spheres on the wall side are tangent to the wall face: each penetrates delta
    pb = one_cell()
    o = Oracle(pb)
    for axis, sign in ((0, -1), (0, 1), (1, -1), (1, 1)):
        x = pb.packing.planted.copy()
        x[0, axis] += sign * delta
        c, _, t = o.place_cost(x)
        assert abs(t[2] - 4 * delta) < 1e-12 and abs(c - pb.params.w_coll * 4 * delta) < 1e-12
        cq, _, tq = o.place_cost(x, quad=True)
        assert abs(tq[2] - 4 * delta ** 2) < 1e-15
        ok, m = o.place_check(x)
        assert abs(m[0] - delta) < 1e-12 and ok == (delta <= pb.params.eps)


def test_overlapping_cubes_penetrate_by_the_overlap():
    # block 1 slides into block 0 by delta: its 4 spheres facing block 0 penetrate delta each
    # and it leaves the right wall; block 0 is untouched
    pb = domino()
    o = Oracle(pb)
    delta = 3e-3
    x = pb.packing.planted.copy()
    x[1, 0] -= delta
    _, g, t = o.place_cost(x)
    assert abs(t[2] - 4 * delta) < 1e-12
    # the pair pushes block 1 back (+x) and block 0 away (-x), each with weight 4
    assert g[1, 0] == pytest.approx(-4.0 * pb.params.w_coll, abs=1e-9)
    assert g[0, 0] == pytest.approx(4.0 * pb.params.w_coll, abs=1e-9)


@pytest.mark.parametrize("theta", [0.05, -0.12, 0.3])
def test_turned_cube_in_a_tight_cell_against_half_spaces(theta):
    # a cube turned by theta inside walls that fit it exactly: every sphere centre
    # (+-u/4, +-u/4) turns, and against a wall (a half-space along its normal) a sphere of
    # radius u/4 penetrates by max(0, |coordinate| + u/4 - u/2) when it is on that side
    pb = one_cell()
    o = Oracle(pb)
    x = pb.packing.planted.copy()
    x[0, 3] = theta
    c, s, q = math.cos(theta), math.sin(theta), U / 4
    expect = 0.0
    for sx in (-1, 1):
        for sy in (-1, 1):
            px, py = c * sx * q - s * sy * q, s * sx * q + c * sy * q
            for v in (px, py):
                expect += 2 * max(0.0, abs(v) + q - U / 2)   # two spheres (z = +-u/4) per xy position
    _, _, t = o.place_cost(x)
    assert abs(t[2] - expect) < 1e-12, (t[2], expect)


def test_height_term_is_absolute_and_weighted():
    pb = one_cell(z_span=0.1, w_height=7.0)
    o = Oracle(pb)
    x = pb.packing.planted.copy()
    x[0, 2] += 0.043
    c, g, t = o.place_cost(x)
    assert abs(t[1] - 0.043) < 1e-15 and abs(c - 7.0 * 0.043) < 1e-12
    assert g[0, 2] == pytest.approx(7.0)
    ok, m = o.place_check(x)
    assert not ok and abs(m[2] - 0.043) < 1e-15   # above eps


@pytest.mark.parametrize("quad", [False, True])
def test_gradient_matches_central_differences(quad):
    pb = scenes.make_packing("tetris5", seed=6, zspan=0.02)
    o = Oracle(pb)
    rng = np.random.default_rng(1)
    checked = 0
    for trial in range(6):
        x = pb.packing.planted.copy()
        x[:, :2] += rng.normal(0, 0.006, (pb.packing.planted.shape[0], 2))
        x[:, 2] += rng.uniform(0.001, 0.01, len(x))
        x[:, 3] += rng.normal(0, 0.05, len(x))
        c, g, t = o.place_cost(x, quad=quad)
        assert t[2] > 0
        h = 1e-6
        fd = np.zeros_like(x)
        for i in range(x.shape[0]):
            for k in range(4):
                xp, xm = x.copy(), x.copy()
                xp[i, k] += h
                xm[i, k] -= h
                fd[i, k] = (o.place_cost(xp, quad=quad, grad=False)[0] - o.place_cost(xm, quad=quad, grad=False)[0]) / (2 * h)
        np.testing.assert_allclose(g, fd, rtol=1e-5, atol=1e-6)
        checked += 1
    assert checked == 6
