"""The re-initialisation loops of both stages run on the device (Alg. 1 restarts until a
particle satisfies, Sec. III-A; max_steps caps the gradient steps, Sec. IV-C).

spasm_place / spasm_optimize enqueue one graph per stage whose conditional while node repeats
attempts; the host waits once, when it reads the outcome.  These tests count the host waits,
and compare the attempt counts the device loop reaches with those of the oracle's host loop
on cases that need several attempts: no satisfying particle at all (every attempt runs until
the cap), and stage 2 with an unreachable start tolerance.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2510_07674_gb300 import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _S():
    from paper_2510_07674_gb300 import spasm as S
    return S


def test_one_host_wait_per_solve():
    S = _S()
    wl = scenes.make_problem("tower1", seed=0)
    pr = S.Problem(wl)
    try:
        for seed in range(3):
            S.spasm_set_seed(pr, seed)
            S.spasm_reset_stats(pr)
            S.spasm_optimize(pr)          # enqueues both stages
            st = S.spasm_get_stats(pr)    # the one wait: reads the outcome
            assert st["host_waits"] == 1, st
            assert st["place_attempts"] >= 1 and st["traj_attempts"] >= 1
            r = S.spasm_result(pr)
            assert r["n_found"] > 0
    finally:
        pr.close()


def test_stage1_attempts_until_the_cap_match_oracle():
    """eps = 1e-9: no particle can satisfy, so both loops run attempts until the step budget
    (max_steps = 100 with K_lin + K_quad = 30 per attempt: 4 attempts) and keep nothing;
    stage 2 then does nothing on the device."""
    S = _S()
    wl = scenes.make_problem("tower4", seed=1, B=2, O=6, W=6, N=512, M=128, eps=1e-9, max_steps=100)
    orc = O.Oracle(wl, n_threads=4)
    sol, att_o, steps_o = orc.place_solve()
    assert len(sol) == 0 and att_o == math.ceil(100 / 30) and steps_o == 120
    pr = S.Problem(wl)
    try:
        S.spasm_reset_stats(pr)
        S.spasm_optimize(pr)
        r = S.spasm_result(pr, allow_empty=True)
        st = S.spasm_get_stats(pr)
        assert r["n_found"] == 0
        assert st["place_attempts"] == att_o
        assert st["traj_attempts"] == 0 and st["particle_iters"] == 0   # stage 2 skipped on the device
        assert st["host_waits"] == 2   # spasm_result's read of the outcome, and of its copies
        pl = S.spasm_placements(pr, allow_empty=True)
        assert pl["n_place"] == 0
    finally:
        pr.close()


def test_stage2_retries_match_oracle():
    """eps_start = 1e-30: stage 1 succeeds, but no trajectory can meet the grasp tolerance, so
    stage 2 re-lifts with attempt counters 0, 1, 2 until max_steps = 150 (K_traj = 50) and
    returns nothing, as the oracle's loop."""
    S = _S()
    wl = scenes.make_problem("tower1", seed=2, Q=8, P=4, eps_start=1e-30, max_steps=150)
    orc = O.Oracle(wl, n_threads=4)
    place, att1, _ = orc.place_solve()
    assert len(place) > 0 and att1 == 1
    q, cost, att2 = orc.traj_solve(place)
    assert len(cost) == 0 and att2 == 3
    pr = S.Problem(wl)
    try:
        S.spasm_reset_stats(pr)
        S.spasm_optimize(pr)
        st = S.spasm_get_stats(pr)
        assert st["host_waits"] == 1
        assert st["place_attempts"] == att1 and st["traj_attempts"] == att2
        assert st["particle_iters"] == 8 * 50 * att2
        r = S.spasm_result(pr, allow_empty=True)
        assert r["n_found"] == 0
    finally:
        pr.close()


def _solve(S, wl, eager, place_only=False):
    pr = S.Problem(wl)
    try:
        if eager:
            S.spasm_set_launch_mode(pr, S.SPASM_LAUNCH_EAGER)
        S.spasm_reset_stats(pr)
        if place_only:
            S.spasm_place(pr)
            out = S.spasm_placements(pr, allow_empty=True)
        else:
            S.spasm_optimize(pr)
            out = S.spasm_result(pr, allow_empty=True)
        return out, S.spasm_get_stats(pr)
    finally:
        pr.close()


@pytest.mark.parametrize("case", ["tower4", "cap", "retries", "p2p", "tetris5"])
def test_eager_mode_gives_the_same_bits_as_the_graphs(case):
    """The eager launch mode runs the graphs' kernels one at a time with the attempt loops on
    the host: the same results and counters, one host wait per attempt and stage."""
    S = _S()
    wl = {"tower4": lambda: scenes.make_problem("tower4", seed=3, Q=256, N=1024, M=256),
          "cap": lambda: scenes.make_problem("tower4", seed=1, B=2, O=6, W=6, N=512, M=128, eps=1e-9, max_steps=100),
          "retries": lambda: scenes.make_problem("tower1", seed=2, Q=8, P=4, eps_start=1e-30, max_steps=150),
          "p2p": lambda: scenes.make_p2p("p2p", seed=4, Q=64),
          "tetris5": lambda: scenes.make_packing("tetris5", seed=5, N=2048, M=512)}[case]()
    place_only = case == "tetris5"
    g, sg = _solve(S, wl, False, place_only)
    e, se = _solve(S, wl, True, place_only)
    assert g.keys() == e.keys()
    for key in g:
        assert np.array_equal(np.asarray(g[key]), np.asarray(e[key])), key
    for key in ("place_attempts", "traj_attempts", "particle_iters", "kernel_launches", "n_found", "n_success"):
        assert sg[key] == se[key], (key, sg[key], se[key])
    # the eager mode adds one wait per attempt of each stage to the result read's waits
    stage2 = 0 if place_only else max(se["traj_attempts"], 1)
    assert se["host_waits"] - sg["host_waits"] == se["place_attempts"] + stage2, (sg, se)
