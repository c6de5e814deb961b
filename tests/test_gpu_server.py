"""Solver service with continuous batching: each request's result is the same alone and in the
mix, epochs batch several requests, a request that does not fit the memory budget beside the
running ones waits for them and then runs, and a queued request can be cancelled."""
import time

import numpy as np
import pytest

from paper_2510_07674_gb300 import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _S():
    from paper_2510_07674_gb300 import spasm as S
    return S


def _alone(wls):
    S = _S()
    out = []
    for wl in wls:
        pr = S.Problem(wl)
        S.spasm_optimize(pr)
        out.append(S.spasm_result(pr))
        pr.close()
    return out


def _same(a, m, i):
    assert m["status"] == 0 and m["n_found"] == a["n_found"], (i, m["status"])
    for key in ("traj", "cost", "placements", "success"):
        x, y = np.asarray(m[key], float), np.asarray(a[key], float)
        assert x.shape == y.shape and np.array_equal(x, y), (i, key, np.abs(x - y).max() if x.shape == y.shape else None)


def test_results_alone_equal_results_in_the_mix():
    S = _S()
    wls = [scenes.make_problem("tower1", seed=s) for s in range(3)] + \
          [scenes.make_problem("tower4", seed=s, Q=512, N=1024, M=256) for s in range(3)]
    alone = _alone(wls)
    sv = S.Server(budget_bytes=8 << 30, max_inflight=4)
    tickets = [S.spasm_server_submit(sv, wl) for wl in wls]
    for t in tickets:
        S.spasm_server_wait(sv, t, 300.0)
    mix = [S.spasm_server_result(sv, t) for t in tickets]
    st = S.spasm_server_get_stats(sv)
    sv.close()
    for i, (a, m) in enumerate(zip(alone, mix)):
        _same(a, m, i)
    assert all(m["latency_ms"] > 0 for m in mix)
    # the epochs batched several requests at once
    assert st["completed"] == len(wls) and st["requests_in_epochs"] > st["epochs"], st


def test_request_over_the_remaining_budget_waits_then_runs():
    S = _S()
    a_wl = scenes.make_problem("tower4", seed=0, Q=1024)
    b_wl = scenes.make_problem("tower4", seed=1, Q=1024)
    need_a, need_b = S.spasm_problem_bytes(a_wl), S.spasm_problem_bytes(b_wl)
    alone = _alone([a_wl, b_wl])
    sv = S.Server(budget_bytes=need_a + need_b - 1, max_inflight=8)   # either fits alone, not both
    try:
        t0 = time.perf_counter()
        ta = S.spasm_server_submit(sv, a_wl)
        tb = S.spasm_server_submit(sv, b_wl)
        gap_ms = (time.perf_counter() - t0) * 1e3
        S.spasm_server_wait(sv, ta, 300.0)
        S.spasm_server_wait(sv, tb, 300.0)
        ra, rb = S.spasm_server_result(sv, ta), S.spasm_server_result(sv, tb)
    finally:
        sv.close()
    _same(alone[0], ra, 0)
    _same(alone[1], rb, 1)
    # b was admitted only once a had finished and returned its memory
    assert rb["queue_ms"] + gap_ms >= ra["latency_ms"], (rb["queue_ms"], ra["latency_ms"], gap_ms)


def test_cancel_a_queued_request():
    S = _S()
    wls = [scenes.make_problem("tower1", seed=s) for s in range(3)]
    alone = _alone(wls[:2])
    sv = S.Server(budget_bytes=8 << 30, max_inflight=1)
    try:
        tickets = [S.spasm_server_submit(sv, wl) for wl in wls]
        S.spasm_server_cancel(sv, tickets[2])          # still queued behind the first two
        assert S.spasm_server_poll(sv, tickets[2]) == 3
        for t in tickets[:2]:
            S.spasm_server_wait(sv, t, 300.0)
        res = [S.spasm_server_result(sv, t) for t in tickets]
    finally:
        sv.close()
    _same(alone[0], res[0], 0)
    _same(alone[1], res[1], 1)
    assert res[2]["status"] == -7 and res[2]["n_found"] == 0
