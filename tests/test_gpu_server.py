"""Continuous batching: every request's result is the same solved alone and in the mix."""
import numpy as np
import pytest

from paper_2510_07674_gb300 import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_results_alone_equal_results_in_the_mix():
    from paper_2510_07674_gb300 import spasm as S
    wls = [scenes.make_problem("tower1", seed=s) for s in range(3)] + \
          [scenes.make_problem("tower4", seed=s, Q=512, N=1024, M=256) for s in range(3)]
    alone = []
    for wl in wls:
        pr = S.Problem(wl)
        S.spasm_optimize(pr)
        alone.append(S.spasm_result(pr))
        pr.close()
    sv = S.Server(budget_bytes=8 << 30, max_inflight=4)
    tickets = [S.spasm_server_submit(sv, wl) for wl in wls]
    for t in tickets:
        S.spasm_server_wait(sv, t, 300.0)
    mix = [S.spasm_server_result(sv, t) for t in tickets]
    sv.close()
    for i, (a, m) in enumerate(zip(alone, mix)):
        assert m["status"] == 0 and m["n_found"] == a["n_found"], (i, m["status"])
        for key in ("traj", "cost", "placements", "success"):
            x, y = np.asarray(m[key], float), np.asarray(a[key], float)
            assert x.shape == y.shape and np.array_equal(x, y), (i, key, np.abs(x - y).max() if x.shape == y.shape else None)
    assert all(m["latency_ms"] > 0 for m in mix)
