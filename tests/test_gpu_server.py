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
    for a, m in zip(alone, mix):
        assert m["status"] == 0 and m["n_found"] == a["n_found"], m["status"]
        np.testing.assert_array_equal(m["traj"], a["traj"])
        np.testing.assert_array_equal(m["cost"], a["cost"])
        np.testing.assert_array_equal(m["placements"], a["placements"])
        np.testing.assert_array_equal(m["success"], a["success"])
    assert all(m["latency_ms"] > 0 for m in mix)
