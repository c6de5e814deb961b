"""Solver service, host-side failure handling (no GPU fault involved): bad requests are
refused at submission, a request whose problem is rejected at creation finishes with that
status, unknown tickets are errors and waits are bounded."""
import pytest

from paper_2510_07674_gb300 import build as Bld
from paper_2510_07674_gb300 import scenes


@pytest.fixture(scope="module")
def S():
    Bld.build()
    from paper_2510_07674_gb300 import spasm
    return spasm


def test_invalid_submission_refused(S):
    sv = S.Server(budget_bytes=1 << 30, max_inflight=2)
    try:
        with pytest.raises(S.SpasmError) as e:
            S.spasm_server_submit(sv, scenes.make_problem("tower1", seed=0, B=17))
        assert e.value.status == -1
        with pytest.raises(S.SpasmError):
            S.spasm_server_wait(sv, 12345, 0.1)
    finally:
        sv.close()


def test_rejected_problem_finishes_with_its_status(S):
    sv = S.Server(budget_bytes=1 << 30, max_inflight=1)
    try:
        t = S.spasm_server_submit(sv, scenes.make_problem("tower1", seed=0), M=300)   # M > N: rejected at creation
        S.spasm_server_wait(sv, t, 30.0)
        assert S.spasm_server_poll(sv, t) == 2
        res = S.spasm_server_result(sv, t)
        assert res["status"] == -1 and res["n_found"] == 0
        S.spasm_server_release(sv, t)
        with pytest.raises(S.SpasmError):
            S.spasm_server_poll(sv, t)
    finally:
        sv.close()
