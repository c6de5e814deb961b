"""Checkpoint and resume: a snapshot restored into a fresh problem built from the same inputs
returns the same placements and solutions; a snapshot taken between the stages resumes with
stage 2 only and gives the same solutions as the uninterrupted solve; snapshots of another
problem, truncated or corrupted ones are refused."""
import numpy as np
import pytest

from paper_2510_07674_gb300 import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _S():
    from paper_2510_07674_gb300 import spasm as S
    return S


def _wl(seed=3):
    return scenes.make_problem("tower4", seed=seed, Q=256, N=1024, M=256)


def _same(a, b):
    assert a["n_found"] == b["n_found"]
    for key in ("placements", "traj", "cost", "success"):
        assert np.array_equal(np.asarray(a[key]), np.asarray(b[key])), key


def test_restored_solve_returns_the_same_results():
    S = _S()
    a = S.Problem(_wl())
    b = S.Problem(_wl())
    try:
        S.spasm_optimize(a)
        ra = S.spasm_result(a)
        snap = S.spasm_snapshot(a)
        assert len(snap) == S.spasm_snapshot_bytes(a)
        S.spasm_restore(b, snap)
        _same(ra, S.spasm_result(b))
        pa, pb = S.spasm_placements(a), S.spasm_placements(b)
        assert pa["n_place"] == pb["n_place"] and np.array_equal(pa["placements"], pb["placements"])
    finally:
        a.close()
        b.close()


def test_snapshot_between_the_stages_resumes_with_stage_2():
    S = _S()
    full, first, resumed = S.Problem(_wl()), S.Problem(_wl()), S.Problem(_wl())
    try:
        S.spasm_optimize(full)
        r_full = S.spasm_result(full)
        S.spasm_place(first)
        snap = S.spasm_snapshot(first)
        S.spasm_restore(resumed, snap)
        S.spasm_reset_stats(resumed)
        S.spasm_optimize(resumed)           # stage 2 only: stage 1 comes from the snapshot
        r = S.spasm_result(resumed)
        st = S.spasm_get_stats(resumed)
        assert st["place_attempts"] == 0 and st["traj_attempts"] >= 1
        _same(r_full, r)
    finally:
        for p in (full, first, resumed):
            p.close()


def test_restore_refuses_another_problem_and_damaged_snapshots():
    S = _S()
    a = S.Problem(_wl(3))
    other_scene = S.Problem(_wl(4))                                        # other obstacles
    other_size = S.Problem(scenes.make_problem("tower4", seed=3, B=3, O=12, W=8, Q=256, N=1024, M=256))
    try:
        S.spasm_optimize(a)
        snap = S.spasm_snapshot(a)
        for target in (other_scene, other_size):
            with pytest.raises(S.SpasmError) as e:
                S.spasm_restore(target, snap)
            assert e.value.status == -1
        for bad in (snap[:-1], snap[:50], bytes(snap[:200]) + bytes([snap[200] ^ 1]) + bytes(snap[201:])):
            with pytest.raises(S.SpasmError) as e:
                S.spasm_restore(a, bad)
            assert e.value.status == -1
        S.spasm_restore(a, snap)   # the intact snapshot still loads
    finally:
        for p in (a, other_scene, other_size):
            p.close()
