"""Batched form (spasm_optimize_batch): every problem of a heterogeneous batch ends with exactly
the result that spasm_optimize gives it alone, under any schedule of the persistent
trajectory launch, and the autotuner returns one of its candidate schedules."""
import numpy as np
import pytest

from paper_2510_07674_gb300 import scenes
from paper_2510_07674_gb300 import spasm as S


def mixed_workloads():
    """Problems of differing block, obstacle, particle and waypoint counts (small enough to run quickly)."""
    out = []
    for i, (B, O, Q, W) in enumerate([(1, 8, 300, 16), (3, 20, 517, 32), (2, 40, 1024, 24), (4, 12, 256, 32),
                                      (1, 64, 130, 12)]):
        out.append(scenes.make_problem("tower4", seed=40 + i, B=B, O=O, Q=Q, W=W, N=1024, M=256))
    return out


def solve_alone(wl, sphere_tiling=0, particles_per_cta=1):
    pr = S.Problem(wl)
    try:
        S.spasm_set_kernel_config(pr, sphere_tiling, particles_per_cta)
        S.spasm_optimize(pr)
        return S.spasm_result(pr, allow_empty=True)
    finally:
        pr.close()


def same(a, b):
    assert a["n_found"] == b["n_found"]
    for key in ("placements", "traj", "cost", "success"):
        np.testing.assert_array_equal(a[key], b[key], err_msg=key)


@pytest.mark.gpu
@pytest.mark.parametrize("config", [None, {"per_fetch": 3, "ctas_per_sm": 1, "order": 1},
                                    {"per_fetch": 1, "ctas_per_sm": 0, "order": 0}])
def test_batch_equals_alone(config):
    import torch
    wls = mixed_workloads()
    alone = [solve_alone(wl) for wl in wls]
    stream = torch.cuda.Stream()
    prs = [S.Problem(wl) for wl in wls]
    try:
        S.spasm_optimize_batch(prs, stream=stream.cuda_stream, config=config)
        batch = [S.spasm_result(p, allow_empty=True) for p in prs]
    finally:
        for p in prs:
            p.close()
    assert all(r["n_found"] > 0 for r in alone)
    for a, b in zip(alone, batch):
        same(a, b)


@pytest.mark.gpu
def test_autotune_returns_a_candidate_and_keeps_results():
    import torch
    wls = mixed_workloads()[:3]
    stream = torch.cuda.Stream()
    prs = [S.Problem(wl) for wl in wls]
    try:
        best = S.spasm_batch_autotune(prs, stream=stream.cuda_stream)
        assert best["per_fetch"] in (1, 2, 4) and best["ctas_per_sm"] in (0, 1) and best["order"] in (0, 1)
        assert best["sphere_tiling"] in (0, 1) and best["particles_per_cta"] in (1, 2)
        assert best["ms"] > 0
        # the problems are placed by the tuner; the tuned batch equals the plain solve with the
        # same launch shape (the sphere tiling reorders float sums)
        S.spasm_optimize_batch(prs, stream=stream.cuda_stream, config=best)
        batch = [S.spasm_result(p, allow_empty=True) for p in prs]
    finally:
        for p in prs:
            p.close()
    for wl, b in zip(wls, batch):
        same(solve_alone(wl, best["sphere_tiling"], best["particles_per_cta"]), b)


@pytest.mark.gpu
def test_batch_rejects_default_stream_and_duplicates():
    wl = mixed_workloads()[0]
    pr = S.Problem(wl)
    try:
        with pytest.raises(ValueError):
            S.spasm_optimize_batch([pr], stream=0)
        import torch
        with pytest.raises(S.SpasmError):
            S.spasm_optimize_batch([pr, pr], stream=torch.cuda.Stream().cuda_stream)
    finally:
        pr.close()
