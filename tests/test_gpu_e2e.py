"""End-to-end parity of the whole method (both stages of Alg. 1 with retries, lift, trajectory
descent, final FP64 check) against the FP64 oracle, as distributions over seeds.

The oracle side is stored in tests/golden/e2e_*.json, written by make_e2e_golden.py from
oracle/ alone.  Per-iteration parity is element-wise (test_gpu_stage1/2); here FP32 and FP64
can reorder near-ties in the elite and best-P selections, so the criterion is distributional:
the success rate over the seeds and a two-sample Kolmogorov-Smirnov test on the best rank cost
of each seed.  Both sides draw the same Philox streams, so most seeds agree closely; the test
also reports that agreement and requires it for the median seed.
"""
import json
import os

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2510_07674_gb300 import scenes
from paper_2510_07674_gb300 import spasm as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
CASES = ["e2e_tower10_Q64_ik_mode1.json", "e2e_tower1_ik_mode1.json", "e2e_tower4_Q64_ik_mode1.json",
         "e2e_p2p_Q64_ik_mode1_max_steps1000.json", "e2e_tower1_ik_mode0.json", "e2e_tower4_Q64_ik_mode0.json",
         "e2e_p2p_Q64_ik_mode0_max_steps1000.json"]


def gpu_best(workload, seed, overrides):
    """(solved, best rank cost among solutions that pass the FP64 check) of one GPU solve."""
    make = scenes.make_p2p if workload in scenes.P2P else scenes.make_problem
    pr = S.Problem(make(workload, seed=seed, **overrides))
    try:
        try:
            S.spasm_optimize(pr)
        except S.SpasmError as e:
            if "NOSOLUTION" not in str(e):
                raise
        r = S.spasm_result(pr, allow_empty=True)
    finally:
        pr.close()
    ok = r["success"] != 0
    if not ok.any():
        return False, np.nan, r["n_found"] > 0
    return True, float(np.min(r["cost"][ok])), True


@pytest.mark.gpu
@pytest.mark.parametrize("fname", CASES)
def test_success_rate_and_cost_distribution_match_oracle(fname):
    stats = pytest.importorskip("scipy.stats")
    with open(os.path.join(GOLDEN, fname)) as f:
        g = json.load(f)
    rows = g["seeds"]
    assert len(rows) >= 30, "golden file holds too few seeds"
    o_ok = np.array([r["n_found"] > 0 for r in rows])
    o_best = np.array([r["cost"][0] if r["cost"] else np.nan for r in rows])
    res = [gpu_best(g["workload"], r["seed"], g["overrides"]) for r in rows]
    g_ok = np.array([a for a, _, _ in res])
    g_best = np.array([b for _, b, _ in res])
    rejected = sum(1 for a, _, f in res if f and not a)   # FP32-satisfying, refused by the FP64 check

    rate_o, rate_g = o_ok.mean(), g_ok.mean()
    both = o_ok & g_ok
    rel = np.abs(g_best[both] - o_best[both]) / np.maximum(np.abs(o_best[both]), 1e-12)
    ks = stats.ks_2samp(g_best[g_ok], o_best[o_ok])
    # paired sign test: on seeds both sides solve and whose best costs differ by more than the
    # float32 rounding of the reported cost (1e-4 relative), the GPU's is above the oracle's
    # about as often as below (no systematic difference between the two descents)
    d = (g_best[both] - o_best[both]) / np.maximum(np.abs(o_best[both]), 1e-12)
    above, below = int(np.sum(d > 1e-4)), int(np.sum(d < -1e-4))
    sign_p = stats.binomtest(above, above + below, 0.5).pvalue if above + below > 0 else 1.0
    print(f"{fname}: seeds {len(rows)}, success oracle {rate_o:.3f} gpu {rate_g:.3f} "
          f"(both {int((o_ok & g_ok).sum())}, oracle only {int((o_ok & ~g_ok).sum())}, gpu only "
          f"{int((~o_ok & g_ok).sum())}, FP64-refused {rejected}), KS p {ks.pvalue:.3f}, sign test p {sign_p:.3f} "
          f"({above} above / {below} below), "
          f"per-seed rel. diff of best cost: median {np.median(rel):.2e}, p90 {np.quantile(rel, 0.9):.2e}")
    # success rates: a 3-sigma band of two binomial proportions (FP32 and FP64 descents can
    # reach different minima where a seed is hard), which shrinks to one seed at 100%
    n = len(rows)
    p_bar = 0.5 * (rate_o + rate_g)
    assert abs(rate_g - rate_o) <= 3.0 * np.sqrt(2.0 * p_bar * (1.0 - p_bar) / n) + 1.0 / n, (rate_o, rate_g)
    # final-cost distributions indistinguishable, and no systematic difference seed by seed
    assert ks.pvalue > 0.01, ks
    assert sign_p > 0.01, (above, below)
    # same Philox streams: the typical seed ends at (nearly) the same best solution.  The
    # 10-block tower descends 621 configurations among 74 obstacles for 50 steps: contacts
    # switch on or off at different steps in FP32 and FP64, and the best of 64 particles ends a
    # few percent apart (the distributions and the sign test above show no bias)
    bound = 1e-1 if "tower10" in fname else 1e-2
    assert np.median(rel) < bound, np.median(rel)


PACK_CASES = ["e2e_tetris5_M512_N2048_max_steps3000.json"]


def gpu_pack(workload, seed, overrides):
    """(solved, best FP64 stage-1 cost of the returned placements, attempts) of one GPU
    packing solve (stage 1 of Alg. 1); the costs are evaluated by the oracle."""
    wl = scenes.make_packing(workload, seed=seed, **overrides)
    pr = S.Problem(wl)
    try:
        try:
            S.spasm_place(pr)
        except S.SpasmError as e:
            if "NOSOLUTION" not in str(e):
                raise
        r = S.spasm_placements(pr, allow_empty=True)
        attempts = S.spasm_get_stats(pr)["place_attempts"]
    finally:
        pr.close()
    if r["n_place"] == 0:
        return False, np.nan, attempts
    o = Oracle(wl)
    return True, min(o.place_cost(x, grad=False)[0] for x in r["placements"]), attempts


@pytest.mark.gpu
@pytest.mark.parametrize("fname", PACK_CASES)
def test_packing_success_attempts_and_cost_match_oracle(fname):
    """The appendix's packing problem, stage 1 end to end: success rate, attempts until the
    first satisfying packing and the best stage-1 cost, GPU against the FP64 oracle over
    seeds (same Philox streams: the typical seed succeeds at the same attempt with nearly the
    same packing)."""
    stats = pytest.importorskip("scipy.stats")
    with open(os.path.join(GOLDEN, fname)) as f:
        g = json.load(f)
    rows = g["seeds"]
    assert len(rows) >= 30, "golden file holds too few seeds"
    o_ok = np.array([r["n_found"] > 0 for r in rows])
    o_best = np.array([r["cost"][0] if r["cost"] else np.nan for r in rows])
    o_att = np.array([r["place_attempts"] for r in rows])
    res = [gpu_pack(g["workload"], r["seed"], g["overrides"]) for r in rows]
    g_ok = np.array([a for a, _, _ in res])
    g_best = np.array([b for _, b, _ in res])
    g_att = np.array([c for _, _, c in res])
    both = o_ok & g_ok
    rel = np.abs(g_best[both] - o_best[both]) / np.maximum(np.abs(o_best[both]), 1e-12)
    ks = stats.ks_2samp(g_best[g_ok], o_best[o_ok])
    same_att = np.mean(g_att[both] == o_att[both])
    print(f"{fname}: seeds {len(rows)}, success oracle {o_ok.mean():.3f} gpu {g_ok.mean():.3f}, same attempt "
          f"{same_att:.2f}, mean attempts oracle {o_att.mean():.2f} gpu {g_att.mean():.2f}, KS p {ks.pvalue:.3f}, "
          f"per-seed rel. diff of best cost: median {np.median(rel):.2e}")
    n = len(rows)
    p_bar = 0.5 * (o_ok.mean() + g_ok.mean())
    assert abs(g_ok.mean() - o_ok.mean()) <= 3.0 * np.sqrt(2.0 * p_bar * (1.0 - p_bar) / n) + 1.0 / n
    assert ks.pvalue > 0.01, ks
    assert same_att >= 0.5, same_att
    # a packing's cost sums many penetrations just under eps; over the 30 descent steps a contact
    # switching on or off at rounding level moves that sum by a few percent while both packings
    # satisfy, so the per-seed bound is looser than for the trajectory costs
    assert np.median(rel) < 5e-2, np.median(rel)
