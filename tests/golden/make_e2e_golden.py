"""Writes the oracle side of the end-to-end distribution tests (tests/golden/e2e_*.json).

For each seed of a workload it runs the FP64 oracle's whole method: the stage-1 loop of
Alg. 1 (sample, elite top-M, K_lin linear and K_quad quadratic steps, satisfying filter, best
P, retries) and stage 2 (lift, augmented-Lagrangian trajectory descent, satisfying filter,
best P, retries).  It stores per seed the number of solutions found, their rank costs in
ascending order and the attempt counts.  Only the oracle and the seeded scene generator are
called.

    python tests/golden/make_e2e_golden.py tower1 --seeds 100
    python tests/golden/make_e2e_golden.py tower4 --seeds 100 --override Q=64
    python tests/golden/make_e2e_golden.py p2p --seeds 100 --override Q=64 --override max_steps=1000
    python tests/golden/make_e2e_golden.py tower1 --seeds 100 --override ik_mode=1
    python tests/golden/make_e2e_golden.py tower4 --seeds 50 --override Q=64 --override ik_mode=1
    python tests/golden/make_e2e_golden.py tower10 --seeds 100 --override Q=64 --override ik_mode=1
    python tests/golden/make_e2e_golden.py tetris5 --seeds 100 --override N=2048 --override M=512 --override max_steps=3000

ik_mode=1 lifts with the analytic IK of the Franka joint layout instead of damped least squares.

For the point-to-point workload (one transit segment to a tool target) only stage 2 runs; for
the packing workloads (the appendix's Tetris problem) only stage 1, and the stored costs are the
stage-1 costs of the returned placements.

The 4- and 10-block cases keep their scenes, stage-1 sizes and waypoint counts, and reduce the
number of trajectory particles to 64 so that the FP64 all-pairs oracle finishes a seed in seconds
(4 blocks) or about a minute (10 blocks, 64 cuboids, 621 configurations) on 8 cores.
"""
import argparse
import json

import numpy as np
import os
import sys
import time

ROOT = os.path.abspath(os.path.join(os.path.dirname(__file__), "..", ".."))
sys.path.insert(0, ROOT)

from oracle.oracle import Oracle  # noqa: E402
from paper_2510_07674_gb300 import scenes  # noqa: E402


def parse_overrides(items):
    out = {}
    for it in items:
        k, v = it.split("=", 1)
        out[k] = float(v) if any(c in v for c in ".e") else int(v)
    return out


def run_seed(name, seed, overrides, threads):
    if name in scenes.PACKINGS:
        wl = scenes.make_packing(name, seed=seed, **overrides)
        o = Oracle(wl, n_threads=threads)
        place, place_attempts, _ = o.place_solve()
        cost = sorted(float(o.place_cost(x, grad=False)[0]) for x in place)
        return {"seed": seed, "n_place": int(len(place)), "n_found": int(len(place)), "cost": cost,
                "place_attempts": int(place_attempts), "traj_attempts": 0}
    if name in scenes.P2P:
        wl = scenes.make_p2p(name, seed=seed, **overrides)
        o = Oracle(wl, n_threads=threads)
        q, cost, traj_attempts = o.traj_solve(np.zeros((1, 1, 4)))
        return {"seed": seed, "n_place": 1, "n_found": int(len(cost)), "cost": [float(c) for c in cost],
                "place_attempts": 0, "traj_attempts": int(traj_attempts)}
    wl = scenes.make_problem(name, seed=seed, **overrides)
    o = Oracle(wl, n_threads=threads)
    place, place_attempts, place_steps = o.place_solve()
    if len(place) == 0:
        return {"seed": seed, "n_place": 0, "n_found": 0, "cost": [], "place_attempts": place_attempts,
                "traj_attempts": 0}
    q, cost, traj_attempts = o.traj_solve(place)
    return {"seed": seed, "n_place": int(len(place)), "n_found": int(len(cost)), "cost": [float(c) for c in cost],
            "place_attempts": int(place_attempts), "traj_attempts": int(traj_attempts)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("workload")
    ap.add_argument("--seeds", type=int, default=100)
    ap.add_argument("--override", action="append", default=[], metavar="PARAM=VALUE")
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    overrides = parse_overrides(args.override)
    tag = args.workload + "".join(f"_{k}{v}" for k, v in sorted(overrides.items()))
    out = args.out or os.path.join(os.path.dirname(__file__), f"e2e_{tag}.json")
    rows = []
    if os.path.exists(out):   # resume
        with open(out) as f:
            rows = json.load(f)["seeds"]
    done = {r["seed"] for r in rows}
    for seed in range(args.seeds):
        if seed in done:
            continue
        t = time.time()
        rows.append(run_seed(args.workload, seed, overrides, args.threads))
        print(f"seed {seed}: found {rows[-1]['n_found']} best "
              f"{rows[-1]['cost'][0] if rows[-1]['cost'] else None} ({time.time() - t:.1f} s)", flush=True)
        rows.sort(key=lambda r: r["seed"])
        with open(out, "w") as f:
            json.dump({"workload": args.workload, "overrides": overrides,
                       "source": "oracle/ (FP64), tests/golden/make_e2e_golden.py", "seeds": rows}, f, indent=0)


if __name__ == "__main__":
    main()
