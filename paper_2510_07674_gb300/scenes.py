"""Seeded synthetic workloads for the tower-stacking and the packing (Tetris) problems.

This module only *generates inputs*: a 7-revolute-joint arm described by modified
Denavit-Hartenberg rows and a set of collision spheres, a table, cuboid clutter,
blocks with their initial poses, a goal region and the solver parameters.  It holds
none of the method's arithmetic (no kinematics, no costs, no optimiser), so both the
CUDA path and the FP64 oracle consume exactly the same arrays.

The problem statement (Sec. III of the paper: known object geometry, initial poses,
environment obstacles and a given action skeleton; robot and objects as collections
of spheres) fixes *what* an input is; the paper's own scenes, the Franka model and its
sphere set are not available, so every instance here is synthetic and seeded:

* arm: Franka-like alternation of twist angles, seeded link lengths/offsets,
  52 spheres (base 4, links 1..7 = 3, 8, 6, 8, 7, 6, 10), radii 0.03-0.08 m on the
  arm links and 0.02-0.035 m on the wrist/gripper link;
* table: a 0.9 x 1.2 x 0.05 m cuboid whose top face is z = 0;
* blocks: 5 cm cubes resting on the table in a start region, seeded yaw;
* goal: a 0.3 x 0.3 m placement box on the other side of the table;
* clutter: cuboids with sides U(0.05, 0.3) m and uniform yaw, rejection-sampled to
  stay out of keep-out volumes (robot base, start region, a central tower column and
  a transport corridor), so that a solution is expected to exist.

Packing (the appendix's Tetris problem): blocks are polyominoes of unit cubes that must
fill a rectangular region on the floor, between four walls, at the resting height z*.
The generator tiles a gx x gy grid of cells with seeded random tetrominoes, so a packing
of zero cost exists (the planted one); each block's frame sits at the centroid of its
cells and is turned by a seeded multiple of 90 degrees.  No benchmark instance is
reproduced.

All arrays are float64 / int32 numpy arrays in row-major order.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict

import numpy as np

# sphere count per link (index 0 = fixed base), 52 in total
SPHERES_PER_LINK = (4, 3, 8, 6, 8, 7, 6, 10)
N_ARM_SPHERES = sum(SPHERES_PER_LINK)
BLOCK_HALF = 0.025

# Named workloads.  B blocks, O clutter cuboids (+ the table), N -> M stage-1
# sample/elite counts, Q trajectory particles, W waypoints per motion segment.
WORKLOADS: Dict[str, dict] = {
    # 1-block pick-and-place, 4 obstacles, 256 particles, 2 x 16 waypoints, 50 iters/stage
    "tower1": dict(B=1, O=4, N=256, M=64, P=8, Q=256, W=16, K_lin=40, K_quad=10, K_traj=50),
    # 4-block stacking, 20 obstacles, 4096 -> 1024 placement / 2048 trajectory particles, 8 x 32
    "tower4": dict(B=4, O=20, N=4096, M=1024, P=32, Q=2048, W=32, K_lin=25, K_quad=5, K_traj=50),
    # 10-block tower in clutter, 64 obstacles, 16384 -> 4096 / 4096 particles, 20 x 32
    "tower10": dict(B=10, O=64, N=16384, M=4096, P=32, Q=4096, W=32, K_lin=25, K_quad=5, K_traj=50),
}


@dataclasses.dataclass
class Robot:
    dh: np.ndarray            # (7, 4) a, alpha, d, theta_offset   (modified DH)
    qlim: np.ndarray          # (7, 2) lower, upper
    sphere_link: np.ndarray   # (S,) int32, 0 = base, k = link k
    sphere: np.ndarray        # (S, 4) x, y, z, r in the link frame
    ee: np.ndarray            # (4, 4) flange -> tool point transform
    q_home: np.ndarray        # (7,)


@dataclasses.dataclass
class Scene:
    cuboid: np.ndarray        # (n, 15) centre(3), R(9, row-major), half extents(3); row 0 = table
    sphere: np.ndarray        # (m, 4) centre(3), radius
    half: np.ndarray          # (B, 3) block half extents, in stack order
    init: np.ndarray          # (B, 4) initial x, y, z, yaw of each block, in stack order
    box: np.ndarray           # (6,) goal box lo(3), hi(3) on block centres
    z_table: float
    grasp_off: float


@dataclasses.dataclass
class Params:
    N: int = 256
    M: int = 64
    P: int = 8
    Q: int = 256
    W: int = 16
    K_lin: int = 25
    K_quad: int = 5
    K_traj: int = 50
    K_al: int = 10
    K_ik: int = 50
    eta_init: float = 0.03
    alpha: float = 0.002
    eta_traj: float = 0.01
    eps: float = 1e-3
    eps_start: float = 1e-4
    w_stable: float = 10.0
    w_height: float = 100.0
    w_coll: float = 1.0
    w_start: float = 10.0
    w_arm: float = 10.0
    w_block: float = 10.0
    w_path: float = 0.01
    w_jl: float = 10.0
    mu0: float = 1.0
    mu_max: float = 8.0
    ik_damp: float = 1e-2
    ik_mode: int = 1          # lift IK: 1 analytic (Franka joint layout, as the paper), 0 damped least squares
    seed: int = 0
    max_steps: int = 30000
    n_threads: int = 1


@dataclasses.dataclass
class Packing:
    n_cells: np.ndarray       # (B,) int32 unit cells of each block
    cell: np.ndarray          # (sum n_cells, 2) cell-centre offsets (x, y) in the block frame
    cell_size: float          # edge of the unit cubes
    region: np.ndarray        # (4,) x_lo, y_lo, x_hi, y_hi (inner faces of the walls)
    z_star: float             # resting height of the block centres
    planted: np.ndarray       # (B, 4) a zero-cost packing (the generator's tiling)


@dataclasses.dataclass
class Problem:
    name: str
    robot: Robot
    scene: Scene
    params: Params
    packing: "Packing | None" = None
    p2p: bool = False         # point-to-point: one segment from q_home to the target init[0]


def _rot_z(yaw: float) -> np.ndarray:
    c, s = math.cos(yaw), math.sin(yaw)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def make_robot(seed: int = 7) -> Robot:
    """A seeded Franka-like 7-R arm: modified DH rows, limits, 52 link spheres."""
    rng = np.random.default_rng(np.random.SeedSequence([0x5A5A, seed]))
    hp = math.pi / 2
    alpha = np.array([0.0, -hp, hp, hp, -hp, hp, hp])
    a = np.zeros(7)
    a[3] = rng.uniform(0.07, 0.09)
    a[4] = -rng.uniform(0.07, 0.09)
    a[6] = rng.uniform(0.07, 0.09)
    d = np.zeros(7)
    d[0] = rng.uniform(0.31, 0.35)
    d[2] = rng.uniform(0.30, 0.33)
    d[4] = rng.uniform(0.36, 0.40)
    dh = np.stack([a, alpha, d, np.zeros(7)], axis=1)

    qlim = np.empty((7, 2))
    for k in range(7):
        span = rng.uniform(2.6, 2.9)
        qlim[k] = (-span, span)
    qlim[1] = (-rng.uniform(1.7, 1.8), rng.uniform(1.7, 1.8))
    qlim[3] = (-rng.uniform(2.9, 3.05), -0.07)
    qlim[5] = (-0.0175, rng.uniform(3.6, 3.75))
    q_home = np.array([0.0, -0.5, 0.0, -2.2, 0.0, 1.7, 0.785])

    tool_len = rng.uniform(0.19, 0.21)
    ee = np.eye(4)
    ee[2, 3] = tool_len

    # Frame l+1's origin expressed in frame l under modified DH rows
    # (input geometry only: where a link ends, to lay its spheres along it).
    def next_origin(l):
        if l == 0:
            return np.array([0.0, 0.0, d[0]])
        if l == 7:
            return np.array([0.0, 0.0, tool_len - 0.06])
        al, aa, dd = alpha[l], a[l], d[l]
        return np.array([aa, -dd * math.sin(al), dd * math.cos(al)])

    links, spheres = [], []
    for l, n in enumerate(SPHERES_PER_LINK):
        end = next_origin(l)
        start = np.zeros(3)
        if l == 7:
            start = np.array([0.0, 0.0, -0.02])
        for i in range(n):
            t = (i + 0.5) / n
            c = start + t * (end - start) + rng.uniform(-0.015, 0.015, 3)
            if l == 7:
                r = rng.uniform(0.02, 0.035)
                c[:2] = rng.uniform(-0.03, 0.03, 2)
            elif l == 0:
                r = rng.uniform(0.06, 0.08)
            else:
                r = rng.uniform(0.04, 0.08)
            links.append(l)
            spheres.append([c[0], c[1], c[2], r])
    return Robot(dh=dh, qlim=qlim, sphere_link=np.array(links, np.int32),
                 sphere=np.array(spheres), ee=ee, q_home=q_home)


def _boxes_overlap(c1, h1, c2, h2, margin=0.0) -> bool:
    return bool(np.all(np.abs(np.asarray(c1) - np.asarray(c2)) < np.asarray(h1) + np.asarray(h2) + margin))


def make_scene(B: int, O: int, seed: int, n_obstacle_spheres: int = 0) -> Scene:
    """A seeded tower scene: table, B blocks in a start region, O clutter cuboids."""
    rng = np.random.default_rng(np.random.SeedSequence([0x70E5, B, O, seed]))
    z_table = 0.0
    table = np.concatenate([[0.55, 0.0, -0.025], np.eye(3).ravel(), [0.45, 0.6, 0.025]])

    # blocks on a jittered grid in the start region (positive y)
    half = np.full((B, 3), BLOCK_HALF)
    cols = 4
    init = np.zeros((B, 4))
    slots = rng.permutation(max(B, 12))[:B]
    for i, s in enumerate(slots):
        r, c = divmod(int(s), cols)
        init[i, 0] = 0.36 + 0.09 * c + rng.uniform(-0.01, 0.01)
        init[i, 1] = 0.22 + 0.09 * r + rng.uniform(-0.01, 0.01)
        init[i, 2] = z_table + half[i, 2]
        init[i, 3] = rng.uniform(-math.pi, math.pi)

    goal_c = np.array([0.5, -0.3])
    tower_h = 2 * BLOCK_HALF * B
    box = np.array([goal_c[0] - 0.15, goal_c[1] - 0.15, z_table + BLOCK_HALF,
                    goal_c[0] + 0.15, goal_c[1] + 0.15, z_table + tower_h + 0.10])

    # keep-out volumes (centre, half) for clutter
    keep = [
        (np.array([0.0, 0.0, 0.6]), np.array([0.28, 0.28, 0.7])),                    # robot base column
        (np.array([0.5, 0.36, 0.25]), np.array([0.24, 0.24, 0.30])),                  # start region
        (np.array([goal_c[0], goal_c[1], 0.5]), np.array([0.11, 0.11, 0.6])),         # tower column
        (np.array([0.5, 0.0, 0.55]), np.array([0.30, 0.42, 0.45])),                   # transport corridor
        (np.array([0.5, -0.3, tower_h + 0.25]), np.array([0.2, 0.2, 0.25])),           # above the tower
    ]
    cub = [table]
    tries = 0
    while len(cub) < O + 1 and tries < 100000:
        tries += 1
        hx, hy, hz = rng.uniform(0.025, 0.15, 3)
        yaw = rng.uniform(-math.pi, math.pi)
        x = rng.uniform(-0.5, 1.25)
        y = rng.uniform(-1.0, 1.0)
        rests = rng.uniform() < 0.5
        z = (z_table + hz) if rests and abs(x - 0.55) < 0.45 and abs(y) < 0.6 else rng.uniform(0.0, 1.2)
        R = _rot_z(yaw)
        ext = np.abs(R) @ np.array([hx, hy, hz])   # axis-aligned bounding half extents
        c = np.array([x, y, z])
        if any(_boxes_overlap(c, ext, kc, kh, 0.02) for kc, kh in keep):
            continue
        # must not cut through the table top unless resting on it
        if abs(x - 0.55) < 0.45 + ext[0] and abs(y) < 0.6 + ext[1] and z - ext[2] < z_table - 1e-9 and z + ext[2] > z_table - 0.05:
            continue
        cub.append(np.concatenate([c, R.ravel(), [hx, hy, hz]]))
    sph = []
    while len(sph) < n_obstacle_spheres:
        c = np.array([rng.uniform(-0.5, 1.25), rng.uniform(-1.0, 1.0), rng.uniform(0.05, 1.2)])
        r = rng.uniform(0.03, 0.12)
        if any(_boxes_overlap(c, [r, r, r], kc, kh, 0.02) for kc, kh in keep):
            continue
        sph.append([c[0], c[1], c[2], r])
    return Scene(cuboid=np.array(cub), sphere=np.array(sph, dtype=np.float64).reshape(-1, 4),
                 half=half, init=init, box=box, z_table=z_table, grasp_off=0.0)


def make_problem(name: str, seed: int = 0, robot_seed: int = 7, **overrides) -> Problem:
    """Named workload (``tower1`` / ``tower4`` / ``tower10``) with a seeded scene."""
    cfg = dict(WORKLOADS[name])
    B, O = cfg.pop("B"), cfg.pop("O")
    n_sph = overrides.pop("n_obstacle_spheres", 0)
    if "B" in overrides:
        B = overrides.pop("B")
    if "O" in overrides:
        O = overrides.pop("O")
    cfg.update(overrides)
    cfg.setdefault("seed", seed)
    params = Params(**cfg)
    return Problem(name=name, robot=make_robot(robot_seed), scene=make_scene(B, O, seed, n_sph), params=params)


# Packing workloads: gx x gy cells of edge 5 cm tiled by tetrominoes (B = gx gy / 4), stage 1
# only (the paper's 5- and 8-block Tetris problems are stage-1 time-to-first-solution runs).
PACKINGS: Dict[str, dict] = {
    # step sizes and batch sizes from a sweep on the GPU (time to first solution, 5 seeds)
    "tetris5": dict(gx=5, gy=4, N=16384, M=4096, P=8, K_lin=25, K_quad=5, eta_init=0.05, alpha=0.02),
    "tetris8": dict(gx=8, gy=4, N=16384, M=4096, P=8, K_lin=100, K_quad=20, eta_init=0.05, alpha=0.02),
}
# Packings are posed in cell units (cube edge 1): plain gradient descent is not unit
# invariant (the yaw gradient carries a lever arm), and in metres the yaw of a 4-cell block
# moves an order of magnitude slower than its position.  eps = 0.02 cell is 1 mm at 5 cm cells.
PACK_PARAMS = dict(eta_init=0.1, alpha=0.05, w_coll=1.0, w_height=1.0, eps=0.02, Q=1, W=3)
CELL = 1.0


def _tile(gx: int, gy: int, size: int, rng) -> np.ndarray:
    """Random partition of a gx x gy grid into connected pieces of `size` cells: the first
    free cell in row-major order grows a piece by random frontier picks; a dead end restarts."""
    for _ in range(100000):
        lab = -np.ones((gx, gy), dtype=np.int64)
        pid, ok = 0, True
        for iy in range(gy):
            for ix in range(gx):
                if lab[ix, iy] >= 0:
                    continue
                piece = [(ix, iy)]
                lab[ix, iy] = pid
                while len(piece) < size:
                    front = sorted({(a + dx, b + dy) for a, b in piece for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1))
                                    if 0 <= a + dx < gx and 0 <= b + dy < gy and lab[a + dx, b + dy] < 0})
                    if not front:
                        ok = False
                        break
                    c = front[int(rng.integers(len(front)))]
                    lab[c] = pid
                    piece.append(c)
                if not ok:
                    break
                pid += 1
            if not ok:
                break
        if ok:
            return lab
    raise RuntimeError("no tiling found")


def packing_problem(blocks, gx: int, gy: int, cell_size: float = CELL, z_span: float = 0.0, turns=None,
                    name: str = "packing", robot_seed: int = 7, slack: float = 0.0, **params) -> Problem:
    """Packing problem from a layout: blocks[b] lists the grid cells (ix, iy) of block b in a
    gx x gy region.  Block b's frame sits at the centroid of its cells, turned by
    turns[b] x 90 degrees (default 0), so the layout itself is a zero-cost packing.  The
    scene's cuboids are the four walls (slabs of thickness and height u just outside the
    region, u = cell_size); the goal box bounds the block origins (x, y in the region, z in
    [z*, z* + z_span]); blocks get cube half extents (z_table = 0 is the floor, z* = u/2)."""
    u = cell_size
    x_lo, y_lo = 0.0, -0.5 * gy * u
    x_hi, y_hi = x_lo + gx * u, y_lo + gy * u
    z_star = 0.5 * u
    # clearance between the tiling and the walls: the region grows by `slack` on every side
    x_lo, y_lo, x_hi, y_hi = x_lo - slack, y_lo - slack, x_hi + slack, y_hi + slack
    B = len(blocks)
    turns = [0] * B if turns is None else list(turns)
    n_cells, cells, planted = [], [], []
    for b, cl in enumerate(blocks):
        idx = np.asarray(cl, dtype=np.float64).reshape(-1, 2)
        centres = np.stack([x_lo + (idx[:, 0] + 0.5) * u, y_lo + (idx[:, 1] + 0.5) * u], axis=1)
        cen = centres.mean(0)
        yaw = 0.5 * math.pi * turns[b]
        Rm = _rot_z(-yaw)[:2, :2]
        cells.append((centres - cen) @ Rm.T)
        n_cells.append(len(idx))
        planted.append([cen[0], cen[1], z_star, (yaw + math.pi) % (2.0 * math.pi) - math.pi])
    xc, yc = 0.5 * (x_lo + x_hi), 0.5 * (y_lo + y_hi)
    hx, hy = 0.5 * (x_hi - x_lo) + u, 0.5 * (y_hi - y_lo) + u
    walls = []
    hz = 0.5 * u
    for c, h in (((x_lo - 0.5 * u, yc, z_star), (0.5 * u, hy, hz)),
                 ((x_hi + 0.5 * u, yc, z_star), (0.5 * u, hy, hz)),
                 ((xc, y_lo - 0.5 * u, z_star), (hx, 0.5 * u, hz)),
                 ((xc, y_hi + 0.5 * u, z_star), (hx, 0.5 * u, hz))):
        walls.append(np.concatenate([np.array(c), np.eye(3).ravel(), np.array(h)]))
    planted = np.array(planted)
    scene = Scene(cuboid=np.array(walls), sphere=np.zeros((0, 4)), half=np.full((B, 3), 0.5 * u),
                  init=planted.copy(), box=np.array([x_lo, y_lo, z_star, x_hi, y_hi, z_star + z_span]),
                  z_table=0.0, grasp_off=0.0)
    prm = dict(PACK_PARAMS)
    prm.update(params)
    pk = Packing(n_cells=np.array(n_cells, dtype=np.int32), cell=np.concatenate(cells), cell_size=u,
                 region=np.array([x_lo, y_lo, x_hi, y_hi]), z_star=z_star, planted=planted)
    return Problem(name=name, robot=make_robot(robot_seed), scene=scene, params=Params(**prm), packing=pk)


def make_packing(name: str, seed: int = 0, robot_seed: int = 7, **overrides) -> Problem:
    """Named packing workload (``tetris5`` / ``tetris8``): a seeded tetromino tiling of the
    region, each block turned by a seeded multiple of 90 degrees."""
    cfg = dict(PACKINGS[name])
    gx, gy = overrides.pop("gx", cfg.pop("gx")), overrides.pop("gy", cfg.pop("gy"))
    u = overrides.pop("cell_size", CELL)
    z_span = overrides.pop("zspan", 0.0)
    rng = np.random.default_rng(np.random.SeedSequence([0x7E7, seed]))
    lab = _tile(gx, gy, 4, rng)
    B = int(lab.max()) + 1
    blocks = [np.argwhere(lab == b) for b in range(B)]
    turns = [int(rng.integers(4)) for _ in range(B)]
    cfg.update(overrides)
    cfg.setdefault("seed", seed)
    return packing_problem(blocks, gx, gy, cell_size=u, z_span=z_span, turns=turns, name=name,
                           robot_seed=robot_seed, **cfg)


# Point-to-point trajectory optimisation (the paper's motion-planning use of stage 2): from
# q_home to a top-down tool target in a cluttered tower scene.
P2P: Dict[str, dict] = {
    "p2p": dict(O=48, N=256, M=64, P=8, Q=1024, W=32, K_traj=50),
}
P2P_LIFT = 0.05   # target height above the top face of a block resting on the table


def make_p2p_scene(O: int, seed: int) -> Scene:
    """Scene of a point-to-point problem: the table, a target over the start region of the
    tower scenes, and O cuboids, half of them small (sides U(0.05, 0.15) m) inside the volume
    between the robot and the target, so that the interpolated path is obstructed.  Keep-out
    volumes: the robot base column and the column above the target."""
    rng = np.random.default_rng(np.random.SeedSequence([0x2B2, O, seed]))
    z_table = 0.0
    table = np.concatenate([[0.55, 0.0, -0.025], np.eye(3).ravel(), [0.45, 0.6, 0.025]])
    tx, ty = 0.36 + 0.27 * rng.uniform(), 0.22 + 0.18 * rng.uniform()
    target = np.array([tx, ty, z_table + 2 * BLOCK_HALF + P2P_LIFT, rng.uniform(-math.pi, math.pi)])
    keep = [
        (np.array([0.0, 0.0, 0.6]), np.array([0.28, 0.28, 0.7])),                      # robot base column
        (np.array([tx, ty, 0.45]), np.array([0.09, 0.09, 0.45])),                      # above the target
    ]
    cub = [table]
    tries = 0
    while len(cub) < O + 1 and tries < 100000:
        tries += 1
        inner = len(cub) <= O // 2
        if inner:   # between the robot and the target
            hx, hy, hz = rng.uniform(0.025, 0.075, 3)
            x, y, z = rng.uniform(0.2, 0.75), rng.uniform(-0.15, 0.45), rng.uniform(0.1, 0.8)
        else:
            hx, hy, hz = rng.uniform(0.025, 0.15, 3)
            x, y, z = rng.uniform(-0.5, 1.25), rng.uniform(-1.0, 1.0), rng.uniform(0.0, 1.2)
        yaw = rng.uniform(-math.pi, math.pi)
        R = _rot_z(yaw)
        ext = np.abs(R) @ np.array([hx, hy, hz])
        c = np.array([x, y, z])
        if any(_boxes_overlap(c, ext, kc, kh, 0.02) for kc, kh in keep):
            continue
        if abs(x - 0.55) < 0.45 + ext[0] and abs(y) < 0.6 + ext[1] and z - ext[2] < z_table:
            continue   # stays above the table top
        cub.append(np.concatenate([c, R.ravel(), [hx, hy, hz]]))
    box = np.array([tx - 0.1, ty - 0.1, target[2], tx + 0.1, ty + 0.1, target[2] + 0.1])
    return Scene(cuboid=np.array(cub), sphere=np.zeros((0, 4)), half=np.zeros((1, 3)), init=target[None].copy(),
                 box=box, z_table=z_table, grasp_off=0.0)


def make_p2p(name: str = "p2p", seed: int = 0, robot_seed: int = 7, **overrides) -> Problem:
    """Point-to-point problem: from q_home to the tool target of make_p2p_scene (tool pointing
    down; any quarter turn of its yaw is accepted by the grasp reading).  The target is a
    zero-size virtual "block": neither an obstacle nor carried."""
    cfg = dict(P2P[name])
    O = overrides.pop("O", cfg.pop("O"))
    cfg.update(overrides)
    cfg.setdefault("seed", seed)
    return Problem(name=name, robot=make_robot(robot_seed), scene=make_p2p_scene(O, seed), params=Params(**cfg),
                   p2p=True)


def heterogeneous_batch(n_problems: int, seed: int = 0):
    """Problems of 1..10 blocks and 8..64 cuboids, 1024..4096 particles each (batched workload)."""
    rng = np.random.default_rng(np.random.SeedSequence([0xBA7C, seed]))
    out = []
    for i in range(n_problems):
        B = int(rng.integers(1, 11))
        O = int(rng.integers(8, 65))
        Q = int(rng.integers(1024, 4097))
        out.append(make_problem("tower10", seed=seed * 1000 + i, B=B, O=O, Q=Q,
                                N=4 * 1024, M=1024))
    return out


def uniforms(n: int, seed: int) -> np.ndarray:
    """Plain seeded uniforms for test inputs (not the method's Philox streams)."""
    return np.random.default_rng(seed).uniform(size=n)
