"""Hand-built test scenes shared by the oracle pins and the GPU parity tests.

* The *probe arm*: all seven joints turn about the world z axis through the origin (every
  DH row zero except an optional offset a along joint 2) with a chosen flange -> tool
  transform, so the tool pose is known by hand: Rz(q_1) Trans_x(a) Rz(q_2 + ... + q_7) ee.
* CheckScene: two blocks on the real synthetic arm, with chosen block poses reached through
  the oracle's analytic IK, and one robot sphere on the fixed base, so that each acceptance
  criterion of the final check can be put at a chosen distance from its threshold.

Inputs only: nothing here computes a cost.
"""
import math

import numpy as np

from oracle import oracle as O
from paper_2510_07674_gb300 import scenes

H = scenes.BLOCK_HALF
GO = 0.01   # tool standoff above the top face


def Rx(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[1.0, 0.0, 0.0], [0.0, c, -s], [0.0, s, c]])


def Ry(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]])


def Rz(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def T4(R=np.eye(3), t=(0.0, 0.0, 0.0)):
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = t
    return T


def cuboid(centre, half, R=np.eye(3)):
    return np.concatenate([np.asarray(centre, float), np.asarray(R, float).ravel(), np.asarray(half, float)])


def probe_problem(B, W, ee, spheres, cuboids=(), half=None, init=None, z_table=0.0, a2=0.0, robot=None, **prm):
    """A tower problem on the probe arm (or on `robot`): spheres = [(link, (x, y, z), r)]."""
    if robot is None:
        dh = np.zeros((7, 4))
        dh[1, 0] = a2
        robot = scenes.Robot(dh=dh, qlim=np.tile([-3.0, 3.0], (7, 1)), sphere_link=None, sphere=None, ee=ee,
                             q_home=np.zeros(7))
    robot = scenes.Robot(dh=robot.dh, qlim=robot.qlim,
                         sphere_link=np.array([s[0] for s in spheres], np.int32),
                         sphere=np.array([[*s[1], s[2]] for s in spheres], float), ee=robot.ee, q_home=robot.q_home)
    half = np.full((B, 3), H) if half is None else np.asarray(half, float)
    init = np.zeros((B, 4)) if init is None else np.asarray(init, float)
    scene = scenes.Scene(cuboid=np.array(cuboids, float).reshape(-1, 15), sphere=np.zeros((0, 4)), half=half,
                         init=init, box=np.array([-1.0, -1.0, 0.0, 1.0, 1.0, 1.0]), z_table=z_table, grasp_off=GO)
    params = scenes.Params(W=W, **prm)
    return scenes.Problem(name="probe", robot=robot, scene=scene, params=params)


def probe_ee(E=np.eye(3), t=(0.3, 0.0, 0.5)):
    """Flange -> tool transform whose held block has orientation Rz(sum q) E (tool pointing
    down when E = I)."""
    return T4(E @ Rx(math.pi), t)


def probe_tool(q, ee, a2=0.0):
    """Tool pose of the probe arm: Rz(q_1) Trans_x(a2) Rz(q_2 + ... + q_7) ee."""
    return T4(Rz(q[0])) @ T4(t=(a2, 0.0, 0.0)) @ T4(Rz(float(np.sum(q[1:])))) @ ee


def held_block(T_tool, hz):
    """Reading 10: the block frame is tool x Rx(pi) x Trans(0, 0, -(hz + standoff))."""
    return T_tool @ T4(Rx(math.pi)) @ T4(t=(0.0, 0.0, -(hz + GO)))


class CheckScene:
    """Two blocks on the real synthetic arm.  Block poses are chosen; configurations come from
    the analytic IK of the tool pose that holds each block (tool = block x Trans(0, 0, hz +
    standoff) x Rx(pi)).  Block 0 rests on the table at xy0, block 1 on top of it shifted by
    dx; the initial poses are the blocks the grasp configurations hold.  The arm is reduced to
    one sphere on the fixed base, far from everything, so only the designed contacts count."""

    def __init__(self, dx=0.0, dz=0.0, tilt=0.0, start_off=(0.0, 0.0, 0.0), box_gap=None, arm_pen=None,
                 z_table=0.0):
        self.robot = scenes.make_robot(7)
        self.z_table = z_table
        xy0 = np.array([0.5, -0.3])
        self.place = [T4(Rz(0.4) @ Rx(tilt), (*xy0, z_table + H + dz)),
                      T4(Rz(0.4), (xy0[0] + dx, xy0[1], z_table + 3 * H + dz))]
        self.grasp = [T4(Rz(-0.3), (0.45, 0.3, z_table + H)), T4(Rz(0.9), (0.55, 0.25, z_table + H))]
        sph = (-0.6, 0.6, 0.3)
        boxes = []
        if arm_pen is not None:   # a box sunk arm_pen into the base sphere from +x
            boxes.append(cuboid((sph[0] + 0.05 - arm_pen + 0.1, sph[1], sph[2]), (0.1, 0.1, 0.1)))
        if box_gap is not None:   # a box whose -x face is box_gap inside block 0's +x face
            # (block 0's footprint axes: yaw 0.4; the box shares them)
            R = Rz(0.4)
            c = self.place[0][:3, 3] + R @ np.array([H - box_gap + 0.05, 0.0, 0.0])
            boxes.append(cuboid(c, (0.05, 0.05, H), R))
        yaws = (-0.3, 0.9)
        init = [[*(self.grasp[b][:3, 3] - np.asarray(start_off if b == 0 else (0, 0, 0))), yaws[b]] for b in range(2)]
        pr = probe_problem(2, 3, None, [(0, sph, 0.05)], boxes, init=init, z_table=z_table, robot=self.robot)
        self.pr, self.orc = pr, O.Oracle(pr)
        self.q = self._configs()

    def _ik(self, T_blk):
        T_tool = T_blk @ T4(t=(0.0, 0.0, H + GO)) @ T4(Rx(math.pi))
        best = None
        for q6 in np.linspace(-2.5, 2.5, 41):
            for s in self.orc.ik_analytic(T_tool, q6):
                d = np.sum((s - self.robot.q_home) ** 2)
                if best is None or d < best[0]:
                    best = (d, s)
        assert best is not None
        q = best[1]
        _, T = self.orc.fk(q)
        np.testing.assert_allclose(T, T_tool, atol=1e-9)
        return q

    def _configs(self):
        qg = [self._ik(T) for T in self.grasp]
        qp = [self._ik(T) for T in self.place]
        h = self.robot.q_home
        # t: 0 home, 1 transit, 2 grasp 0, 3 transfer (held at the grasp), 4 place 0,
        #    5 transit, 6 grasp 1, 7 transfer (held at the grasp), 8 place 1
        return np.stack([h, 0.5 * (h + qg[0]), qg[0], qg[0], qp[0], 0.5 * (qp[0] + qg[1]), qg[1], qg[1], qp[1]])


