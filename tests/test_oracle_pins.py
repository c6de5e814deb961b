"""Pins of the FP64 oracle against facts fixed outside the oracle itself.

Each test checks the oracle against a closed form, a library routine, brute force, or
central differences -- never against a re-typed copy of its own formula.
"""
import ctypes
import ctypes.util
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2510_07674_gb300 import scenes


# ------------------------------------------------------------------------------- Philox
def _curand():
    for cand in ("/usr/local/cuda/lib64/libcurand.so", ctypes.util.find_library("curand")):
        if cand and os.path.exists(cand) if cand.startswith("/") else cand:
            try:
                return ctypes.CDLL(cand)
            except OSError:
                pass
    return None


def test_philox_matches_curand_host_generator():
    """cuRAND's host Philox4_32_10 generator (a library, run on the CPU) emits block j of
    subsequence j at offset 0: counter (0, 0, j, 0), key = seed."""
    cr = _curand()
    if cr is None:
        pytest.skip("libcurand not available")
    for seed in (0, 1, 0x123456789ABCDEF, 0xFFFFFFFFFFFFFFFF, 7 << 32):
        gen = ctypes.c_void_p()
        assert cr.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0   # CURAND_RNG_PSEUDO_PHILOX4_32_10
        assert cr.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        n = 4 * 64
        buf = (ctypes.c_uint32 * n)()
        assert cr.curandGenerate(gen, buf, ctypes.c_size_t(n)) == 0
        got = np.array(list(buf), dtype=np.uint32).reshape(64, 4)
        for j in range(64):
            np.testing.assert_array_equal(O.philox4x32_10((0, 0, j, 0), seed), got[j])
        cr.curandDestroyGenerator(gen)


def test_u01_is_exact_top24():
    assert O.u01(0) == 0.0
    assert O.u01(0xFFFFFFFF) == 1.0 - 2.0 ** -24
    assert O.u01(0x100) == 2.0 ** -24
    assert O.u01(0x80000000) == 0.5


def test_philox_streams_distinct_and_uniform():
    vals = np.array([O.philox4x32_10((i, 3, 0, 0), 42) for i in range(4096)]).ravel()
    assert len(np.unique(vals)) == len(vals)
    u = vals / 2.0 ** 32
    hist, _ = np.histogram(u, bins=16, range=(0, 1))
    chi2 = ((hist - len(u) / 16) ** 2 / (len(u) / 16)).sum()
    assert chi2 < 40.0   # 15 dof, p ~ 5e-4


# ------------------------------------------------------------------------------- FK
class _P:
    """Minimal problem wrapper for FK-only pins."""

    def __init__(self, dh, ee=None):
        base = scenes.make_problem("tower1", seed=0)
        self.robot = scenes.Robot(dh=np.asarray(dh, float), qlim=base.robot.qlim, sphere_link=base.robot.sphere_link,
                                  sphere=base.robot.sphere, ee=np.eye(4) if ee is None else ee,
                                  q_home=base.robot.q_home)
        self.scene, self.params = base.scene, base.params


def test_fk_planar_chain_closed_form():
    """alpha = d = 0: the 7-R chain is a planar arm, x = sum a_k cos(sum_{i<k} q_i)."""
    rng = np.random.default_rng(1)
    a = rng.uniform(0.05, 0.4, 7)
    orc = O.Oracle(_P(np.stack([a, np.zeros(7), np.zeros(7), np.zeros(7)], 1)))
    for _ in range(20):
        q = rng.uniform(-3, 3, 7)
        _, tee = orc.fk(q)
        cum = np.concatenate([[0.0], np.cumsum(q)])
        x = sum(a[k] * math.cos(cum[k]) for k in range(7))
        y = sum(a[k] * math.sin(cum[k]) for k in range(7))
        np.testing.assert_allclose(tee[:3, 3], [x, y, 0.0], atol=1e-12)
        np.testing.assert_allclose(math.atan2(tee[1, 0], tee[0, 0]), math.remainder(cum[7], 2 * math.pi), atol=1e-12)


def test_fk_single_twisted_joint_closed_form():
    """One joint (a, alpha, d): origin (a, -d sin alpha, d cos alpha), axis (0, -sin alpha, cos alpha),
    x-axis (cos q, sin q cos alpha, sin q sin alpha)."""
    a, al, d = 0.3, 0.7, 0.2
    dh = np.zeros((7, 4))
    dh[0] = (a, al, d, 0.0)
    orc = O.Oracle(_P(dh))
    for q1 in (0.0, 0.4, -2.0):
        fr, _ = orc.fk(np.array([q1, 0, 0, 0, 0, 0, 0.0]))
        T = fr[1]
        np.testing.assert_allclose(T[:3, 3], [a, -d * math.sin(al), d * math.cos(al)], atol=1e-14)
        np.testing.assert_allclose(T[:3, 2], [0, -math.sin(al), math.cos(al)], atol=1e-14)
        np.testing.assert_allclose(T[:3, 0], [math.cos(q1), math.sin(q1) * math.cos(al), math.sin(q1) * math.sin(al)],
                                   atol=1e-14)


def test_fk_rotations_orthonormal():
    pr = scenes.make_problem("tower1", seed=0)
    orc = O.Oracle(pr)
    rng = np.random.default_rng(2)
    for _ in range(50):
        fr, tee = orc.fk(rng.uniform(-2.5, 2.5, 7))
        for T in list(fr) + [tee]:
            R = T[:3, :3]
            assert np.abs(R.T @ R - np.eye(3)).max() < 1e-12
            assert abs(np.linalg.det(R) - 1.0) < 1e-12
            np.testing.assert_array_equal(T[3], [0, 0, 0, 1])


def test_fk_link_lengths_invariant():
    """Distance between consecutive joint origins does not depend on q: sqrt(a^2 + d^2)."""
    pr = scenes.make_problem("tower1", seed=0)
    orc = O.Oracle(pr)
    rng = np.random.default_rng(3)
    for _ in range(10):
        fr, _ = orc.fk(rng.uniform(-2.5, 2.5, 7))
        for k in range(1, 7):
            dist = np.linalg.norm(fr[k + 1][:3, 3] - fr[k][:3, 3])
            a, d = pr.robot.dh[k, 0], pr.robot.dh[k, 2]
            assert abs(dist - math.hypot(a, d)) < 1e-12


# ------------------------------------------------------------------------------- SDF
def _rand_rot(rng):
    A = rng.normal(size=(3, 3))
    Qm, Rr = np.linalg.qr(A)
    Qm = Qm @ np.diag(np.sign(np.diag(Rr)))
    if np.linalg.det(Qm) < 0:
        Qm[:, 0] *= -1
    return Qm


def _cub(centre, R, half):
    return np.concatenate([centre, np.asarray(R).ravel(), half])


def test_sdf_special_cases():
    cub = _cub([0, 0, 0], np.eye(3), [1, 1, 1])
    assert O.box_sd([2, 0, 0], 0.5, cub)[0] == pytest.approx(0.5, abs=1e-15)        # face
    assert O.box_sd([2, 2, 0], 0.1, cub)[0] == pytest.approx(math.sqrt(2) - 0.1)   # edge
    assert O.box_sd([2, 2, 2], 0.0, cub)[0] == pytest.approx(math.sqrt(3))         # corner
    assert O.box_sd([0.5, 0, 0], 0.2, cub)[0] == pytest.approx(-0.5 - 0.2)         # inside
    assert O.box_sd([0, 0, 0], 0.0, cub)[0] == pytest.approx(-1.0)                 # centre
    # separated primitives give exactly zero penetration and zero gradient
    pen, gc, gp = O.pen_box([3, 0, 0], 0.5, [0, 0, 0], np.eye(3), [1, 1, 1])
    assert pen == 0.0 and not gc.any() and not gp.any()
    pen, g = O.pen_sph([0, 0, 3], 1.0, [0, 0, 0, 1.0])
    assert pen == 0.0 and not g.any()
    pen, g = O.pen_sph([0, 0, 1.5], 1.0, [0, 0, 0, 1.0])
    assert pen == pytest.approx(0.5) and g == pytest.approx([0, 0, -1])   # moving apart reduces pen


def test_sdf_brute_force_surface_sampling():
    """|signed distance| equals the distance to the nearest of densely sampled surface points."""
    rng = np.random.default_rng(4)
    n = 161
    g = np.linspace(-1, 1, n)
    U, V = np.meshgrid(g, g, indexing="ij")
    for _ in range(6):
        half = rng.uniform(0.05, 0.3, 3)
        R = _rand_rot(rng)
        centre = rng.uniform(-1, 1, 3)
        faces = []
        for ax in range(3):
            o1, o2 = [k for k in range(3) if k != ax]
            for sgn in (-1, 1):
                P = np.zeros((n * n, 3))
                P[:, ax] = sgn * half[ax]
                P[:, o1] = U.ravel() * half[o1]
                P[:, o2] = V.ravel() * half[o2]
                faces.append(P)
        surf = np.concatenate(faces) @ R.T + centre
        spacing = 2 * half.max() / (n - 1)
        for _ in range(20):
            c = centre + rng.normal(0, 0.3, 3)
            sd, _ = O.box_sd(c, 0.0, _cub(centre, R, half))
            dmin = np.sqrt(((surf - c) ** 2).sum(1)).min()
            p = R.T @ (c - centre)
            inside = np.all(np.abs(p) <= half)
            assert (sd <= 0) == inside
            assert abs(abs(sd) - dmin) <= spacing + 1e-12


def test_sdf_gradient_central_difference():
    rng = np.random.default_rng(5)
    for _ in range(200):
        half = rng.uniform(0.05, 0.3, 3)
        cub = _cub(rng.uniform(-1, 1, 3), _rand_rot(rng), half)
        c = cub[:3] + rng.normal(0, 0.3, 3)
        sd, g = O.box_sd(c, 0.1, cub)
        h = 1e-6
        fd = np.array([(O.box_sd(c + h * e, 0.1, cub)[0] - O.box_sd(c - h * e, 0.1, cub)[0]) / (2 * h)
                       for e in np.eye(3)])
        assert np.allclose(fd, g, atol=1e-7), (fd, g)
        assert abs(np.linalg.norm(g) - 1.0) < 1e-12   # an SDF has unit gradient


# ------------------------------------------------------------------------------- argsort
def test_argsort_is_numpy_stable_argsort():
    rng = np.random.default_rng(6)
    c = rng.integers(0, 20, 1000).astype(float)   # many ties
    c[::37] = np.nan
    got = O.argsort(c)
    ref = np.argsort(np.where(np.isnan(c), np.inf, c), kind="stable")
    np.testing.assert_array_equal(got, ref)
