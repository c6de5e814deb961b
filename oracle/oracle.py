"""ctypes binding of the FP64 CPU oracle -- test infrastructure only.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg use
this module.  It compiles ``spasm_oracle.c`` with gcc into ``liboracle.so`` next to
it and exposes each oracle function on numpy float64 arrays.  It imports nothing from
the CUDA package: a problem is any object with ``robot``, ``scene`` and ``params``
attributes holding numpy arrays (the seeded workload generator provides those).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "spasm_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

NG = 6
G_START, G_ARM, G_BLOCK, G_COLL, G_STABLE, G_HEIGHT = range(NG)


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, -O2, OpenMP) unless an up-to-date build exists."""
    deps = [SRC, os.path.join(HERE, "spasm_oracle.h")]
    if not force and os.path.exists(LIB) and all(os.path.getmtime(LIB) >= os.path.getmtime(d) for d in deps):
        return LIB
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=HERE)
    os.close(fd)
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-Wall",
                           SRC, "-o", tmp, "-lm"])
    os.replace(tmp, LIB)
    return LIB


_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int32)


class _Problem(ctypes.Structure):
    _fields_ = [
        ("dh", _D), ("qlim", _D), ("n_spheres", ctypes.c_int), ("sphere_link", _I), ("sphere", _D),
        ("ee", _D), ("q_home", _D),
        ("n_cub", ctypes.c_int), ("cub", _D), ("n_sph", ctypes.c_int), ("sph", _D),
        ("B", ctypes.c_int), ("half", _D), ("init", _D), ("box", _D),
        ("z_table", ctypes.c_double), ("grasp_off", ctypes.c_double),
        ("N", ctypes.c_int), ("M", ctypes.c_int), ("P", ctypes.c_int), ("Q", ctypes.c_int), ("W", ctypes.c_int),
        ("K_lin", ctypes.c_int), ("K_quad", ctypes.c_int), ("K_traj", ctypes.c_int), ("K_al", ctypes.c_int),
        ("K_ik", ctypes.c_int),
        ("eta_init", ctypes.c_double), ("alpha", ctypes.c_double), ("eta_traj", ctypes.c_double),
        ("eps", ctypes.c_double), ("eps_start", ctypes.c_double),
        ("w_stable", ctypes.c_double), ("w_height", ctypes.c_double), ("w_coll", ctypes.c_double),
        ("w_start", ctypes.c_double), ("w_arm", ctypes.c_double), ("w_block", ctypes.c_double),
        ("w_path", ctypes.c_double), ("w_jl", ctypes.c_double),
        ("mu0", ctypes.c_double), ("mu_max", ctypes.c_double), ("ik_damp", ctypes.c_double),
        ("seed", ctypes.c_uint64), ("max_steps", ctypes.c_int), ("n_threads", ctypes.c_int),
        ("kind", ctypes.c_int), ("cell_start", _I), ("cell", _D), ("cell_size", ctypes.c_double),
        ("z_star", ctypes.c_double), ("ik_mode", ctypes.c_int),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        L = _lib
        P = ctypes.POINTER(_Problem)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        L.or_philox4x32_10.argtypes = [u32p, ctypes.c_uint64, u32p]
        L.or_u01.restype = ctypes.c_double
        L.or_u01.argtypes = [ctypes.c_uint32]
        L.or_fk.argtypes = [P, _D, _D, _D]
        L.or_box_sd.restype = ctypes.c_double
        L.or_box_sd.argtypes = [_D, ctypes.c_double, _D, _D]
        L.or_pen_box.restype = ctypes.c_double
        L.or_pen_box.argtypes = [_D, ctypes.c_double, _D, _D, _D, _D, _D]
        L.or_pen_sph.restype = ctypes.c_double
        L.or_pen_sph.argtypes = [_D, ctypes.c_double, _D, _D]
        L.or_place_cost.restype = ctypes.c_double
        L.or_place_cost.argtypes = [P, _D, ctypes.c_int, _D, _D]
        L.or_place_check.argtypes = [P, _D, _D]
        L.or_place_sample.argtypes = [P, ctypes.c_int, ctypes.c_uint32, _D]
        L.or_argsort.argtypes = [ctypes.c_int, _D, _I]
        L.or_place_descend.argtypes = [P, ctypes.c_int, _D, ctypes.c_int, ctypes.c_int]
        L.or_place_solve.argtypes = [P, _D, _I, _I, _I]
        L.or_n_configs.argtypes = [P]
        L.or_ik.argtypes = [P, _D, _D, _D]
        L.or_ik_analytic_supported.argtypes = [P]
        L.or_ik_analytic.argtypes = [P, _D, ctypes.c_double, _D]
        L.or_ik_select.argtypes = [P, _D, _D, _D, ctypes.c_int, _D]
        L.or_lift.argtypes = [P, _D, ctypes.c_int, ctypes.c_uint32, _D]
        L.or_lift_ex.argtypes = [P, _D, ctypes.c_int, ctypes.c_uint32, _D, _I]
        L.or_traj_cost.restype = ctypes.c_double
        L.or_n_residuals.argtypes = [P]
        L.or_traj_cost.argtypes = [P, _D, _D, ctypes.c_double, _D, _D, _D, _D, _D]
        L.or_traj_check.argtypes = [P, _D, _D]
        L.or_traj_rank_cost.restype = ctypes.c_double
        L.or_traj_rank_cost.argtypes = [P, _D]
        L.or_traj_descend.argtypes = [P, ctypes.c_int, _D, _D, _D, ctypes.c_int]
        L.or_traj_solve.argtypes = [P, _D, ctypes.c_int, _D, _D, _I, _I]
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def philox4x32_10(counter, seed: int) -> np.ndarray:
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in counter])
    out = (ctypes.c_uint32 * 4)()
    lib().or_philox4x32_10(c, ctypes.c_uint64(seed), out)
    return np.array(list(out), dtype=np.uint32)


def u01(u: int) -> float:
    return lib().or_u01(ctypes.c_uint32(u))


def box_sd(c, r, cuboid):
    c, cub, g = _f64(c), _f64(cuboid), np.zeros(3)
    sd = lib().or_box_sd(_dp(c), float(r), _dp(cub), _dp(g))
    return sd, g


def pen_box(c, r, centre, R, half):
    c, ce, RR, h = _f64(c), _f64(centre), _f64(R).ravel().copy(), _f64(half)
    gc, gp = np.zeros(3), np.zeros(3)
    pen = lib().or_pen_box(_dp(c), float(r), _dp(ce), _dp(RR), _dp(h), _dp(gc), _dp(gp))
    return pen, gc, gp


def pen_sph(c, r, sph):
    c, s, g = _f64(c), _f64(sph), np.zeros(3)
    pen = lib().or_pen_sph(_dp(c), float(r), _dp(s), _dp(g))
    return pen, g


def argsort(cost) -> np.ndarray:
    c = _f64(cost)
    idx = np.zeros(len(c), dtype=np.int32)
    lib().or_argsort(len(c), _dp(c), idx.ctypes.data_as(_I))
    return idx


class Oracle:
    """One problem instance bound to the oracle; arrays are kept alive by the object."""

    def __init__(self, problem, n_threads: int = 1, **param_overrides):
        r, s = problem.robot, problem.scene
        prm = dict(vars(problem.params))
        prm.update(param_overrides)
        self.params = prm
        self._keep = {
            "dh": _f64(r.dh), "qlim": _f64(r.qlim), "sphere_link": np.ascontiguousarray(r.sphere_link, np.int32),
            "sphere": _f64(r.sphere), "ee": _f64(r.ee), "q_home": _f64(r.q_home),
            "cub": _f64(s.cuboid).reshape(-1, 15), "sph": _f64(s.sphere).reshape(-1, 4),
            "half": _f64(s.half), "init": _f64(s.init), "box": _f64(s.box),
        }
        k = self._keep
        st = _Problem()
        st.dh, st.qlim, st.sphere, st.ee, st.q_home = (_dp(k["dh"]), _dp(k["qlim"]), _dp(k["sphere"]),
                                                        _dp(k["ee"]), _dp(k["q_home"]))
        st.n_spheres = len(k["sphere_link"])
        st.sphere_link = k["sphere_link"].ctypes.data_as(_I)
        st.n_cub, st.cub = len(k["cub"]), _dp(k["cub"])
        st.n_sph, st.sph = len(k["sph"]), _dp(k["sph"])
        st.B, st.half, st.init, st.box = len(k["half"]), _dp(k["half"]), _dp(k["init"]), _dp(k["box"])
        st.z_table, st.grasp_off = float(s.z_table), float(s.grasp_off)
        for name in ("N", "M", "P", "Q", "W", "K_lin", "K_quad", "K_traj", "K_al", "K_ik", "max_steps"):
            setattr(st, name, int(prm[name]))
        for name in ("eta_init", "alpha", "eta_traj", "eps", "eps_start", "w_stable", "w_height", "w_coll",
                     "w_start", "w_arm", "w_block", "w_path", "w_jl", "mu0", "mu_max", "ik_damp"):
            setattr(st, name, float(prm[name]))
        st.seed = int(prm["seed"]) & 0xFFFFFFFFFFFFFFFF
        st.n_threads = int(n_threads)
        st.ik_mode = int(prm.get("ik_mode", 0))
        pk = getattr(problem, "packing", None)
        if pk is not None:   # the appendix's packing (Tetris) problem
            k["cell_start"] = np.ascontiguousarray(np.concatenate([[0], np.cumsum(pk.n_cells)]), np.int32)
            k["cell"] = _f64(pk.cell).reshape(-1, 2)
            st.kind = 1
            st.cell_start = k["cell_start"].ctypes.data_as(_I)
            st.cell = _dp(k["cell"])
            st.cell_size, st.z_star = float(pk.cell_size), float(pk.z_star)
        elif getattr(problem, "p2p", False):   # point-to-point trajectory optimisation
            st.kind = 2
        else:
            st.kind = 0
        self.st = st
        self.B = st.B
        self.ptr = ctypes.byref(st)
        self.C = lib().or_n_configs(self.ptr)
        self.NR = lib().or_n_residuals(self.ptr)

    # -- kinematics ------------------------------------------------------------------
    def fk(self, q):
        q = _f64(q)
        frames, tee = np.zeros((8, 4, 4)), np.zeros((4, 4))
        lib().or_fk(self.ptr, _dp(q), _dp(frames), _dp(tee))
        return frames, tee

    def ik(self, target, q0):
        t, q0 = _f64(target), _f64(q0)
        q = np.zeros(7)
        lib().or_ik(self.ptr, _dp(t), _dp(q0), _dp(q))
        return q

    def ik_analytic_supported(self) -> bool:
        return bool(lib().or_ik_analytic_supported(self.ptr))

    def ik_analytic(self, target, q6: float) -> np.ndarray:
        """All in-limit analytic IK solutions of a tool pose for a given last joint, (n, 7)."""
        t = _f64(target)
        sol = np.zeros((8, 7))
        n = lib().or_ik_analytic(self.ptr, _dp(t), float(q6), _dp(sol))
        return sol[:n].copy()

    def ik_select(self, target, seed, q6s):
        """(found, q): the analytic solution nearest to seed over the last-joint values q6s."""
        t, sd, c = _f64(target), _f64(seed), _f64(q6s)
        q = np.zeros(7)
        found = lib().or_ik_select(self.ptr, _dp(t), _dp(sd), _dp(c), len(c), _dp(q))
        return bool(found), q

    # -- stage 1 -----------------------------------------------------------------------
    def place_cost(self, x, quad: bool = False, grad: bool = True):
        x = _f64(x).reshape(self.B, 4)
        g = np.zeros((self.B, 4))
        terms = np.zeros(3)
        c = lib().or_place_cost(self.ptr, _dp(x), int(quad), _dp(g) if grad else None, _dp(terms))
        return c, g, terms

    def place_check(self, x):
        x = _f64(x).reshape(self.B, 4)
        m = np.zeros(3)
        ok = lib().or_place_check(self.ptr, _dp(x), _dp(m))
        return bool(ok), m

    def place_sample(self, n: int, attempt: int = 0):
        x = np.zeros((n, self.B, 4))
        lib().or_place_sample(self.ptr, n, attempt, _dp(x))
        return x

    def place_descend(self, x, k_lin=None, k_quad=None):
        x = _f64(x).reshape(-1, self.B, 4).copy()
        k_lin = self.params["K_lin"] if k_lin is None else k_lin
        k_quad = self.params["K_quad"] if k_quad is None else k_quad
        lib().or_place_descend(self.ptr, len(x), _dp(x), int(k_lin), int(k_quad))
        return x

    def place_solve(self):
        P = int(self.params["P"])
        out = np.zeros((P, self.B, 4))
        nf, att, steps = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        lib().or_place_solve(self.ptr, _dp(out), ctypes.byref(nf), ctypes.byref(att), ctypes.byref(steps))
        return out[: nf.value], att.value, steps.value

    # -- stage 2 -----------------------------------------------------------------------
    def lift(self, place, particle: int, attempt: int = 0):
        p = _f64(place).reshape(self.B, 4)
        q = np.zeros((self.C, 7))
        lib().or_lift(self.ptr, _dp(p), int(particle), int(attempt), _dp(q))
        return q

    def lift_methods(self, place, particle: int, attempt: int = 0):
        """(q, analytic): the lift and, per block, whether its grasp / place configuration
        came from the analytic IK (B x 2 booleans)."""
        p = _f64(place).reshape(self.B, 4)
        q = np.zeros((self.C, 7))
        flags = np.zeros(2 * self.B, np.int32)
        lib().or_lift_ex(self.ptr, _dp(p), int(particle), int(attempt), _dp(q), flags.ctypes.data_as(_I))
        return q, flags.reshape(self.B, 2).astype(bool)

    def traj_cost(self, q, lam=None, mu=None, grad: bool = True):
        """L, dL/dq (C x 7), appendix terms (6), path, jl, residuals h (NR)."""
        q = _f64(q).reshape(self.C, 7)
        lam = np.zeros(self.NR) if lam is None else _f64(lam).reshape(self.NR)
        mu = self.params["mu0"] if mu is None else float(mu)
        g = np.zeros((self.C, 7))
        cg = np.zeros(NG)
        h = np.zeros(self.NR)
        path, jl = ctypes.c_double(), ctypes.c_double()
        L = lib().or_traj_cost(self.ptr, _dp(q), _dp(lam), mu, _dp(g) if grad else None, _dp(cg),
                               ctypes.byref(path), ctypes.byref(jl), _dp(h))
        return L, g, cg, path.value, jl.value, h

    def traj_check(self, q):
        q = _f64(q).reshape(self.C, 7)
        m = np.zeros(6)
        ok = lib().or_traj_check(self.ptr, _dp(q), _dp(m))
        return bool(ok), m

    def traj_rank_cost(self, q):
        return lib().or_traj_rank_cost(self.ptr, _dp(_f64(q).reshape(self.C, 7)))

    def traj_descend(self, q, lam=None, mu=None, k_steps=None):
        q = _f64(q).reshape(-1, self.C, 7).copy()
        n = len(q)
        lam = np.zeros((n, self.NR)) if lam is None else _f64(lam).reshape(n, self.NR).copy()
        mu = np.full(n, float(self.params["mu0"])) if mu is None else _f64(mu).reshape(n).copy()
        k = self.params["K_traj"] if k_steps is None else int(k_steps)
        lib().or_traj_descend(self.ptr, n, _dp(q), _dp(lam), _dp(mu), k)
        return q, lam, mu

    def traj_solve(self, place):
        place = _f64(place).reshape(-1, self.B, 4)
        P = int(self.params["P"])
        out_q = np.zeros((P, self.C, 7))
        out_c = np.zeros(P)
        nf, att = ctypes.c_int32(), ctypes.c_int32()
        lib().or_traj_solve(self.ptr, _dp(place), len(place), _dp(out_q), _dp(out_c), ctypes.byref(nf),
                            ctypes.byref(att))
        return out_q[: nf.value], out_c[: nf.value], att.value
