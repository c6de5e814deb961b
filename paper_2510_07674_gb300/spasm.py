"""Thin ctypes binding of ``libspasm.so`` (argument marshalling only).

Every function here has the name of the C entry point it calls (see ``include/spasm.h``)
and forwards its arguments: device buffers are torch CUDA tensors (passed as raw
pointers), host outputs are numpy arrays.  Nothing is computed here; if the library is
missing the import of a function fails loudly -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

from . import build as _build

LIB_PATH = _build.LIB

SPASM_OK = 0
STATUS = {0: "SPASM_OK", -1: "SPASM_ERR_INVALID", -2: "SPASM_ERR_NOMEM", -3: "SPASM_ERR_CUDA",
          -4: "SPASM_ERR_NOSOLUTION", -5: "SPASM_ERR_TIMEOUT", -6: "SPASM_ERR_DEVICE", -7: "SPASM_ERR_CANCELLED"}

EXPORTED = ["spasm_create_problem", "spasm_destroy_problem", "spasm_last_error", "spasm_place", "spasm_optimize",
            "spasm_result", "spasm_sizes", "spasm_place_sample", "spasm_place_eval", "spasm_place_descend",
            "spasm_select_topk", "spasm_lift", "spasm_traj_eval", "spasm_traj_descend", "spasm_set_seed",
            "spasm_set_timing", "spasm_get_stats", "spasm_reset_stats", "spasm_place_select_static",
            "spasm_server_create", "spasm_server_submit", "spasm_server_poll", "spasm_server_wait",
            "spasm_server_result", "spasm_server_release", "spasm_server_destroy", "spasm_batch_default_config",
            "spasm_optimize_batch", "spasm_batch_autotune", "spasm_create_packing", "spasm_placements",
            "spasm_create_p2p", "spasm_traj_check", "spasm_fp32_fma_peak", "spasm_synchronize",
            "spasm_inject_wait_timeout", "spasm_inject_alloc_failure", "spasm_problem_bytes", "spasm_server_cancel",
            "spasm_server_get_stats", "spasm_set_kernel_config", "spasm_set_launch_mode",
            "spasm_snapshot_bytes", "spasm_snapshot", "spasm_restore", "spasm_traj_residency"]
SPASM_LAUNCH_GRAPH, SPASM_LAUNCH_EAGER = 0, 1


class SpasmError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int32)
_V = ctypes.c_void_p


class _Robot(ctypes.Structure):
    _fields_ = [("dof", ctypes.c_int), ("dh", _D), ("qlim", _D), ("n_spheres", ctypes.c_int), ("sphere_link", _I),
                ("sphere", _D), ("ee", _D), ("q_home", _D)]


class _Obstacles(ctypes.Structure):
    _fields_ = [("n_cuboids", ctypes.c_int), ("cuboid", _D), ("n_spheres", ctypes.c_int), ("sphere", _D)]


class _Goal(ctypes.Structure):
    _fields_ = [("n_blocks", ctypes.c_int), ("half_ext", _D), ("init_pose", _D), ("goal_box", _D),
                ("z_table", ctypes.c_double), ("grasp_off", ctypes.c_double)]


class _Packing(ctypes.Structure):
    _fields_ = [("n_blocks", ctypes.c_int), ("n_cells", ctypes.POINTER(ctypes.c_int32)), ("cell", _D),
                ("cell_size", ctypes.c_double), ("region", _D), ("z_star", ctypes.c_double),
                ("z_span", ctypes.c_double)]


_INT_PARAMS = ("N", "M", "P", "Q", "W", "K_lin", "K_quad", "K_traj", "K_al", "K_ik")
_DBL_PARAMS = ("eta_init", "alpha", "eta_traj", "eps", "eps_start", "w_stable", "w_height", "w_coll", "w_start",
               "w_arm", "w_block", "w_path", "w_jl", "mu0", "mu_max", "ik_damp")


class _Params(ctypes.Structure):
    _fields_ = ([(n, ctypes.c_int) for n in _INT_PARAMS] + [(n, ctypes.c_double) for n in _DBL_PARAMS] +
                [("seed", ctypes.c_uint64), ("max_steps", ctypes.c_int), ("ik_mode", ctypes.c_int)])


class _Stats(ctypes.Structure):
    _fields_ = [("place_attempts", ctypes.c_int), ("traj_attempts", ctypes.c_int), ("n_found", ctypes.c_int),
                ("n_success", ctypes.c_int), ("kernel_launches", ctypes.c_longlong), ("traj_launches", ctypes.c_int),
                ("particle_iters", ctypes.c_longlong), ("ms_place", ctypes.c_double), ("ms_lift", ctypes.c_double),
                ("ms_traj", ctypes.c_double), ("ms_finish", ctypes.c_double), ("h2d_bytes", ctypes.c_longlong),
                ("d2h_bytes", ctypes.c_longlong), ("tests_executed", ctypes.c_longlong),
                ("cull_configs", ctypes.c_longlong), ("cand_configs", ctypes.c_longlong), ("ms_retry", ctypes.c_double),
                ("host_waits", ctypes.c_longlong)]


class _ServerStats(ctypes.Structure):
    _fields_ = [("epochs", ctypes.c_longlong), ("requests_in_epochs", ctypes.c_longlong),
                ("particles_in_epochs", ctypes.c_longlong), ("completed", ctypes.c_longlong),
                ("bytes_in_use", ctypes.c_longlong)]


class _BatchConfig(ctypes.Structure):
    _fields_ = [("per_fetch", ctypes.c_int), ("ctas_per_sm", ctypes.c_int), ("order", ctypes.c_int),
                ("sphere_tiling", ctypes.c_int), ("particles_per_cta", ctypes.c_int)]


class _KernelConfig(ctypes.Structure):
    _fields_ = [("sphere_tiling", ctypes.c_int), ("particles_per_cta", ctypes.c_int)]


_lib = None


def lib():
    """The loaded CUDA library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run paper_2510_07674_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        L.spasm_last_error.restype = ctypes.c_char_p
        L.spasm_create_problem.argtypes = [ctypes.POINTER(_Robot), ctypes.POINTER(_Obstacles), ctypes.POINTER(_Goal),
                                           ctypes.POINTER(_Params), _V, ctypes.POINTER(_V)]
        L.spasm_destroy_problem.argtypes = [_V]
        L.spasm_place.argtypes = [_V]
        L.spasm_optimize.argtypes = [_V]
        L.spasm_result.argtypes = [_V, _I, _D, _D, _D, _I]
        L.spasm_sizes.argtypes = [_V, _I, _I]
        L.spasm_place_sample.argtypes = [_V, ctypes.c_int, ctypes.c_uint32, _V, _V]
        L.spasm_place_eval.argtypes = [_V, ctypes.c_int, _V, ctypes.c_int, _V, _V, _V, _V]
        L.spasm_place_descend.argtypes = [_V, ctypes.c_int, _V, ctypes.c_int, ctypes.c_int, _V, _V]
        L.spasm_select_topk.argtypes = [_V, ctypes.c_int, _V, ctypes.c_int, _V]
        L.spasm_lift.argtypes = [_V, ctypes.c_int, _V, ctypes.c_int, ctypes.c_uint32, _V]
        L.spasm_traj_eval.argtypes = [_V, ctypes.c_int, _V, _V, _V, _V, _V, _V, _V]
        L.spasm_traj_descend.argtypes = [_V, ctypes.c_int, _V, _V, _V, ctypes.c_int, ctypes.c_int, _V, _V]
        L.spasm_set_seed.argtypes = [_V, ctypes.c_uint64]
        L.spasm_set_timing.argtypes = [_V, ctypes.c_int]
        L.spasm_get_stats.argtypes = [_V, ctypes.POINTER(_Stats)]
        L.spasm_reset_stats.argtypes = [_V]
        L.spasm_place_select_static.argtypes = [_V, ctypes.c_int, ctypes.c_uint32, ctypes.c_int, _V, _V]
        L.spasm_traj_check.argtypes = [_V, ctypes.c_int, _V, _V, _V]
        L.spasm_fp32_fma_peak.argtypes = [ctypes.c_double, _D, _D, _D]
        L.spasm_synchronize.argtypes = [_V]
        L.spasm_set_kernel_config.argtypes = [_V, ctypes.POINTER(_KernelConfig)]
        L.spasm_set_launch_mode.argtypes = [_V, ctypes.c_int]
        L.spasm_snapshot_bytes.argtypes = [_V, ctypes.POINTER(ctypes.c_size_t)]
        L.spasm_traj_residency.argtypes = [_V, _I, _I]
        L.spasm_snapshot.argtypes = [_V, _V, ctypes.c_size_t]
        L.spasm_restore.argtypes = [_V, _V, ctypes.c_size_t]
        L.spasm_problem_bytes.argtypes = [ctypes.POINTER(_Obstacles), ctypes.POINTER(_Goal), ctypes.POINTER(_Params),
                                          ctypes.POINTER(ctypes.c_longlong)]
        L.spasm_inject_wait_timeout.argtypes = [_V, ctypes.c_int]
        L.spasm_inject_alloc_failure.argtypes = [ctypes.c_int]
        LL = ctypes.c_longlong
        L.spasm_server_create.argtypes = [LL, ctypes.c_int, ctypes.POINTER(_V)]
        L.spasm_server_submit.argtypes = [_V, ctypes.POINTER(_Robot), ctypes.POINTER(_Obstacles), ctypes.POINTER(_Goal),
                                          ctypes.POINTER(_Params), ctypes.POINTER(LL)]
        L.spasm_server_poll.argtypes = [_V, LL, _I]
        L.spasm_server_wait.argtypes = [_V, LL, ctypes.c_double]
        L.spasm_server_result.argtypes = [_V, LL, _I, _I, _D, _D, _D, _I, _D, _D]
        L.spasm_server_release.argtypes = [_V, LL]
        L.spasm_server_cancel.argtypes = [_V, LL]
        L.spasm_server_get_stats.argtypes = [_V, ctypes.POINTER(_ServerStats)]
        L.spasm_server_destroy.argtypes = [_V]
        L.spasm_batch_default_config.argtypes = [ctypes.POINTER(_BatchConfig)]
        L.spasm_create_packing.argtypes = [ctypes.POINTER(_Robot), ctypes.POINTER(_Packing), ctypes.POINTER(_Params), _V,
                                           ctypes.POINTER(_V)]
        L.spasm_placements.argtypes = [_V, _I, _D]
        L.spasm_create_p2p.argtypes = [ctypes.POINTER(_Robot), ctypes.POINTER(_Obstacles), _D, ctypes.POINTER(_Params),
                                       _V, ctypes.POINTER(_V)]
        L.spasm_optimize_batch.argtypes = [ctypes.POINTER(_V), ctypes.c_int, _V, ctypes.POINTER(_BatchConfig)]
        L.spasm_batch_autotune.argtypes = [ctypes.POINTER(_V), ctypes.c_int, _V, ctypes.POINTER(_BatchConfig), _D]
        for name in EXPORTED:
            if name != "spasm_last_error":
                getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def _check(status: int):
    if status != SPASM_OK:
        raise SpasmError(status, lib().spasm_last_error().decode(errors="replace"))


def _dev(t) -> Optional[int]:
    """Raw device pointer of a contiguous CUDA tensor (or None)."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return t.data_ptr()


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


class ProblemDesc:
    """The C structs describing one workload (arrays kept alive by this object)."""

    def __init__(self, workload, **param_overrides):
        r, s = workload.robot, workload.scene
        prm = dict(vars(workload.params))
        prm.update(param_overrides)
        self.params = prm
        self._arrays = {
            "dh": _f64(r.dh), "qlim": _f64(r.qlim), "sphere_link": np.ascontiguousarray(r.sphere_link, np.int32),
            "sphere": _f64(r.sphere), "ee": _f64(r.ee), "q_home": _f64(r.q_home),
            "cub": _f64(s.cuboid).reshape(-1, 15), "sph": _f64(s.sphere).reshape(-1, 4),
            "half": _f64(s.half), "init": _f64(s.init), "box": _f64(s.box),
        }
        a = self._arrays
        dp = lambda x: x.ctypes.data_as(_D)   # noqa: E731
        self._robot = _Robot(7, dp(a["dh"]), dp(a["qlim"]), len(a["sphere_link"]), a["sphere_link"].ctypes.data_as(_I),
                             dp(a["sphere"]), dp(a["ee"]), dp(a["q_home"]))
        self._obs = _Obstacles(len(a["cub"]), dp(a["cub"]), len(a["sph"]), dp(a["sph"]))
        self._goal = _Goal(len(a["half"]), dp(a["half"]), dp(a["init"]), dp(a["box"]), float(s.z_table),
                           float(s.grasp_off))
        p = _Params()
        for n in _INT_PARAMS:
            setattr(p, n, int(prm[n]))
        for n in _DBL_PARAMS:
            setattr(p, n, float(prm[n]))
        p.seed = int(prm["seed"]) & 0xFFFFFFFFFFFFFFFF
        p.max_steps = int(prm["max_steps"])
        p.ik_mode = int(prm.get("ik_mode", 0))
        self._params = p
        self.B = len(a["half"])
        self.C = 2 * self.B * (int(prm["W"]) - 1) + 1
        self._packing = None
        pk = getattr(workload, "packing", None)
        if pk is not None:   # the appendix's packing (Tetris) goal
            a["n_cells"] = np.ascontiguousarray(pk.n_cells, np.int32)
            a["cell"] = _f64(pk.cell).reshape(-1, 2)
            a["region"] = _f64(pk.region)
            z_span = float(s.box[5] - s.box[2])
            self._packing = _Packing(len(a["n_cells"]), a["n_cells"].ctypes.data_as(_I), dp(a["cell"]),
                                     float(pk.cell_size), dp(a["region"]), float(pk.z_star), z_span)

    def refs(self):
        return (ctypes.byref(self._robot), ctypes.byref(self._obs), ctypes.byref(self._goal),
                ctypes.byref(self._params))


class Problem(ProblemDesc):
    """Owns one ``spasm_problem_t`` created from a seeded workload description."""

    def __init__(self, workload, stream=None, **param_overrides):
        super().__init__(workload, **param_overrides)
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        self.stream = int(stream)
        h = _V()
        if getattr(workload, "p2p", False):   # point-to-point trajectory optimisation
            self._arrays["target"] = _f64(workload.scene.init[0])
            _check(lib().spasm_create_p2p(ctypes.byref(self._robot), ctypes.byref(self._obs),
                                          self._arrays["target"].ctypes.data_as(_D), ctypes.byref(self._params),
                                          _V(self.stream), ctypes.byref(h)))
        elif self._packing is not None:
            _check(lib().spasm_create_packing(ctypes.byref(self._robot), ctypes.byref(self._packing),
                                              ctypes.byref(self._params), _V(self.stream), ctypes.byref(h)))
        else:
            _check(lib().spasm_create_problem(*self.refs(), _V(self.stream), ctypes.byref(h)))
        self.handle = h
        C, NR = ctypes.c_int32(), ctypes.c_int32()
        _check(lib().spasm_sizes(h, ctypes.byref(C), ctypes.byref(NR)))
        self.C, self.NR = C.value, NR.value

    def close(self):
        if getattr(self, "handle", None):
            lib().spasm_destroy_problem(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------------- entry points
def spasm_place(problem: Problem):
    _check(lib().spasm_place(problem.handle))


def spasm_optimize(problem: Problem):
    _check(lib().spasm_optimize(problem.handle))


def spasm_placements(problem: Problem, allow_empty: bool = False) -> dict:
    """Stage-1 result: the satisfying placements found (best first)."""
    P, B = int(problem.params["P"]), problem.B
    n = ctypes.c_int32()
    place = np.zeros((P, B, 4))
    st = lib().spasm_placements(problem.handle, ctypes.byref(n), place.ctypes.data_as(_D))
    if st != SPASM_OK and not (allow_empty and st == -4):
        _check(st)
    return {"n_place": n.value, "placements": place[: n.value]}


def spasm_result(problem: Problem, allow_empty: bool = False) -> dict:
    P, B, C = int(problem.params["P"]), problem.B, problem.C
    nf = ctypes.c_int32()
    place = np.zeros((P, B, 4))
    traj = np.zeros((P, C, 7))
    cost = np.zeros(P)
    succ = np.zeros(P, dtype=np.int32)
    st = lib().spasm_result(problem.handle, ctypes.byref(nf), place.ctypes.data_as(_D), traj.ctypes.data_as(_D),
                            cost.ctypes.data_as(_D), succ.ctypes.data_as(_I))
    if st != SPASM_OK and not (allow_empty and st == -4):
        _check(st)
    n = nf.value
    return {"n_found": n, "placements": place, "traj": traj[:n], "cost": cost[:n], "success": succ[:n]}


def spasm_place_sample(problem: Problem, n: int, attempt: int, x, cost):
    _check(lib().spasm_place_sample(problem.handle, n, attempt, _dev(x), _dev(cost)))


def spasm_place_eval(problem: Problem, n: int, x, quadratic: int, cost, grad=None, metrics=None, terms=None):
    _check(lib().spasm_place_eval(problem.handle, n, _dev(x), int(quadratic), _dev(cost), _dev(grad), _dev(metrics),
                                  _dev(terms)))


def spasm_place_descend(problem: Problem, n: int, x, k_lin: int, k_quad: int, cost=None, sat=None):
    _check(lib().spasm_place_descend(problem.handle, n, _dev(x), k_lin, k_quad, _dev(cost), _dev(sat)))


def spasm_select_topk(problem: Problem, n: int, cost, k: int, idx):
    _check(lib().spasm_select_topk(problem.handle, n, _dev(cost), k, _dev(idx)))


def spasm_lift(problem: Problem, n: int, placements, n_place: int, attempt: int, q):
    _check(lib().spasm_lift(problem.handle, n, _dev(placements), n_place, attempt, _dev(q)))


def spasm_traj_eval(problem: Problem, n: int, q, lam, mu, L, grad=None, groups=None, h=None):
    _check(lib().spasm_traj_eval(problem.handle, n, _dev(q), _dev(lam), _dev(mu), _dev(L), _dev(grad), _dev(groups),
                                 _dev(h)))


def spasm_traj_descend(problem: Problem, n: int, q, lam, mu, k_steps: int, init_multipliers: int, metrics=None,
                       sat=None):
    _check(lib().spasm_traj_descend(problem.handle, n, _dev(q), _dev(lam), _dev(mu), int(k_steps),
                                    int(init_multipliers), _dev(metrics), _dev(sat)))


def spasm_traj_check(problem: Problem, n: int, q, metrics, ok):
    _check(lib().spasm_traj_check(problem.handle, n, _dev(q), _dev(metrics), _dev(ok)))


def spasm_fp32_fma_peak(target_ms: float = 200.0) -> dict:
    """Measured FP32 FMA throughput of the current device (TFLOP/s, time, flop)."""
    tf, ms, fl = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib().spasm_fp32_fma_peak(float(target_ms), ctypes.byref(tf), ctypes.byref(ms), ctypes.byref(fl)))
    return {"tflops": tf.value, "ms": ms.value, "flop": fl.value}


def spasm_problem_bytes(workload, **overrides) -> int:
    """Device bytes spasm_create_problem would allocate for this workload."""
    d = ProblemDesc(workload, **overrides)
    b = ctypes.c_longlong()
    _check(lib().spasm_problem_bytes(ctypes.byref(d._obs), ctypes.byref(d._goal), ctypes.byref(d._params), ctypes.byref(b)))
    return b.value


def spasm_synchronize(problem: Problem):
    _check(lib().spasm_synchronize(problem.handle))


def spasm_inject_wait_timeout(problem: Problem, max_polls: int):
    _check(lib().spasm_inject_wait_timeout(problem.handle, int(max_polls)))


def spasm_inject_alloc_failure(nth: int):
    _check(lib().spasm_inject_alloc_failure(int(nth)))


def spasm_set_seed(problem: Problem, seed: int):
    _check(lib().spasm_set_seed(problem.handle, int(seed) & 0xFFFFFFFFFFFFFFFF))


def spasm_set_timing(problem: Problem, enable: bool):
    _check(lib().spasm_set_timing(problem.handle, int(bool(enable))))


def spasm_get_stats(problem: Problem) -> dict:
    st = _Stats()
    _check(lib().spasm_get_stats(problem.handle, ctypes.byref(st)))
    return {name: getattr(st, name) for name, _ in _Stats._fields_}


def spasm_reset_stats(problem: Problem):
    _check(lib().spasm_reset_stats(problem.handle))


def spasm_place_select_static(problem: Problem, n: int, attempt: int, m: int, x_elite, cost_elite):
    """Sampling + elite selection with the library's fixed device scratch (no allocation)."""
    _check(lib().spasm_place_select_static(problem.handle, n, attempt, m, _dev(x_elite), _dev(cost_elite)))


def _handles(problems):
    arr = (_V * len(problems))()
    for i, p in enumerate(problems):
        arr[i] = p.handle
    return arr


def _batch_stream(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    if int(stream) == 0:
        raise ValueError("the batched form needs a created (non-default) CUDA stream")
    return _V(int(stream))


_BATCH_KEYS = [name for name, _ in _BatchConfig._fields_]


def spasm_batch_default_config() -> dict:
    c = _BatchConfig()
    _check(lib().spasm_batch_default_config(ctypes.byref(c)))
    return {k: getattr(c, k) for k in _BATCH_KEYS}


def spasm_set_kernel_config(problem: Problem, sphere_tiling: int = 0, particles_per_cta: int = 1):
    c = _KernelConfig(int(sphere_tiling), int(particles_per_cta))
    _check(lib().spasm_set_kernel_config(problem.handle, ctypes.byref(c)))


def spasm_set_launch_mode(problem: Problem, mode: int):
    """SPASM_LAUNCH_GRAPH (default) or SPASM_LAUNCH_EAGER (kernel by kernel, host attempt loop)."""
    _check(lib().spasm_set_launch_mode(problem.handle, int(mode)))


def spasm_traj_residency(problem: Problem) -> dict:
    """Resident CTAs per SM of the problem's trajectory kernels (per problem and batched)."""
    a, b = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().spasm_traj_residency(problem.handle, ctypes.byref(a), ctypes.byref(b)))
    return {"single": a.value, "batched": b.value}


def spasm_snapshot_bytes(problem: Problem) -> int:
    n = ctypes.c_size_t()
    _check(lib().spasm_snapshot_bytes(problem.handle, ctypes.byref(n)))
    return n.value


def spasm_snapshot(problem: Problem) -> bytes:
    """The problem's search state after its last stage (see spasm_restore)."""
    n = spasm_snapshot_bytes(problem)
    buf = ctypes.create_string_buffer(n)
    _check(lib().spasm_snapshot(problem.handle, buf, n))
    return buf.raw


def spasm_restore(problem: Problem, snapshot: bytes):
    buf = ctypes.create_string_buffer(bytes(snapshot), len(snapshot))
    _check(lib().spasm_restore(problem.handle, buf, len(snapshot)))


def spasm_optimize_batch(problems, stream=None, config: Optional[dict] = None):
    """Solve the problems together (batched form); read each with spasm_result."""
    cfg = None
    if config is not None:
        base = spasm_batch_default_config()
        base.update({k: v for k, v in config.items() if k in _BATCH_KEYS})
        cfg = _BatchConfig(*[int(base[k]) for k in _BATCH_KEYS])
    _check(lib().spasm_optimize_batch(_handles(problems), len(problems), _batch_stream(stream),
                                      ctypes.byref(cfg) if cfg is not None else None))


def spasm_batch_autotune(problems, stream=None) -> dict:
    """Fastest schedule of the batched trajectory launch for these problems (and its time)."""
    c = _BatchConfig()
    ms = ctypes.c_double()
    _check(lib().spasm_batch_autotune(_handles(problems), len(problems), _batch_stream(stream), ctypes.byref(c),
                                      ctypes.byref(ms)))
    out = {k: getattr(c, k) for k in _BATCH_KEYS}
    out["ms"] = ms.value
    return out


class Server:
    """Owns one ``spasm_server_t`` (continuous-batching solver service)."""

    def __init__(self, budget_bytes: int, max_inflight: int):
        h = _V()
        _check(lib().spasm_server_create(int(budget_bytes), int(max_inflight), ctypes.byref(h)))
        self.handle = h
        self._descs = {}

    def close(self):
        if getattr(self, "handle", None):
            lib().spasm_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def spasm_server_submit(server: Server, workload, **overrides) -> int:
    d = ProblemDesc(workload, **overrides)
    t = ctypes.c_longlong()
    _check(lib().spasm_server_submit(server.handle, *d.refs(), ctypes.byref(t)))
    server._descs[t.value] = d
    return t.value


def spasm_server_poll(server: Server, ticket: int) -> int:
    st = ctypes.c_int32()
    _check(lib().spasm_server_poll(server.handle, ticket, ctypes.byref(st)))
    return st.value


def spasm_server_wait(server: Server, ticket: int, timeout_s: float):
    _check(lib().spasm_server_wait(server.handle, ticket, float(timeout_s)))


def spasm_server_result(server: Server, ticket: int) -> dict:
    d = server._descs[ticket]
    P, B, C = int(d.params["P"]), d.B, d.C
    st, nf = ctypes.c_int32(), ctypes.c_int32()
    place, traj, cost = np.zeros((P, B, 4)), np.zeros((P, C, 7)), np.zeros(P)
    succ = np.zeros(P, dtype=np.int32)
    lat, qms = ctypes.c_double(), ctypes.c_double()
    _check(lib().spasm_server_result(server.handle, ticket, ctypes.byref(st), ctypes.byref(nf), place.ctypes.data_as(_D),
                                     traj.ctypes.data_as(_D), cost.ctypes.data_as(_D), succ.ctypes.data_as(_I),
                                     ctypes.byref(lat), ctypes.byref(qms)))
    n = nf.value
    return {"status": st.value, "n_found": n, "placements": place, "traj": traj[:n], "cost": cost[:n],
            "success": succ[:n], "latency_ms": lat.value, "queue_ms": qms.value}


def spasm_server_cancel(server: Server, ticket: int):
    _check(lib().spasm_server_cancel(server.handle, ticket))


def spasm_server_get_stats(server: Server) -> dict:
    st = _ServerStats()
    _check(lib().spasm_server_get_stats(server.handle, ctypes.byref(st)))
    return {name: getattr(st, name) for name, _ in _ServerStats._fields_}


def spasm_server_release(server: Server, ticket: int):
    _check(lib().spasm_server_release(server.handle, ticket))
    server._descs.pop(ticket, None)
