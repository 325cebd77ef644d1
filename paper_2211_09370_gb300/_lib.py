"""ctypes binding of the qslbm C ABI (include/qslbm.h).

Argument marshalling only: every step of the method runs in the CUDA library.
The functions keep the C names (``qslbm_create``, ``qslbm_step``, ...); the
``Solver`` class is a thin convenience over them.  Loading fails loudly if the
library has not been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import threading

import numpy as np

from . import build as _build

OK, EINVAL, ENOMEM, ECUDA, EUNSTABLE, ETIMEOUT, EBUDGET, ENOTFOUND, EARCH = 0, -1, -2, -3, -4, -5, -6, -7, -8
CHANNEL, PIPE, PERIODIC = 0, 1, 2
B0_UNIFORM, B0_TANH, B0_FIELD = 0, 1, 2
FP32, FP64 = 0, 1
SWEEP_AUTO, SWEEP_PLANES, SWEEP_RESIDENT, SWEEP_SPLIT, SWEEP_FUSED = 0, 1, 2, 3, 4
SWEEP_KERNEL = {"auto": SWEEP_AUTO, "planes": SWEEP_PLANES, "resident": SWEEP_RESIDENT, "split": SWEEP_SPLIT,
                "fused": SWEEP_FUSED}
GEOMETRY = {"channel": CHANNEL, "pipe": PIPE, "none": PERIODIC, "periodic": PERIODIC}
B0_KIND = {"uniform": B0_UNIFORM, "tanh": B0_TANH, "field": B0_FIELD}
PRECISION = {"fp32": FP32, "fp64": FP64}


class qslbm_params(C.Structure):
    _fields_ = [
        ("dim", C.c_int32), ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("geometry", C.c_int32),
        ("diameter", C.c_double), ("center", C.c_double * 2), ("marker_spacing", C.c_double),
        ("Re", C.c_double), ("Ha", C.c_double), ("Rm", C.c_double), ("U0", C.c_double),
        ("b0_kind", C.c_int32), ("b0_dir", C.c_double * 3), ("ramp_center", C.c_double),
        ("ramp_width", C.c_double), ("force_amp", C.c_double), ("force_period", C.c_double),
        ("n_mag", C.c_int32), ("n_mag_cap", C.c_int32), ("nu_ref", C.c_double), ("eta_ref", C.c_double),
        ("precision", C.c_int32), ("strict_qs", C.c_int32), ("seed", C.c_uint64), ("perturb", C.c_double),
        ("init_kind", C.c_int32), ("sweep_kernel", C.c_int32), ("alpha", C.c_double),
        ("mag_scheme", C.c_int32), ("gamma", C.c_double), ("b0_field", C.c_void_p), ("flow_q", C.c_int32),
        ("flow_scheme", C.c_int32), ("stream", C.c_void_p),
    ]


class qslbm_units(C.Structure):
    _fields_ = [(k, C.c_double) for k in
                ("R", "U0", "nu", "tau", "eta", "B0", "F0", "c_mag", "lambda_", "lambda_m", "cs2", "cm2")]
    _fields_ += [("n_mag", C.c_int32), ("n_markers", C.c_int32), ("nodes", C.c_int64), ("device_bytes", C.c_int64),
                ("shell_nodes", C.c_int64), ("sweep_kernel", C.c_int32), ("tau_m", C.c_double),
                ("flow_q", C.c_int32), ("gamma", C.c_double), ("fused_rows", C.c_int32),
                ("fused_bands", C.c_int32), ("fused_chunk", C.c_int32), ("fused_ctas", C.c_int32),
                ("sweep_us_fused", C.c_double), ("sweep_us_split", C.c_double)]


class qslbm_obs(C.Structure):
    _fields_ = [("step", C.c_int64)] + [(k, C.c_double) for k in (
        "mass", "mass_drift", "E_k", "E_m", "pump", "visc", "joule", "qs_residual", "steady_residual")] + [
        ("nan_flag", C.c_int32)]


class qslbm_batch_info_t(C.Structure):
    _fields_ = [("count", C.c_int32), ("max_n_mag", C.c_int32), ("sweep_threads", C.c_int32),
                ("sweep_grid", C.c_int32), ("launches_per_step", C.c_int32), ("nodes", C.c_int64),
                ("node_sweeps_per_step", C.c_int64), ("device_bytes", C.c_int64), ("steps", C.c_int64),
                ("tune_us", C.c_double * 32), ("resident_instances", C.c_int32), ("resident_groups", C.c_int32),
                ("graph_steps", C.c_int32), ("march_chunk", C.c_int32), ("sweep_pdl", C.c_int32)]


class qslbm_server_config(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_int64), ("chunk_steps", C.c_int32), ("max_running", C.c_int32),
                ("precision", C.c_int32), ("stream", C.c_void_p), ("admit", C.c_int32)]


ADMIT = {"fifo": 0, "smallest": 1}


class qslbm_result(C.Structure):
    _fields_ = [("id", C.c_int64), ("status", C.c_int32), ("steps", C.c_int64), ("nodes", C.c_int64),
                ("residual", C.c_double), ("t_submit", C.c_double), ("t_admit", C.c_double),
                ("t_done", C.c_double), ("obs", qslbm_obs)]


class qslbm_server_stats_t(C.Structure):
    _fields_ = [("running", C.c_int32), ("pending", C.c_int32), ("sweep_threads", C.c_int32),
                ("sweep_grid", C.c_int32), ("chunks", C.c_int64), ("rebuilds", C.c_int64), ("steps", C.c_int64),
                ("node_steps", C.c_int64), ("device_bytes", C.c_int64)]


# every symbol the header declares (checked by the CPU test-suite)
EXPORTS = ("qslbm_params_init", "qslbm_create", "qslbm_get_units", "qslbm_step", "qslbm_mag_sweeps",
           "qslbm_observables", "qslbm_get_state", "qslbm_set_state", "qslbm_step_host", "qslbm_sync",
           "qslbm_destroy", "qslbm_strerror", "qslbm_last_error", "qslbm_observables_static",
           "qslbm_check_bounded_wait",
           "qslbm_batch_create", "qslbm_batch_step", "qslbm_batch_handle", "qslbm_batch_info",
           "qslbm_batch_destroy", "qslbm_server_create", "qslbm_server_submit", "qslbm_server_run",
           "qslbm_server_poll", "qslbm_server_fields", "qslbm_server_release", "qslbm_server_stats",
           "qslbm_server_destroy")

_lib = None


def load(path: str | None = None):
    """Load libqslbm.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.build()
    L = C.CDLL(path)
    dp = C.POINTER(C.c_double)
    hp = C.c_void_p
    L.qslbm_params_init.argtypes = [C.POINTER(qslbm_params)]
    L.qslbm_params_init.restype = None
    L.qslbm_create.argtypes = [C.POINTER(qslbm_params), C.POINTER(hp)]
    L.qslbm_get_units.argtypes = [hp, C.POINTER(qslbm_units)]
    L.qslbm_step.argtypes = [hp, C.c_int64]
    L.qslbm_mag_sweeps.argtypes = [hp, C.c_int32]
    L.qslbm_observables.argtypes = [hp, C.POINTER(qslbm_obs), dp, dp, dp]
    L.qslbm_get_state.argtypes = [hp, dp, dp, dp, C.POINTER(C.c_int64)]
    L.qslbm_set_state.argtypes = [hp, dp, dp, dp, C.c_int64]
    L.qslbm_step_host.argtypes = [hp, dp, dp, dp, C.c_int64, C.c_int64, dp, dp, dp, C.POINTER(qslbm_obs)]
    L.qslbm_sync.argtypes = [hp]
    L.qslbm_destroy.argtypes = [hp]
    L.qslbm_strerror.argtypes = [C.c_int]
    L.qslbm_strerror.restype = C.c_char_p
    L.qslbm_observables_static.argtypes = [hp, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double,
                                           C.c_int64, C.c_void_p, C.c_void_p]
    L.qslbm_observables_static.restype = C.c_int
    L.qslbm_check_bounded_wait.argtypes = [C.c_double, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_double)]
    L.qslbm_check_bounded_wait.restype = C.c_int
    L.qslbm_batch_create.argtypes = [C.POINTER(qslbm_params), C.c_int32, C.c_void_p, C.POINTER(C.c_void_p)]
    L.qslbm_batch_step.argtypes = [C.c_void_p, C.c_int64]
    L.qslbm_batch_handle.argtypes = [C.c_void_p, C.c_int32, C.POINTER(C.c_void_p)]
    L.qslbm_batch_info.argtypes = [C.c_void_p, C.POINTER(qslbm_batch_info_t)]
    L.qslbm_batch_destroy.argtypes = [C.c_void_p]
    for name in ("qslbm_batch_create", "qslbm_batch_step", "qslbm_batch_handle", "qslbm_batch_info",
                 "qslbm_batch_destroy"):
        getattr(L, name).restype = C.c_int
    L.qslbm_server_create.argtypes = [C.POINTER(qslbm_server_config), C.POINTER(C.c_void_p)]
    L.qslbm_server_submit.argtypes = [C.c_void_p, C.POINTER(qslbm_params), C.c_double, C.c_int64, C.c_int32,
                                      C.POINTER(C.c_int64)]
    L.qslbm_server_run.argtypes = [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
    L.qslbm_server_poll.argtypes = [C.c_void_p, C.POINTER(qslbm_result), C.c_int32, C.POINTER(C.c_int32)]
    L.qslbm_server_fields.argtypes = [C.c_void_p, C.c_int64, dp, dp, dp]
    L.qslbm_server_release.argtypes = [C.c_void_p, C.c_int64]
    L.qslbm_server_stats.argtypes = [C.c_void_p, C.POINTER(qslbm_server_stats_t)]
    L.qslbm_server_destroy.argtypes = [C.c_void_p]
    for name in ("qslbm_server_create", "qslbm_server_submit", "qslbm_server_run", "qslbm_server_poll",
                 "qslbm_server_fields", "qslbm_server_release", "qslbm_server_stats", "qslbm_server_destroy"):
        getattr(L, name).restype = C.c_int
    L.qslbm_last_error.argtypes = []
    L.qslbm_last_error.restype = C.c_char_p
    for name in ("qslbm_create", "qslbm_get_units", "qslbm_step", "qslbm_mag_sweeps", "qslbm_observables",
                 "qslbm_get_state", "qslbm_set_state", "qslbm_step_host", "qslbm_sync", "qslbm_destroy"):
        getattr(L, name).restype = C.c_int
    _lib = L
    return L


class QSLBMError(RuntimeError):
    def __init__(self, code: int, where: str):
        L = load()
        msg = L.qslbm_strerror(code).decode()
        last = L.qslbm_last_error().decode()
        super().__init__(f"{where}: {msg} ({code})" + (f": {last}" if last else ""))
        self.code = code


def check(code: int, where: str) -> int:
    if code != OK:
        raise QSLBMError(code, where)
    return code


def make_params(p: dict, stream: int | None = None) -> qslbm_params:
    """Fill the C parameter struct from a workload dictionary."""
    q = qslbm_params()
    load().qslbm_params_init(C.byref(q))
    q.dim = int(p.get("dim", 3))
    q.nx, q.ny = int(p["nx"]), int(p["ny"])
    q.nz = int(p.get("nz", 1)) if q.dim == 3 else 1
    g = p.get("geometry", "pipe")
    q.geometry = GEOMETRY[g] if isinstance(g, str) else int(g)
    q.diameter = float(p["diameter"])
    c = p.get("center") or (math.nan, math.nan)
    q.center[0], q.center[1] = float(c[0]), float(c[1])
    q.marker_spacing = float(p.get("marker_spacing", 1.0))
    q.Re, q.Ha, q.Rm = float(p["Re"]), float(p["Ha"]), float(p["Rm"])
    q.U0 = float(p.get("U0", 0.0))
    k = p.get("b0_kind", "uniform")
    q.b0_kind = B0_KIND[k] if isinstance(k, str) else int(k)
    d = p.get("b0_dir", (1.0, 0.0, 0.0))
    for i in range(3):
        q.b0_dir[i] = float(d[i])
    q.ramp_center = float(p.get("ramp_center", 0.0))
    q.ramp_width = float(p.get("ramp_width", 1.0))
    q.force_amp = float(p.get("force_amp", 0.0))
    q.force_period = float(p.get("force_period", 0.0))
    q.n_mag = int(p.get("n_mag", 0))
    q.n_mag_cap = int(p.get("n_mag_cap", 270))
    q.nu_ref = float(p.get("nu_ref", 0.0))
    q.eta_ref = float(p.get("eta_ref", 0.0))
    pr = p.get("precision", "fp32")
    q.precision = PRECISION[pr] if isinstance(pr, str) else int(pr)
    q.strict_qs = int(p.get("strict_qs", 0))
    q.seed = int(p.get("seed", 0)) & ((1 << 64) - 1)
    q.perturb = float(p.get("perturb", 0.0))
    ik = p.get("init_kind", "rest")
    q.init_kind = {"rest": 0, "poiseuille": 1}[ik] if isinstance(ik, str) else int(ik)
    k = p.get("sweep_kernel", "auto")
    q.sweep_kernel = SWEEP_KERNEL[k] if isinstance(k, str) else int(k)
    q.alpha = float(p.get("alpha", 1.0))
    q.mag_scheme = int(p.get("mag_scheme", 0))
    q.gamma = float(p.get("gamma", 1.0))
    q.flow_q = int(p.get("flow_q", 0))
    q.flow_scheme = {"single_step": 0, "macroscopic": 1}[p.get("flow_scheme", "single_step")]
    f = p.get("b0_field")
    if f is not None:  # read by qslbm_create; the array only has to outlive that call
        q._field = np.ascontiguousarray(f, dtype=np.float64)
        q.b0_field = q._field.ctypes.data
    q.stream = stream
    return q


def _dptr(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_double))


OBS_KEYS = ("step", "mass", "mass_drift", "E_k", "E_m", "pump", "visc", "joule", "qs_residual",
            "steady_residual", "nan_flag")


def obs_dict(o: qslbm_obs) -> dict:
    return {k: getattr(o, k) for k in OBS_KEYS}


class Solver:
    """One simulated pipe (or channel) held on the GPU by the C library."""

    def __init__(self, params: dict, stream: int | None = None, _handle=None):
        self.L = load()
        self.params = dict(params)
        self._q = make_params(params, stream)
        self._owned = _handle is None
        if _handle is None:
            h = C.c_void_p()
            check(self.L.qslbm_create(C.byref(self._q), C.byref(h)), "qslbm_create")
        else:
            h = _handle
        self.h = h
        u = qslbm_units()
        check(self.L.qslbm_get_units(self.h, C.byref(u)), "qslbm_get_units")
        self.units = {k: getattr(u, k) for k, _ in qslbm_units._fields_}
        self.units["lambda"] = self.units.pop("lambda_")
        self.units["sweep_kernel"] = {SWEEP_PLANES: "planes", SWEEP_RESIDENT: "resident",
                                      SWEEP_SPLIT: "split", SWEEP_FUSED: "fused"}.get(u.sweep_kernel)
        self.n = int(u.nodes)
        self.shape = (self._q.nz, self._q.ny, self._q.nx)

    def close(self):
        if getattr(self, "h", None):
            if self._owned:
                self.L.qslbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def step(self, n: int = 1):
        check(self.L.qslbm_step(self.h, int(n)), "qslbm_step")

    def mag_sweeps(self, n: int):
        check(self.L.qslbm_mag_sweeps(self.h, int(n)), "qslbm_mag_sweeps")

    def sync(self):
        check(self.L.qslbm_sync(self.h), "qslbm_sync")

    def observables(self, fields: bool = False, allow_unstable: bool = False):
        o = qslbm_obs()
        rho = u = b = None
        if fields:
            rho, u, b = np.empty(self.n), np.empty(3 * self.n), np.empty(3 * self.n)
        rc = self.L.qslbm_observables(self.h, C.byref(o), _dptr(rho), _dptr(u), _dptr(b))
        if not (allow_unstable and rc == EUNSTABLE):
            check(rc, "qslbm_observables")
        d = obs_dict(o)
        if fields:
            return d, (rho.reshape(self.shape), u.reshape((3,) + self.shape), b.reshape((3,) + self.shape))
        return d

    def state(self):
        rho, u, b = np.empty(self.n), np.empty(3 * self.n), np.empty(3 * self.n)
        t = C.c_int64()
        check(self.L.qslbm_get_state(self.h, _dptr(rho), _dptr(u), _dptr(b), C.byref(t)), "qslbm_get_state")
        return rho.reshape(self.shape), u.reshape((3,) + self.shape), b.reshape((3,) + self.shape)

    @property
    def t(self) -> int:
        t = C.c_int64()
        check(self.L.qslbm_get_state(self.h, None, None, None, C.byref(t)), "qslbm_get_state")
        return t.value

    def set_state(self, rho=None, u=None, b=None, t: int = 0):
        a = [None if x is None else np.ascontiguousarray(x, dtype=np.float64).ravel() for x in (rho, u, b)]
        check(self.L.qslbm_set_state(self.h, _dptr(a[0]), _dptr(a[1]), _dptr(a[2]), int(t)), "qslbm_set_state")


class Batch:
    """Independent instances advanced together by the library's batched kernels."""

    def __init__(self, params_list, stream: int | None = None):
        self.L = load()
        self.params = [dict(p) for p in params_list]
        arr = (qslbm_params * len(self.params))(*[make_params(p) for p in self.params])
        h = C.c_void_p()
        check(self.L.qslbm_batch_create(arr, len(self.params), stream, C.byref(h)), "qslbm_batch_create")
        self.h = h

    def step(self, n: int = 1):
        check(self.L.qslbm_batch_step(self.h, int(n)), "qslbm_batch_step")

    def member(self, i: int) -> Solver:
        """A non-owning view of instance i (observables and state transfer)."""
        hh = C.c_void_p()
        check(self.L.qslbm_batch_handle(self.h, int(i), C.byref(hh)), "qslbm_batch_handle")
        return Solver(self.params[i], _handle=hh)

    def info(self) -> dict:
        inf = qslbm_batch_info_t()
        check(self.L.qslbm_batch_info(self.h, C.byref(inf)), "qslbm_batch_info")
        d = {k: getattr(inf, k) for k, _ in qslbm_batch_info_t._fields_ if k != "tune_us"}
        d["tune_us"] = list(inf.tune_us)
        return d

    def close(self):
        if getattr(self, "h", None):
            self.L.qslbm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Server:
    """Continuous-batching request loop of the library (qslbm_server_*)."""

    def __init__(self, hbm_budget_bytes: int, chunk_steps: int = 100, max_running: int = 0,
                 precision: str = "fp32", stream: int | None = None, admit: str = "fifo"):
        self.L = load()
        cfg = qslbm_server_config(int(hbm_budget_bytes), int(chunk_steps), int(max_running),
                                  PRECISION[precision], stream, ADMIT[admit])
        h = C.c_void_p()
        check(self.L.qslbm_server_create(C.byref(cfg), C.byref(h)), "qslbm_server_create")
        self.h = h
        self.params = {}
        # a result can be ready as soon as its request is queued (a request
        # above the budget is answered at once): submit records the request's
        # parameters before poll may return its result
        self._lock = threading.Lock()

    def submit(self, params: dict, tol: float = 1e-6, max_steps: int = 100000, keep_fields: bool = False) -> int:
        q = make_params(params)
        rid = C.c_int64()
        with self._lock:
            check(self.L.qslbm_server_submit(self.h, C.byref(q), float(tol), int(max_steps), int(keep_fields),
                                             C.byref(rid)), "qslbm_server_submit")
            self.params[rid.value] = dict(params)
        return rid.value

    def run(self):
        nr, npd = C.c_int32(), C.c_int32()
        check(self.L.qslbm_server_run(self.h, C.byref(nr), C.byref(npd)), "qslbm_server_run")
        return nr.value, npd.value

    def poll(self, max_results: int = 1024):
        arr = (qslbm_result * max_results)()
        n = C.c_int32()
        with self._lock:
            check(self.L.qslbm_server_poll(self.h, arr, int(max_results), C.byref(n)), "qslbm_server_poll")
        out = []
        for r in arr[: n.value]:
            d = {k: getattr(r, k) for k in ("id", "status", "steps", "nodes", "residual", "t_submit", "t_admit",
                                            "t_done")}
            d["obs"] = obs_dict(r.obs)
            out.append(d)
        return out

    def fields(self, rid: int):
        p = self.params[rid]
        nz = int(p.get("nz", 1)) if int(p.get("dim", 3)) == 3 else 1
        n = int(p["nx"]) * int(p["ny"]) * nz
        shape = (nz, int(p["ny"]), int(p["nx"]))
        rho, u, b = np.empty(n), np.empty(3 * n), np.empty(3 * n)
        check(self.L.qslbm_server_fields(self.h, int(rid), _dptr(rho), _dptr(u), _dptr(b)), "qslbm_server_fields")
        return rho.reshape(shape), u.reshape((3,) + shape), b.reshape((3,) + shape)

    def release(self, rid: int):
        check(self.L.qslbm_server_release(self.h, int(rid)), "qslbm_server_release")

    def stats(self) -> dict:
        st = qslbm_server_stats_t()
        check(self.L.qslbm_server_stats(self.h, C.byref(st)), "qslbm_server_stats")
        return {k: getattr(st, k) for k, _ in qslbm_server_stats_t._fields_}

    def close(self):
        if getattr(self, "h", None):
            self.L.qslbm_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
