"""Plain FP64 CPU oracle for the single-step simplified LBM of arXiv 2211.09370.

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
benchmark's ``cpu_baseline`` / reference leg may use this package; the product
library never imports, links or calls it.  The arithmetic lives in
``qslbm_oracle.c`` (plain C, binary64, ``-ffp-contract=off``); this module only
builds it and marshals arguments through ctypes.

Parity status of each oracle function is recorded in the header of
``qslbm_oracle.c`` and pinned by ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qslbm_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libqslbm_oracle.so")
_lock = threading.Lock()
_lib = None

GEOMETRY = {"channel": 0, "pipe": 1, "none": 2}
B0_KIND = {"uniform": 0, "tanh": 1, "field": 2}
FLOW_SCHEME = {"single_step": 0, "macroscopic": 1}


class _Params(C.Structure):
    _fields_ = [
        ("dim", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("geometry", C.c_int),
        ("diameter", C.c_double), ("cx", C.c_double), ("cy", C.c_double), ("marker_spacing", C.c_double),
        ("Re", C.c_double), ("Ha", C.c_double), ("Rm", C.c_double), ("U0", C.c_double),
        ("b0_kind", C.c_int), ("b0_dir", C.c_double * 3), ("ramp_center", C.c_double),
        ("ramp_width", C.c_double), ("force_amp", C.c_double), ("force_period", C.c_double),
        ("n_mag", C.c_int), ("n_mag_cap", C.c_int), ("nu_ref", C.c_double), ("eta_ref", C.c_double),
        ("seed", C.c_uint64), ("perturb", C.c_double), ("strict_qs", C.c_int), ("alpha", C.c_double),
        ("mag_scheme", C.c_int), ("gamma", C.c_double), ("b0_field", C.c_void_p), ("flow_q", C.c_int),
        ("flow_scheme", C.c_int),
    ]


class _Derived(C.Structure):
    _fields_ = [(k, C.c_double) for k in
                ("R", "U0", "nu", "tau", "eta", "B0", "F0", "c_mag", "lambda_", "lambda_m", "cs2", "cm2")]
    _fields_ += [("n_mag", C.c_int), ("n_markers", C.c_int), ("tau_m", C.c_double), ("gamma", C.c_double)]


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build`` (gcc, OpenMP, no FP contraction)."""
    with _lock:
        if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
            return _LIB
        os.makedirs(os.path.dirname(_LIB), exist_ok=True)
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = C.CDLL(path)
        L.orc_create.restype = C.c_void_p
        L.orc_create.argtypes = [C.POINTER(_Params)]
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_step.argtypes = [C.c_void_p, C.c_long]
        L.orc_mag_sweeps.argtypes = [C.c_void_p, C.c_int]
        L.orc_get_derived.argtypes = [C.c_void_p, C.POINTER(_Derived)]
        L.orc_derive.argtypes = [C.POINTER(_Params), C.POINTER(_Derived)]
        L.orc_derive.restype = C.c_int
        L.orc_nodes.restype = C.c_long
        L.orc_nodes.argtypes = [C.c_void_p]
        L.orc_time.restype = C.c_long
        L.orc_time.argtypes = [C.c_void_p]
        dp = C.POINTER(C.c_double)
        L.orc_get_state.argtypes = [C.c_void_p, dp, dp, dp]
        L.orc_set_state.argtypes = [C.c_void_p, dp, dp, dp, C.c_long]
        L.orc_markers.restype = C.c_int
        L.orc_markers.argtypes = [C.c_void_p, dp, dp, dp, dp, dp, dp]
        L.orc_ib_apply_field.argtypes = [C.c_void_p, dp, C.c_int]
        L.orc_observables.argtypes = [C.c_void_p, dp]
        L.orc_kernel1d.restype = C.c_double
        L.orc_kernel1d.argtypes = [C.c_double]
        L.orc_splitmix64.restype = C.c_uint64
        L.orc_splitmix64.argtypes = [C.c_uint64]
        L.orc_gzs_terms.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, dp, dp, dp, C.POINTER(C.c_int),
                                    C.POINTER(C.c_int)]
        L.orc_flow_update_with_force.argtypes = [C.c_void_p, dp]
        L.orc_force.argtypes = [C.c_void_p, dp]
        L.orc_flow_lattice.restype = C.c_int
        L.orc_flow_lattice.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_int), dp]
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_double))


def make_params(p: dict) -> _Params:
    """Fill the oracle's own parameter struct from a workload dictionary."""
    q = _Params()
    q.dim = int(p.get("dim", 3))
    q.nx, q.ny = int(p["nx"]), int(p["ny"])
    q.nz = int(p.get("nz", 1)) if q.dim == 3 else 1
    g = p.get("geometry", "pipe")
    q.geometry = GEOMETRY[g] if isinstance(g, str) else int(g)
    q.diameter = float(p["diameter"])
    cx = p.get("center", (float("nan"), float("nan")))
    q.cx = (q.nx - 1) / 2.0 if cx is None or math.isnan(cx[0]) else float(cx[0])
    q.cy = (q.ny - 1) / 2.0 if cx is None or math.isnan(cx[1]) else float(cx[1])
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
    q.seed = int(p.get("seed", 0)) & ((1 << 64) - 1)
    q.perturb = float(p.get("perturb", 0.0))
    q.strict_qs = int(p.get("strict_qs", 0))
    q.alpha = float(p.get("alpha", 1.0))
    q.mag_scheme = int(p.get("mag_scheme", 0))
    q.gamma = float(p.get("gamma", 1.0))
    q.flow_q = int(p.get("flow_q", 0))
    q.flow_scheme = FLOW_SCHEME[p.get("flow_scheme", "single_step")]
    f = p.get("b0_field")
    if f is not None:  # copied by orc_create; the array only has to outlive the call
        q._field = np.ascontiguousarray(f, dtype=np.float64)
        q.b0_field = q._field.ctypes.data
    return q


def derive(p: dict) -> dict:
    d = _Derived()
    rc = lib().orc_derive(C.byref(make_params(p)), C.byref(d))
    if rc != 0:
        raise ValueError("invalid parameters")
    return _derived_dict(d)


def _derived_dict(d: _Derived) -> dict:
    out = {k: getattr(d, k) for k, _ in _Derived._fields_}
    out["lambda"] = out.pop("lambda_")
    return out


OBS_KEYS = ("mass", "mass_drift", "E_k", "E_m", "pump", "visc", "joule", "qs_residual", "steady_residual",
            "nan_flag", "time")


class Oracle:
    """One simulated instance held by the C oracle (fields in FP64)."""

    def __init__(self, params: dict):
        self._p = make_params(params)
        self._h = lib().orc_create(C.byref(self._p))
        if not self._h:
            raise ValueError("oracle rejected the parameters")
        self.n = lib().orc_nodes(self._h)
        self.shape = (self._p.nz, self._p.ny, self._p.nx)

    def close(self):
        if self._h:
            lib().orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def derived(self) -> dict:
        d = _Derived()
        lib().orc_get_derived(self._h, C.byref(d))
        return _derived_dict(d)

    def step(self, n: int = 1):
        lib().orc_step(self._h, int(n))

    def flow_update_with_force(self, F):
        """One flow update with a given force field F [3][nz][ny][nx] (no IB on u)."""
        F = np.ascontiguousarray(F, dtype=np.float64)
        lib().orc_flow_update_with_force(self._h, _ptr(F))

    def force(self):
        """The force field [3][nz][ny][nx] the next flow update adds: the body
        force plus the Lorentz force J x (B^ext + b) of the current state."""
        F = np.empty(3 * self.n)
        lib().orc_force(self._h, _ptr(F))
        return F.reshape((3,) + self.shape)

    def mag_sweeps(self, n: int):
        lib().orc_mag_sweeps(self._h, int(n))

    @property
    def t(self) -> int:
        return lib().orc_time(self._h)

    def state(self):
        rho = np.empty(self.n)
        u = np.empty(3 * self.n)
        b = np.empty(3 * self.n)
        lib().orc_get_state(self._h, _ptr(rho), _ptr(u), _ptr(b))
        return rho.reshape(self.shape), u.reshape((3,) + self.shape), b.reshape((3,) + self.shape)

    def set_state(self, rho=None, u=None, b=None, t=None):
        a = [None if x is None else np.ascontiguousarray(x, dtype=np.float64).ravel() for x in (rho, u, b)]
        lib().orc_set_state(self._h, _ptr(a[0]), _ptr(a[1]), _ptr(a[2]), int(self.t if t is None else t))

    def markers(self) -> dict:
        m = lib().orc_markers(self._h, None, None, None, None, None, None)
        arr = {k: np.empty(m) for k in ("X", "Y", "Z", "d", "s", "sm")}
        lib().orc_markers(self._h, *[_ptr(arr[k]) for k in ("X", "Y", "Z", "d", "s", "sm")])
        return arr

    def ib_apply(self, field, magnetic: bool):
        f = np.ascontiguousarray(field, dtype=np.float64).copy()
        lib().orc_ib_apply_field(self._h, _ptr(f), 1 if magnetic else 0)
        return f.reshape(np.shape(field))

    def observables(self) -> dict:
        out = np.empty(11)
        lib().orc_observables(self._h, _ptr(out))
        return dict(zip(OBS_KEYS, out.tolist()))


def kernel1d(r: float) -> float:
    return lib().orc_kernel1d(float(r))


def splitmix64(x: int) -> int:
    return int(lib().orc_splitmix64(int(x) & ((1 << 64) - 1)))


def gzs_terms(dim: int, tau: float, u, F, gamma: float = 1.0, flow_q: int = 0):
    """GZS forcing terms F_i for every flow-lattice direction (with the time
    step rescaled by gamma; flow_q = 27 for the D3Q27 lattice); returns
    (F_i, c_i)."""
    u = np.asarray(u, dtype=np.float64)
    F = np.asarray(F, dtype=np.float64)
    Fi = np.zeros(27)
    c = np.zeros(81, dtype=np.int32)
    q = C.c_int(0)
    lib().orc_gzs_terms(int(dim), int(flow_q), float(tau), float(gamma), _ptr(u), _ptr(F), _ptr(Fi), C.byref(q),
                        c.ctypes.data_as(C.POINTER(C.c_int)))
    return Fi[: q.value], c.reshape(27, 3)[: q.value]


def flow_lattice(dim: int, flow_q: int = 0):
    """The oracle's flow lattice: (c_i [q, 3], w_i [q])."""
    c = np.zeros(81, dtype=np.int32)
    w = np.zeros(27)
    q = lib().orc_flow_lattice(int(dim), int(flow_q), c.ctypes.data_as(C.POINTER(C.c_int)), _ptr(w))
    return c.reshape(27, 3)[:q].copy(), w[:q].copy()
