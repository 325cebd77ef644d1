"""Host-side checks of the C ABI that need no GPU: the library builds, loads,
exports every symbol the header declares, and rejects invalid parameters
before touching the device."""
import ctypes as C
import math
import os
import re

import pytest

from paper_2211_09370_gb300 import _lib
from paper_2211_09370_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "qslbm.h")) as f:
        src = f.read()
    return sorted(set(re.findall(r"\b(qslbm_[a-z_0-9]+)\s*\(", src)))


def test_header_and_binding_agree():
    assert sorted(_lib.EXPORTS) == _declared()


def test_library_exports_every_declared_symbol():
    L = _lib.load()
    for name in _declared():
        assert hasattr(L, name), name


def test_struct_layouts_match_header_sizes():
    # defaults written by the library match the header comments
    p = _lib.qslbm_params()
    _lib.load().qslbm_params_init(C.byref(p))
    assert p.dim == 3 and p.geometry == _lib.PIPE and p.n_mag_cap == 270 and p.marker_spacing == 1.0
    assert math.isnan(p.center[0]) and p.b0_dir[0] == 1.0 and p.precision == _lib.FP32 and p.alpha == 1.0


@pytest.mark.parametrize("bad,why", [
    (dict(dim=4), "dim must be"), (dict(nx=0), "at least 1"), (dict(diameter=-1.0), "diameter"),
    (dict(Re=0.0), "Re and Rm"), (dict(Rm=-1.0), "Re and Rm"), (dict(Ha=-2.0), "Ha must not"),
    (dict(marker_spacing=0.0), "marker_spacing"), (dict(b0_kind=7), "b0_kind"),
    (dict(b0_kind="tanh", ramp_width=0.0), "ramp_width"), (dict(force_amp=0.2, force_period=0.0), "force_period"),
    (dict(precision=5), "precision"), (dict(n_mag=-3), "not be negative"), (dict(perturb=-1.0), "not be negative"),
    (dict(alpha=0.7), "alpha outside"), (dict(alpha=1.5), "alpha outside"), (dict(alpha=-1.0), "alpha outside"),
    (dict(mag_scheme=2), "mag_scheme"),
    (dict(mag_scheme=1), "tau_m"),  # tau_m far above 7/6 at Rm = 1e-3
    (dict(mag_scheme=1, Rm=3.0, U0=0.05, alpha=0.8), "no alpha"), (dict(gamma=-1.0), "gamma outside"),
    (dict(b0_kind="field"), "b0_field"),
    (dict(flow_q=15), "3-D flow_q"), (dict(flow_q=9), "3-D flow_q"), (dict(dim=2, nz=1, flow_q=27), "2-D flow_q"),
    (dict(flow_scheme="macroscopic"), "6 nu"),  # Re = 100: 6 nu < 1, tau < 1
    (dict(flow_scheme="macroscopic", Re=1.0, Ha=5.0, gamma=2.0), "sets gamma"),
])
def test_invalid_parameters_rejected_before_device(bad, why):
    p = W.small_pipe(**bad)
    q = _lib.make_params(p)
    h = C.c_void_p()
    L = _lib.load()
    rc = L.qslbm_create(C.byref(q), C.byref(h))
    assert rc == _lib.EINVAL
    assert not h.value
    # the reason is left in qslbm_last_error
    msg = L.qslbm_last_error().decode()
    assert msg.startswith("invalid parameters: ") and why in msg, msg


def test_null_arguments():
    L = _lib.load()
    assert L.qslbm_create(None, None) == _lib.EINVAL
    assert b"NULL" in L.qslbm_last_error()
    for fn, args in (("qslbm_step", (None, 1)), ("qslbm_observables", (None, None, None, None, None)),
                     ("qslbm_get_state", (None, None, None, None, None)), ("qslbm_sync", (None,)),
                     ("qslbm_mag_sweeps", (None, 1)), ("qslbm_destroy", (None,))):
        assert getattr(L, fn)(*args) == _lib.EINVAL
        assert L.qslbm_last_error().decode().startswith(fn + ":")
    assert L.qslbm_strerror(_lib.EBUDGET).decode().startswith("request exceeds")
    # the step cap and a bounded device wait that gave up share one code
    t = L.qslbm_strerror(_lib.ETIMEOUT).decode()
    assert "step cap" in t and "wait" in t


def test_batch_and_server_refusals_before_the_device():
    # refused on the host, before any device work, with the reason left in
    # qslbm_last_error
    L = _lib.load()
    out = C.c_void_p()
    assert L.qslbm_batch_create(None, 0, None, C.byref(out)) == _lib.EINVAL
    assert b"qslbm_batch_create" in L.qslbm_last_error()
    mixed = (_lib.qslbm_params * 2)(_lib.make_params(W.small_pipe()), _lib.make_params(W.small_pipe(precision="fp64")))
    assert L.qslbm_batch_create(mixed, 2, None, C.byref(out)) == _lib.EINVAL and not out.value
    assert b"member 1" in L.qslbm_last_error()
    flat = (_lib.qslbm_params * 1)(_lib.make_params(W.hartmann_channel_2d(precision="fp32")))
    assert L.qslbm_batch_create(flat, 1, None, C.byref(out)) == _lib.EINVAL
    assert b"not 3-D" in L.qslbm_last_error()
    for cfg, why in (((0, 100, 0, _lib.FP32, None, 0), b"positive"), ((1 << 30, 0, 0, _lib.FP32, None, 0), b"positive"),
                     ((1 << 30, 100, 0, 9, None, 0), b"precision"), ((1 << 30, 100, 0, _lib.FP32, None, 5), b"admission")):
        c = _lib.qslbm_server_config(*cfg)
        assert L.qslbm_server_create(C.byref(c), C.byref(out)) == _lib.EINVAL and not out.value
        assert why in L.qslbm_last_error()
    assert L.qslbm_server_create(None, C.byref(out)) == _lib.EINVAL
    assert b"NULL" in L.qslbm_last_error()
    assert L.qslbm_server_submit(None, None, 1e-6, 10, 0, None) == _lib.EINVAL
    assert b"qslbm_server_submit" in L.qslbm_last_error()
    n = C.c_int32()
    for fn, args in (("qslbm_batch_step", (None, 1)), ("qslbm_batch_handle", (None, 0, C.byref(out))),
                     ("qslbm_batch_info", (None, None)), ("qslbm_batch_destroy", (None,)),
                     ("qslbm_server_run", (None, None, None)), ("qslbm_server_poll", (None, None, 0, C.byref(n))),
                     ("qslbm_server_fields", (None, 1, None, None, None)), ("qslbm_server_release", (None, 1)),
                     ("qslbm_server_stats", (None, None)), ("qslbm_server_destroy", (None,))):
        assert getattr(L, fn)(*args) == _lib.EINVAL
        assert L.qslbm_last_error().decode().startswith(fn + ":")


def test_bounded_wait_check_rejects_bad_limits_before_the_device():
    L = _lib.load()
    g, w = C.c_int32(), C.c_double()
    assert L.qslbm_check_bounded_wait(0.0, 0, C.byref(g), C.byref(w)) == _lib.EINVAL
    assert L.qslbm_check_bounded_wait(5.0, 0, C.byref(g), C.byref(w)) == _lib.EINVAL
    assert L.qslbm_check_bounded_wait(0.1, 0, None, C.byref(w)) == _lib.EINVAL


def test_static_diagnostics_null_arguments_set_the_error_text():
    # a NULL handle or a negative step count is refused on the host, and the
    # reason is left in qslbm_last_error like every other refusal
    L = _lib.load()
    rc = L.qslbm_observables_static(None, None, None, None, None, 0.0, 0, None, None)
    assert rc == _lib.EINVAL
    assert b"NULL" in L.qslbm_last_error()


STRUCTS = ["qslbm_params", "qslbm_units", "qslbm_obs", "qslbm_batch_info_t", "qslbm_server_config",
           "qslbm_result", "qslbm_server_stats_t"]


def test_struct_sizes_and_offsets_match_the_header(tmp_path):
    # a C program built against the header prints every struct's size and
    # every field's offset; the binding's ctypes layouts must agree
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "qslbm.h"', "int main(void) {"]
    for name in STRUCTS:
        lines.append(f'  printf("{name} . %zu\\n", sizeof({name}));')
        for field, _ in getattr(_lib, name)._fields_:
            cfield = field[:-1] if field.endswith("_") else field  # a Python keyword in the binding
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {cfield}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    for line in out.splitlines():
        name, field, value = line.split()
        cls = getattr(_lib, name)
        want = C.sizeof(cls) if field == "." else getattr(cls, field).offset
        assert int(value) == want, (name, field, int(value), want)
