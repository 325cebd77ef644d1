"""The allocation-free diagnostics entry point (qslbm_observables_static).

It exists for callers that cannot allocate device memory when they need the
diagnostics (a stream being captured into a CUDA graph refuses cudaMalloc; a
framework allocator may own the whole pool).  Its partial sums live in a fixed
array inside the library.  Here it is called through the C ABI on fields the
test holds in torch tensors and compared with qslbm_observables, which
reduces the same fields with its own allocated scratch, on two calls in a row.
This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2211_09370_gb300 import _lib
from paper_2211_09370_gb300 import workloads as W

pytestmark = pytest.mark.gpu

KEYS = ("mass", "mass_drift", "E_k", "E_m", "pump", "visc", "joule", "qs_residual", "steady_residual", "nan_flag")


def _device_fields(torch, state, dtype):
    rho, u, b = state
    dev = "cuda"
    return (torch.tensor(rho - 1.0, dtype=dtype, device=dev).contiguous(),
            torch.tensor(u, dtype=dtype, device=dev).contiguous(),
            torch.tensor(b, dtype=dtype, device=dev).contiguous())


@pytest.mark.parametrize("flow_q", [0, 27])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_static_diagnostics_match_allocating_entry(precision, flow_q):
    # on the default D3Q19 flow lattice and on the paper's D3Q27, whose
    # Laplacian and isotropic gradient the viscous, Joule and Lorentz terms use
    torch = pytest.importorskip("torch")
    dtype = torch.float64 if precision == "fp64" else torch.float32
    p = W.small_pipe(nx=26, ny=24, nz=10, diameter=18.0, precision=precision, Ha=10.0, Rm=1e-2, n_mag=40,
                     perturb=0.01, flow_q=flow_q)
    with _lib.Solver(p) as s:
        s.step(5)
        s.observables()  # the allocating entry's reference velocity is now u(t = 5)
        _, u_prev, _ = s.state()
        s.step(3)
        state = s.state()
        want = s.observables()
        drho, u, b = _device_fields(torch, state, dtype)
        up = torch.tensor(u_prev, dtype=dtype, device="cuda").contiguous()
        fb = s.units["F0"]  # constant body force in this workload
        for call in range(2):
            out = torch.full((10,), float("nan"), dtype=torch.float64, device="cuda")
            stream = torch.cuda.current_stream().cuda_stream
            rc = s.L.qslbm_observables_static(s.h, C.c_void_p(drho.data_ptr()), C.c_void_p(u.data_ptr()),
                                              C.c_void_p(b.data_ptr()), C.c_void_p(up.data_ptr()), fb, 3,
                                              C.c_void_p(out.data_ptr()), C.c_void_p(stream))
            assert rc == 0, _lib.load().qslbm_last_error()
            torch.cuda.synchronize()
            got = dict(zip(KEYS, out.cpu().numpy().tolist()))
            for k in KEYS:
                # mass_drift is itself a round-off-sized number: bound it absolutely
                tol_abs = 1e-12 if k == "mass_drift" else 1e-300
                assert got[k] == pytest.approx(want[k], rel=1e-12, abs=tol_abs), (call, k, got[k], want[k])


def test_static_diagnostics_reject_too_many_planes():
    torch = pytest.importorskip("torch")
    nz = 4097
    p = W.small_pipe(nx=4, ny=4, nz=nz, diameter=2.0, geometry="none", perturb=0.0, n_mag=1)
    with _lib.Solver(p) as s:
        x = torch.zeros(3 * s.n, dtype=torch.float32, device="cuda")
        out = torch.zeros(10, dtype=torch.float64, device="cuda")
        rc = s.L.qslbm_observables_static(s.h, C.c_void_p(x.data_ptr()), C.c_void_p(x.data_ptr()),
                                          C.c_void_p(x.data_ptr()), C.c_void_p(x.data_ptr()), 0.0, 0,
                                          C.c_void_p(out.data_ptr()), None)
        assert rc == _lib.EINVAL
        assert "4096" in _lib.load().qslbm_last_error().decode()
