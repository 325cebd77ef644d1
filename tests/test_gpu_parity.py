"""GPU parity: the CUDA library, called through its C ABI, against the CPU oracle.

Tolerances (relative L2 over the compared nodes): FP64 path <= 1e-12 on rho,
u and b, and |rho - rho_oracle| <= 1e-12 at every node (rho is close to one, so
its relative L2 alone would hide density errors); FP32 path <= 1e-4 on u and b,
and rho within 1e-3 of the oracle's rho - 1 scale (FP32 stores rho - 1).
"""
import importlib.util
import os

import numpy as np
import pytest

import oracle
from paper_2211_09370_gb300 import workloads as W
from paper_2211_09370_gb300._lib import EUNSTABLE, QSLBMError, Solver
from tests.parity_cases import DEGENERATE, FP64_CASES, MAC_CASES, Q27_CASES, degenerate, mac_case

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
_spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "golden", "make_golden.py"))
golden = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(golden)

TOL = {"fp64": 1e-12, "fp32": 1e-4}


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / nb if nb > 0 else np.linalg.norm(a)


def check_fields(got, want, precision, what=""):
    rho, u, b = got
    orho, ou, ob = want
    tol = TOL[precision]
    assert rel(u, ou) <= tol, f"{what} u rel-L2 {rel(u, ou):.3e}"
    if np.linalg.norm(ob) > 0:
        assert rel(b, ob) <= tol, f"{what} b rel-L2 {rel(b, ob):.3e}"
    else:
        assert np.abs(b).max() == 0.0
    if precision == "fp64":
        # rho is close to one; the bound is also applied node by node
        assert rel(rho, orho) <= 1e-12, f"{what} rho rel-L2 {rel(rho, orho):.3e}"
        assert np.abs(rho - orho).max() <= 1e-12, f"{what} rho max {np.abs(rho - orho).max():.3e}"
    else:
        scale = max(np.abs(orho - 1).max(), 1e-300)
        assert np.abs(rho - orho).max() / scale <= 1e-3 or np.abs(rho - orho).max() <= 1e-7


def run_both(p, steps, t0=0):
    o = oracle.Oracle(p)
    with Solver(p) as s:
        if t0:
            rho, u, b = s.state()
            s.set_state(rho, u, b, t=t0)
            r, uu, bb = o.state()
            o.set_state(r, uu, bb, t=t0)
        s.step(steps)
        got = s.state()
    o.step(steps)
    return got, o.state(), o


# ------------------------------------------------------- small, ragged sizes

KERNELS = ["planes", "resident", "split"]


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("name", sorted(FP64_CASES))
def test_parity_cases(name, precision, kernel):
    # ragged planes (e.g. 29 x 27 = 783 nodes: two 512-thread strides plus a
    # tail), ramped field with a pulsating force, an odd 2-D channel, and a
    # smooth start over 150 steps; each on both sweep kernels
    p, steps, t0 = FP64_CASES[name]
    got, want, _ = run_both(dict(p, precision=precision, sweep_kernel=kernel), steps, t0=t0)
    check_fields(got, want, precision, name)


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("case", sorted(DEGENERATE))
def test_degenerate_cases_fp64(case, kernel):
    p, steps = degenerate(case)
    got, want, _ = run_both(dict(p, precision="fp64", sweep_kernel=kernel), steps)
    check_fields(got, want, "fp64", case)


@pytest.mark.parametrize("kernel", KERNELS)
def test_mag_sweeps_with_frozen_velocity_fp64(kernel):
    p = W.small_pipe(nx=22, ny=22, nz=6, diameter=15.0, precision="fp64", sweep_kernel=kernel)
    z, y, x = np.meshgrid(np.arange(6.0), np.arange(22.0), np.arange(22.0), indexing="ij")
    u = np.stack([0.01 * np.sin(2 * np.pi * y / 22), 0.02 * np.cos(2 * np.pi * x / 22), 0.03 + 0.0 * x])
    o = oracle.Oracle(p)
    o.set_state(np.ones_like(x), u, np.zeros_like(u), t=0)
    o.mag_sweeps(300)
    with Solver(p) as s:
        s.set_state(np.ones_like(x), u, np.zeros_like(u), t=0)
        s.mag_sweeps(300)
        _, gu, gb = s.state()
    _, ou, ob = o.state()
    assert rel(gb, ob) <= 1e-12
    np.testing.assert_array_equal(gu, u)


@pytest.mark.parametrize("kernel", KERNELS + ["fused"])
@pytest.mark.parametrize("shape", [(22, 22, 6), (36, 21, 7), (64, 40, 9)])
def test_mag_sweeps_with_frozen_velocity_fp32(kernel, shape):
    # FP32 sweeps (the flux-component form and, for even nx, the node-pair
    # kernel; the fused kernel for nx a multiple of 4): tiles with ghost
    # columns and rows, ramped field
    nx, ny, nz = shape
    if kernel == "fused" and nx % 4:
        pytest.skip("the fused kernel takes nx a multiple of 4")
    p = W.small_pipe(nx=nx, ny=ny, nz=nz, diameter=min(nx, ny) - 6.0, precision="fp32", sweep_kernel=kernel,
                     b0_kind="tanh", ramp_center=nz / 2, ramp_width=2.0, Ha=30.0, Rm=0.05)
    z, y, x = np.meshgrid(np.arange(float(nz)), np.arange(float(ny)), np.arange(float(nx)), indexing="ij")
    u = np.stack([0.01 * np.sin(2 * np.pi * y / ny), 0.02 * np.cos(2 * np.pi * x / nx), 0.03 + 0.001 * z])
    o = oracle.Oracle(dict(p, precision="fp64"))
    o.set_state(np.ones_like(x), u, np.zeros_like(u), t=0)
    o.mag_sweeps(120)
    with Solver(p) as s:
        s.set_state(np.ones_like(x), u, np.zeros_like(u), t=0)
        s.mag_sweeps(120)
        _, gu, gb = s.state()
    _, ou, ob = o.state()
    assert rel(gb, ob) <= 1e-4
    np.testing.assert_array_equal(gu, u.astype(np.float32).astype(np.float64))


ACCEL_CASES = {
    # accelerated sweep (Sec. V.H) at the smallest stable alpha of each lattice
    "pipe_ramp": (dict(nx=24, ny=22, nz=10, diameter=16.0, Re=200.0, Ha=30.0, Rm=0.05, b0_kind="tanh",
                       ramp_center=5.0, ramp_width=2.0, perturb=0.0, n_mag=30, alpha=0.75), 30),
    "pipe_odd": (dict(nx=21, ny=19, nz=6, diameter=14.0, perturb=0.0, n_mag=20, alpha=0.8), 25),
}


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("name", sorted(ACCEL_CASES))
def test_accelerated_sweep_parity(name, precision, kernel):
    kw, steps = ACCEL_CASES[name]
    p = W.small_pipe(precision=precision, sweep_kernel=kernel, **kw)
    got, want, _ = run_both(p, steps)
    check_fields(got, want, precision, name)


def test_accelerated_sweep_parity_2d_channel():
    p = W.hartmann_channel_2d(nx=37, ny=20, diameter=19.0, n_mag=40, perturb=0.0, alpha=2.0 / 3.0,
                              precision="fp64")
    got, want, _ = run_both(p, 40)
    check_fields(got, want, "fp64", "channel alpha 2/3")


TIME_CASES = {
    # time-resolved magnetic update (Sec. III.D, one per flow step), tau_m 0.9 and 0.7
    "pipe_ramp": (dict(nx=24, ny=22, nz=10, diameter=16.0, U0=0.05, Re=50.0, Ha=10.0, Rm=4.0, b0_kind="tanh",
                       ramp_center=5.0, ramp_width=2.0, perturb=0.0, mag_scheme=1), 60),
    "pipe_odd": (dict(nx=21, ny=19, nz=6, diameter=14.0, U0=0.05, Re=30.0, Ha=8.0, Rm=7.0, perturb=0.0,
                      mag_scheme=1), 60),
}


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("name", sorted(TIME_CASES))
def test_time_resolved_update_parity(name, precision, kernel):
    kw, steps = TIME_CASES[name]
    p = W.small_pipe(precision=precision, sweep_kernel=kernel, **kw)
    with Solver(p) as s:
        assert s.units["n_mag"] == 1 and 0.5 < s.units["tau_m"] <= 7 / 6
    got, want, _ = run_both(p, steps)
    check_fields(got, want, precision, name)


def test_time_resolved_update_parity_2d_channel():
    p = W.hartmann_channel_2d(nx=37, ny=20, diameter=19.0, U0=0.05, Rm=3.0, perturb=0.0, mag_scheme=1,
                              precision="fp64")
    got, want, _ = run_both(p, 80)
    check_fields(got, want, "fp64", "channel time-resolved")


GAMMA_CASES = {
    # time step rescaled by gamma (Sec. VII): quasi-static sweeps, gamma = 2
    "qs_ramp": (dict(nx=24, ny=22, nz=10, diameter=16.0, U0=0.05, Re=50.0, Ha=20.0, Rm=0.05, b0_kind="tanh",
                     ramp_center=5.0, ramp_width=2.0, perturb=0.0, n_mag=30, force_amp=0.2, force_period=40.0,
                     gamma=2.0), 40),
    # Pr_m = 4 as in the paper's example (nu = 0.08, eta = 0.02), gamma = 4, time-resolved
    # update; U0 = 0.02 keeps the cell Peclet number U0 / eta at one
    "time_prm4": (dict(nx=22, ny=20, nz=8, diameter=16.0, U0=0.02, Re=2.0, Ha=6.0, Rm=8.0, perturb=0.0,
                       mag_scheme=1, gamma=4.0), 60),
}


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("name", sorted(GAMMA_CASES))
def test_rescaled_time_step_parity(name, precision, kernel):
    kw, steps = GAMMA_CASES[name]
    p = W.small_pipe(precision=precision, sweep_kernel=kernel, **kw)
    got, want, o = run_both(p, steps)
    check_fields(got, want, precision, name)


def _magnet_case(**kw):
    nx, ny, D = 26, 24, 18.0
    return W.small_pipe(nx=nx, ny=ny, nz=8, diameter=D, U0=0.05, Re=60.0, Ha=15.0, Rm=5e-3, perturb=0.0,
                        n_mag=40, b0_kind="field", b0_field=W.six_magnet_field(nx, ny, D), **kw)


@pytest.mark.parametrize("kernel", ["planes", "split"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_six_magnet_field_parity(precision, kernel):
    # the six-magnet applied field of Sec. VI as a z-invariant in-plane field
    p = _magnet_case(precision=precision, sweep_kernel=kernel)
    got, want, o = run_both(p, 30)
    check_fields(got, want, precision, "six magnets")
    with Solver(p) as s:
        assert s.units["sweep_kernel"] in ("planes", "split")


def test_six_magnet_field_observables_and_auto_kernel_fp64():
    p = _magnet_case(precision="fp64")
    o = oracle.Oracle(p)
    with Solver(p) as s:
        assert s.units["sweep_kernel"] == "split"  # the resident kernel takes uniform / per-plane fields only
        s.step(10)
        s.observables()
        o.step(10)
        o.observables()
        s.step(5)
        o.step(5)
        g, w = s.observables(), o.observables()
    for k in ("E_k", "E_m", "pump", "visc", "joule", "qs_residual", "steady_residual"):
        assert g[k] == pytest.approx(w[k], rel=1e-9, abs=1e-300), k


# the paper's own D3Q27 flow lattice: the 3-D cases above on it, every sweep
# kernel, both precisions
@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("name", sorted(Q27_CASES))
def test_d3q27_parity(name, precision, kernel):
    p, steps, t0 = Q27_CASES[name]
    p = dict(p, precision=precision, sweep_kernel=kernel)
    with Solver(p) as s:
        assert s.units["flow_q"] == 27
    got, want, _ = run_both(p, steps, t0=t0)
    check_fields(got, want, precision, name + " D3Q27")


# the macroscopic scheme for tau >= 1 (Sec. V.G), every sweep kernel, both precisions
@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("name", sorted(MAC_CASES))
def test_macroscopic_scheme_parity(name, precision, kernel):
    p, steps = mac_case(name, precision=precision, sweep_kernel=kernel)
    with Solver(p) as s:
        u = s.units
        assert u["tau"] == 1.0 and u["gamma"] == pytest.approx(6 * u["nu"], rel=1e-15) and u["gamma"] > 1
    got, want, _ = run_both(p, steps)
    check_fields(got, want, precision, name + " macroscopic")


def test_d3q27_differs_from_d3q19():
    # the lattice choice reaches the result: the same case on the two lattices
    # differs far beyond the FP64 bound
    p, steps, t0 = FP64_CASES["smooth_pipe_long"]
    outs = []
    for q in (0, 27):
        with Solver(dict(p, precision="fp64", flow_q=q)) as s:
            s.step(steps)
            outs.append(s.state()[1])
    assert rel(outs[1], outs[0]) > 1e-6


@pytest.mark.parametrize("flow_q", [0, 27])
def test_observables_match_oracle_fp64(flow_q):
    p = W.small_pipe(nx=26, ny=26, nz=8, diameter=18.0, precision="fp64", Ha=10.0, Rm=1e-2, perturb=0.0,
                     flow_q=flow_q)
    o = oracle.Oracle(p)
    with Solver(p) as s:
        s.step(10)
        s.observables()
        o.step(10)
        o.observables()
        s.step(7)
        o.step(7)
        g = s.observables()
        w = o.observables()
    assert g["step"] == 17
    for k in ("mass", "E_k", "E_m", "pump", "visc", "joule", "qs_residual", "steady_residual"):
        assert g[k] == pytest.approx(w[k], rel=1e-9, abs=1e-300), k
    assert abs(g["mass_drift"]) < 1e-13 and g["nan_flag"] == 0


# ---------------------------------------------------------- full workloads

@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_hartmann_channel_full_horizon(precision):
    g = golden.load("hartmann_2000")
    p = W.hartmann_channel_2d(precision=precision)
    with Solver(p) as s:
        s.step(int(g["steps"]))
        got = s.state()
    check_fields(got, (g["rho"], g["u"], g["b"]), precision, "hartmann 2000")


def _sampled(p, g, precision):
    with Solver(p) as s:
        t0 = int(g["t0"])
        if t0:
            rho, u, b = s.state()
            s.set_state(rho, u, b, t=t0)
        s.step(int(g["steps"]))
        rho, u, b = s.state()
    idx = g["idx"]
    got = np.concatenate([rho.reshape(1, -1), u.reshape(3, -1), b.reshape(3, -1)])[:, idx]
    want = g["fields"]
    check_fields((got[0], got[1:4], got[4:7]), (want[0], want[1:4], want[4:7]), precision, "sampled")


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_pipe_64x64x128_full_size_sampled(precision):
    g = golden.load("pipe_64x64x128")
    _sampled(W.pipe_64x64x128(precision=precision), g, precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_ramp_96x96x512_full_size_sampled(precision):
    g = golden.load("ramp_96x96x512")
    _sampled(W.pipe_ramp_96x96x512(Rm=1e-2, precision=precision, perturb=0.01, seed=7), g, precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("rm", ["1e-4", "1e-3", "1e-1", "1"])
def test_ramp_96x96x512_rm_sweep_sampled(rm, precision):
    # the other four magnetic Reynolds numbers of the ramped pipe's sweep
    # (N_mag = 270, 270, 176, 18), each against its oracle fixture
    g = golden.load(f"ramp_96x96x512_rm{rm}")
    _sampled(W.pipe_ramp_96x96x512(Rm=float(rm), precision=precision, perturb=0.01, seed=7), g, precision)


@pytest.mark.parametrize("shape", [(72, 72), (71, 72)], ids=["pairs", "odd_nx"])
def test_resident_large_plane_form_fp32(shape):
    # planes of 4097 to 8192 nodes take the resident kernel's large-plane shape
    # (512 threads x 16 nodes in FP32); even nx moves node pairs, odd nx single
    # nodes
    nx, ny = shape
    p = W.small_pipe(nx=nx, ny=ny, nz=10, diameter=64.0, perturb=0.0, n_mag=60, precision="fp32",
                     sweep_kernel="resident")
    assert 4096 < nx * ny <= 8192
    with Solver(p) as s:
        assert s.units["sweep_kernel"] == "resident"
    got, want, _ = run_both(p, 8)
    check_fields(got, want, "fp32", f"resident {nx}x{ny}")


def test_resident_large_plane_form_fp64():
    # in FP64 a plane above 4096 nodes fits the resident kernel's shared memory
    # only without wall tables: a periodic box of 65 x 64 planes
    p = W.small_pipe(nx=65, ny=64, nz=6, diameter=40.0, geometry="none", perturb=0.02, seed=5, n_mag=40,
                     precision="fp64", sweep_kernel="resident")
    with Solver(p) as s:
        assert s.units["sweep_kernel"] == "resident"
    got, want, _ = run_both(p, 3)
    check_fields(got, want, "fp64", "resident 65x64 periodic")


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("name", ["small_pipe", "smooth_pipe_long"])
def test_viscosity_scaled_ib_parity(name, precision, kernel):
    # Sec. V.E with a reference viscosity below nu: lambda = nu / nu_ref = 2, so
    # the wall correction on u carries s_j = lambda / (d (1 + d (lambda - 1)))
    # instead of 1/d; two of the parity cases above with nu_ref = nu / 2
    p, steps, t0 = FP64_CASES[name]
    nu = oracle.derive(dict(p, precision="fp64"))["nu"]
    p = dict(p, nu_ref=nu / 2.0, precision=precision, sweep_kernel=kernel)
    assert oracle.derive(dict(p, precision="fp64"))["lambda"] == pytest.approx(2.0, rel=1e-14)
    with Solver(p) as s:
        assert s.units["lambda"] == pytest.approx(2.0, rel=1e-14)
    got, want, _ = run_both(p, steps, t0=t0)
    check_fields(got, want, precision, name + " lambda 2")


# ------------------------------------------------ the fused sweep + IB kernel

# (nx, ny, nz, diameter): two bands sharing rows, four bands with the last one
# shifted, eight equal bands; chunks of one plane up to several planes; the
# widths 64, 96 and 128 take the kernel's compile-time instantiations
FUSED_SHAPES = [(24, 22, 10, 16.0), (28, 27, 11, 19.0), (64, 64, 12, 56.0), (96, 96, 8, 88.0), (40, 36, 64, 28.0),
                (128, 40, 12, 32.0), (96, 96, 512, 88.0)]


@pytest.mark.parametrize("shape", FUSED_SHAPES, ids=lambda s: "x".join(map(str, s[:3])))
def test_fused_kernel_equals_split_path_bitwise(shape):
    # the same EMF-form sweep and the same IB sums in the same order as the
    # marching sweep + staged IB, so every field is bitwise the split path's
    nx, ny, nz, D = shape
    p = W.small_pipe(nx=nx, ny=ny, nz=nz, diameter=D, Re=300.0, Ha=40.0, Rm=1e-2, b0_kind="tanh",
                     ramp_center=nz / 2, ramp_width=2.0, force_amp=0.2, force_period=9.0, perturb=0.01, seed=13,
                     n_mag=25, precision="fp32")
    outs = []
    for k in ("fused", "split"):
        with Solver(dict(p, sweep_kernel=k)) as s:
            assert s.units["sweep_kernel"] == k
            s.step(3)
            s.mag_sweeps(7)
            outs.append(s.state())
            s.observables()  # reports a timed-out copy wait as an error
    for a, b in zip(*outs):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("name", ["ramp_pulsating", "shared_rows"])
def test_fused_kernel_parity_fp32(name):
    if name == "ramp_pulsating":
        p, steps, t0 = FP64_CASES[name]
    else:
        p, steps, t0 = W.small_pipe(nx=28, ny=27, nz=11, diameter=19.0, perturb=0.0, n_mag=60), 20, 0
    got, want, _ = run_both(dict(p, precision="fp32", sweep_kernel="fused"), steps, t0=t0)
    check_fields(got, want, "fp32", name + " fused")


def test_fused_kernel_six_magnet_field_fp32():
    # the in-plane applied field variant of the kernel (Sec. VI)
    nx, ny, D = 28, 24, 18.0
    p = W.small_pipe(nx=nx, ny=ny, nz=8, diameter=D, U0=0.05, Re=60.0, Ha=15.0, Rm=5e-3, perturb=0.0, n_mag=40,
                     b0_kind="field", b0_field=W.six_magnet_field(nx, ny, D), precision="fp32",
                     sweep_kernel="fused")
    got, want, _ = run_both(p, 30)
    check_fields(got, want, "fp32", "six magnets fused")


# ------------------------------------------------------------- API behaviour

@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_step_host_equals_device_stepping(precision):
    p = W.small_pipe(nx=20, ny=20, nz=9, diameter=14.0, precision=precision, n_mag=30)
    with Solver(p) as a, Solver(p) as b:
        rho, u, bb = a.state()
        a.step(9)
        ra, ua, ba = a.state()
        import ctypes as C
        ro, uo, bo = np.empty(a.n), np.empty(3 * a.n), np.empty(3 * a.n)
        from paper_2211_09370_gb300 import _lib
        obs = _lib.qslbm_obs()
        dp = lambda z: z.ctypes.data_as(C.POINTER(C.c_double))  # noqa: E731
        rc = b.L.qslbm_step_host(b.h, dp(rho.ravel().copy()), dp(u.ravel().copy()), dp(bb.ravel().copy()), 0, 9,
                                 dp(ro), dp(uo), dp(bo), C.byref(obs))
        assert rc == 0 and obs.step == 9
    np.testing.assert_array_equal(uo.reshape(ua.shape), ua)
    np.testing.assert_array_equal(bo.reshape(ba.shape), ba)
    np.testing.assert_array_equal(ro.reshape(ra.shape), ra)


@pytest.mark.parametrize("kernel", KERNELS)
def test_fp32_runs_are_deterministic(kernel):
    p = W.small_pipe(nx=30, ny=30, nz=10, diameter=22.0, n_mag=50, sweep_kernel=kernel)
    outs = []
    for _ in range(2):
        with Solver(p) as s:
            s.step(11)
            outs.append(s.state())
    for a, b in zip(*outs):
        np.testing.assert_array_equal(a, b)


def test_zero_steps_and_state_roundtrip():
    p = W.small_pipe(nx=16, ny=16, nz=5, diameter=10.0, precision="fp64")
    rng = np.random.default_rng(0)
    with Solver(p) as s:
        s.step(0)
        assert s.t == 0
        rho = 1 + 1e-3 * rng.standard_normal((5, 16, 16))
        u = 1e-2 * rng.standard_normal((3, 5, 16, 16))
        b = 1e-4 * rng.standard_normal((3, 5, 16, 16))
        s.set_state(rho, u, b, t=42)
        r2, u2, b2 = s.state()
        assert s.t == 42
    np.testing.assert_array_equal(u2, u)
    np.testing.assert_array_equal(b2, b)
    np.testing.assert_allclose(r2, rho, rtol=0, atol=2e-16)


def test_non_finite_state_is_reported():
    # fault injected on the host: a NaN in the uploaded velocity
    p = W.small_pipe(nx=12, ny=12, nz=4, diameter=8.0)
    with Solver(p) as s:
        rho, u, b = s.state()
        u[1, 2, 3, 4] = np.nan
        s.set_state(rho, u, b, t=0)
        with pytest.raises(QSLBMError) as e:
            s.observables()
        assert e.value.code == EUNSTABLE
        assert s.observables(allow_unstable=True)["nan_flag"] == 1


def test_kernel_selection_reported():
    with Solver(W.pipe_64x64x128(nz=16)) as s:
        assert s.units["sweep_kernel"] == "resident"
    with Solver(W.pipe_64x64x128(nz=16, sweep_kernel="planes")) as s:
        assert s.units["sweep_kernel"] == "planes"
    # 96 x 96 planes exceed the resident kernel's 8192-node plane limit: in
    # FP32 AUTO times the fused kernel and the split path and keeps the fused
    # kernel only when it is at least 2 % faster; in FP64 it takes the split path
    with Solver(W.pipe_ramp_96x96x512(nz=8)) as s:
        u = s.units
        assert u["sweep_us_fused"] > 0 and u["sweep_us_split"] > 0
        assert u["sweep_kernel"] == ("fused" if u["sweep_us_fused"] < 0.98 * u["sweep_us_split"] else "split")
    with Solver(W.pipe_ramp_96x96x512(nz=8, precision="fp64")) as s:
        assert s.units["sweep_kernel"] == "split" and s.units["sweep_us_fused"] == 0
    with pytest.raises(QSLBMError):
        Solver(W.pipe_ramp_96x96x512(nz=8, sweep_kernel="resident"))
    for bad in (dict(precision="fp64"), dict(nx=95)):  # the fused kernel: FP32, nx a multiple of 4
        with pytest.raises(QSLBMError):
            Solver(W.pipe_ramp_96x96x512(nz=8, sweep_kernel="fused", **bad))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_resident_and_plane_kernels_agree(precision):
    # the two sweep kernels evaluate the same expressions; FP32 contraction may
    # differ between them, so they are compared within the FP32 bound
    p = W.small_pipe(nx=40, ny=36, nz=12, diameter=28.0, precision=precision, n_mag=80)
    outs = []
    for k in KERNELS:
        with Solver(dict(p, sweep_kernel=k)) as s:
            s.step(6)
            outs.append(s.state())
    tol = 1e-13 if precision == "fp64" else 1e-5
    for other in outs[1:]:
        for a, b in zip(outs[0], other):
            assert rel(a, b) <= tol
