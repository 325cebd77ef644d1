"""Parity cases shared by the GPU parity tests and the CPU conditioning check.

Every FP64 case uses a horizon at which the oracle itself reproduces its own
result to better than 1e-13 when its initial velocity is perturbed by one unit
in the last place: the 1 % random start at tau close to 1/2 amplifies such
perturbations about a thousandfold over the first tens of steps before viscosity
damps them (measured with the oracle), so a longer horizon on a noisy start
would test the conditioning of the flow rather than the arithmetic.
"""
from paper_2211_09370_gb300 import workloads as W

# name -> (params, steps, t0)
FP64_CASES = {
    "small_pipe": (W.small_pipe(nx=29, ny=27, nz=11, diameter=19.0), 4, 0),
    "ramp_pulsating": (W.small_pipe(nx=24, ny=22, nz=40, diameter=16.0, Re=500.0, Ha=50.0, Rm=0.1,
                                    b0_kind="tanh", ramp_center=20.0, ramp_width=4.0, force_amp=0.2,
                                    force_period=50.0, perturb=0.01, seed=9), 3, 13),
    "channel_odd": (W.hartmann_channel_2d(nx=37, ny=20, diameter=19.0, n_mag=60, perturb=0.02, seed=3), 10, 0),
    "smooth_pipe_long": (W.small_pipe(nx=23, ny=21, nz=9, diameter=15.0, perturb=0.0, n_mag=60), 150, 0),
}

# the paper's own D3Q27 flow lattice (Sec. III.A, Table I): the 3-D cases above on it
Q27_CASES = {k: (dict(p, flow_q=27), steps, t0) for k, (p, steps, t0) in FP64_CASES.items() if p["dim"] == 3}

# the macroscopic scheme for tau >= 1 (Sec. V.G): tau = 1 at c = 6 nu, rho and
# rho u from the neighbours' equilibria; Re = 1 puts 6 nu well above one
MAC_CASES = {
    "pipe": (dict(nx=29, ny=27, nz=11, diameter=19.0, Re=1.0, Ha=5.0, Rm=1e-2, perturb=0.01, seed=21), 20),
    "ramp_pulsating_d3q27": (dict(nx=24, ny=22, nz=12, diameter=16.0, Re=0.8, Ha=6.0, Rm=2e-2, b0_kind="tanh",
                                  ramp_center=6.0, ramp_width=2.0, force_amp=0.2, force_period=30.0,
                                  perturb=0.01, seed=22, flow_q=27), 20),
}


def mac_case(name, **kw):
    params, steps = MAC_CASES[name]
    return W.small_pipe(flow_scheme="macroscopic", **params, **kw), steps


DEGENERATE = {
    "periodic": dict(geometry="none"),
    "single_plane": dict(nz=1),
    "two_planes": dict(nz=2),
    "strict_qs": dict(strict_qs=1),
    "no_field": dict(Ha=0.0),
    "one_sweep": dict(n_mag=1),
}


def degenerate(case):
    base = dict(nx=13, ny=11, nz=7, diameter=8.0, perturb=0.05, seed=11, n_mag=20)
    base.update(DEGENERATE[case])
    return W.small_pipe(**base), 4
