"""Seeded synthetic workloads (parameters only, no arithmetic of the method).

The five workloads follow the paper's problem statement (grid, Re, Ha, Rm,
applied field, pipe geometry, body force) at the sizes the benchmark and the
parity tests use.  Both the CUDA library and the CPU oracle receive these
dictionaries; each side maps them to lattice units on its own.

Keys: dim, nx, ny, nz, geometry ('channel' | 'pipe'), diameter, center,
marker_spacing, Re, Ha, Rm, U0 (0 = automatic), b0_kind ('uniform' | 'tanh' |
'field'), b0_dir, ramp_center, ramp_width, b0_field ([3][ny][nx] for 'field'), force_amp, force_period, n_mag (0 = automatic),
n_mag_cap (0 = no cap), nu_ref, eta_ref, precision ('fp32' | 'fp64'), seed,
perturb, steps (horizon of the workload), flow_q (3-D flow lattice: 0 or 19 for
D3Q19, 27 for the paper's D3Q27), flow_scheme ('single_step' | 'macroscopic',
the tau >= 1 scheme).
"""
from __future__ import annotations

import math
import random

import numpy as np

NAN2 = (float("nan"), float("nan"))


def _base(**kw):
    p = dict(dim=3, geometry="pipe", center=NAN2, marker_spacing=1.0, U0=0.0, b0_kind="uniform",
             b0_dir=(1.0, 0.0, 0.0), ramp_center=0.0, ramp_width=1.0, force_amp=0.0, force_period=0.0,
             n_mag=0, n_mag_cap=270, nu_ref=0.0, eta_ref=0.0, precision="fp32", seed=0, perturb=0.0,
             strict_qs=0, flow_q=0, flow_scheme="single_step")
    p.update(kw)
    return p


def hartmann_channel_2d(**kw):
    """2-D Hartmann channel: D2Q9 + D2Q5, 64x32, walls on nodes y = 0 and 31,
    transverse uniform field, Re = 10, Ha = 10, Rm = 1e-2, from rest, 2000 steps,
    FP64, N_mag uncapped (465)."""
    p = _base(dim=2, nx=64, ny=32, nz=1, geometry="channel", diameter=31.0, Re=10.0, Ha=10.0, Rm=1e-2,
              b0_dir=(0.0, 1.0, 0.0), n_mag_cap=0, precision="fp64", steps=2000)
    p.update(kw)
    return p


def pipe_64x64x128(**kw):
    """3-D circular pipe, D3Q19 + D3Q7, 64x64x128, D = 56 along z, uniform B0
    along x, Re = 100, Ha = 20, Rm = 1e-3, N_mag = 270 (capped), seed 2211, 1 %
    velocity perturbation, 10k steps, FP32."""
    p = _base(nx=64, ny=64, nz=128, diameter=56.0, Re=100.0, Ha=20.0, Rm=1e-3, seed=2211, perturb=0.01,
              steps=10000)
    p.update(kw)
    return p


def pipe_ramp_96x96x512(Rm=1e-2, **kw):
    """3-D pipe in a tanh-ramped transverse field: 96x96x512, D = 88,
    B0_x(z) = 0.5 B_max (1 + tanh((z - 256)/16)), Ha_max = 50, Re = 500, Rm in
    {1e-4 .. 1}, body force modulated by (1 + 0.2 sin(2 pi t / 2000)), 20k steps."""
    p = _base(nx=96, ny=96, nz=512, diameter=88.0, Re=500.0, Ha=50.0, Rm=Rm, b0_kind="tanh",
              ramp_center=256.0, ramp_width=16.0, force_amp=0.2, force_period=2000.0, steps=20000)
    p.update(kw)
    return p


RAMP_RM_SWEEP = (1e-4, 1e-3, 1e-2, 1e-1, 1.0)


def small_pipe(nx=20, ny=20, nz=12, diameter=14.0, **kw):
    """A small pipe with the 64x64x128 workload's dimensionless numbers, sized
    so that the oracle finishes many steps in seconds; several CUDA tiles and a
    ragged tail."""
    p = _base(nx=nx, ny=ny, nz=nz, diameter=diameter, Re=100.0, Ha=20.0, Rm=1e-3, seed=2211, perturb=0.01,
              steps=50)
    p.update(kw)
    return p


def batched_pipes(n=64, seed=4, **kw):
    """Independent pipes of uneven size: D ~ U[24, 80] (rounded), L ~ U[4D, 8D]
    (rounded), box (D + 8)^2 x L, Ha ~ U[0, 100], Re log-uniform [10, 1000],
    Rm log-uniform [1e-4, 1e-1], field uniform or tanh ramp (centre L/2, width
    D/4) with probability 1/2 each."""
    rng = random.Random(seed)
    out = []
    for i in range(n):
        D = round(rng.uniform(24, 80))
        L = round(rng.uniform(4 * D, 8 * D))
        Ha = rng.uniform(0, 100)
        Re = 10 ** rng.uniform(1, 3)
        Rm = 10 ** rng.uniform(-4, -1)
        ramp = rng.random() < 0.5
        p = _base(nx=D + 8, ny=D + 8, nz=L, diameter=float(D), Re=Re, Ha=Ha, Rm=Rm,
                  b0_kind="tanh" if ramp else "uniform", ramp_center=L / 2.0, ramp_width=D / 4.0,
                  seed=seed * 1000 + i, perturb=0.01, steps=1000)
        p.update(kw)
        out.append(p)
    return out


def serving_requests(n=256, seed=5, rate=20.0, **kw):
    """Poisson arrivals (mean ``rate`` per second) of steady-state pipe solves:
    D in {16, 32, 48, 64, 96, 128}, box (D + 8)^2 x 6D, Ha ~ U[0, 80],
    Re ~ U[10, 500], Rm log-uniform [1e-4, 1e-2], stop at residual 1e-6."""
    rng = random.Random(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += rng.expovariate(rate)
        D = rng.choice((16, 32, 48, 64, 96, 128))
        p = _base(nx=D + 8, ny=D + 8, nz=6 * D, diameter=float(D), Re=rng.uniform(10, 500),
                  Ha=rng.uniform(0, 80), Rm=10 ** rng.uniform(-4, -2), seed=seed * 1000 + i, perturb=0.0)
        p.update(kw)
        out.append({"arrival_s": t, "params": p, "tol": 1e-6})
    return out


def nodes(p: dict) -> int:
    return int(p["nx"]) * int(p["ny"]) * (int(p.get("nz", 1)) if int(p.get("dim", 3)) == 3 else 1)


def isclose(a, b):
    return math.isclose(a, b, rel_tol=1e-12)


def six_magnet_field(nx, ny, diameter, center=None, gap=2.0, half_width=None):
    """Applied field of six slab magnets with alternating poles on a hexagon
    around the pipe (the non-uniform-field configuration of Sec. VI), as an
    in-plane array [3][ny][nx] (the z component of the pipe frame is zero).

    Each magnet's field in its own frame (y' along its face, z' from its face
    toward the pipe axis) is the Biot-Savart field of a slab of half width L:
    B_y' = 2 [atan((y' - L)/z') - atan((y' + L)/z')],
    B_z' = log(((y' + L)^2 + z'^2) / ((y' - L)^2 + z'^2)), L = R/6.  The faces
    sit at R + gap from the axis at angles k pi/3; pole signs alternate; the sum
    is scaled to max |B| = 1 inside the pipe.  Outside the pipe z' is kept
    >= 1/2 (those nodes are computed but not physical)."""
    R = 0.5 * float(diameter)
    if center is None:
        center = ((nx - 1) / 2.0, (ny - 1) / 2.0)
    L = R / 6.0 if half_width is None else float(half_width)
    y, x = np.meshgrid(np.arange(ny, dtype=float), np.arange(nx, dtype=float), indexing="ij")
    B = magnet_ring_at(x - center[0], y - center[1], R, gap, L)
    inside = (x - center[0]) ** 2 + (y - center[1]) ** 2 <= R * R
    scale = np.sqrt(B[0] ** 2 + B[1] ** 2)[inside].max()
    return np.stack([B[0] / scale, B[1] / scale, np.zeros_like(x)])


def magnet_ring_at(X, Y, R, gap, L):
    """Unscaled field (B_x, B_y) of the six-magnet ring at offsets (X, Y) from
    the pipe axis (see six_magnet_field)."""
    X = np.asarray(X, dtype=float)
    Y = np.asarray(Y, dtype=float)
    Bx = np.zeros_like(X)
    By = np.zeros_like(X)
    for k in range(6):
        th = k * math.pi / 3.0
        nxk, nyk = math.cos(th), math.sin(th)  # outward normal of magnet k
        txk, tyk = -nyk, nxk                    # along its face
        zp = np.maximum((R + gap) - (X * nxk + Y * nyk), 0.5)
        yp = X * txk + Y * tyk
        b_t = 2.0 * (np.arctan((yp - L) / zp) - np.arctan((yp + L) / zp))
        b_n = np.log(((yp + L) ** 2 + zp ** 2) / ((yp - L) ** 2 + zp ** 2))
        sgn = -1.0 if k % 2 else 1.0
        # z' points inward, along -normal
        Bx += sgn * (b_t * txk - b_n * nxk)
        By += sgn * (b_t * tyk - b_n * nyk)
    return Bx, By
