"""Batched stepping (many pipes in fused launches) against single-instance runs
and the oracle."""
import numpy as np
import pytest

import oracle
from paper_2211_09370_gb300 import workloads as W
from paper_2211_09370_gb300._lib import Batch, Solver

pytestmark = pytest.mark.gpu


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / nb if nb > 0 else np.linalg.norm(a)


def uneven(precision, n=5):
    # different sizes, fields, N_mag (270 down to 9) and forcing
    ps = [
        W.small_pipe(nx=26, ny=24, nz=9, diameter=18.0, precision=precision, seed=1),
        W.small_pipe(nx=17, ny=19, nz=13, diameter=12.0, Re=30.0, Ha=8.0, Rm=0.05, precision=precision, seed=2),
        W.small_pipe(nx=30, ny=30, nz=6, diameter=22.0, Re=300.0, Ha=40.0, Rm=1e-2, b0_kind="tanh",
                     ramp_center=3.0, ramp_width=1.5, precision=precision, seed=3),
        W.small_pipe(nx=21, ny=23, nz=11, diameter=15.0, Re=50.0, Ha=0.0, Rm=0.2, force_amp=0.2,
                     force_period=7.0, precision=precision, seed=4),
        W.small_pipe(nx=20, ny=20, nz=7, diameter=14.0, Rm=1.0, n_mag=9, precision=precision, seed=5),
        # the six-magnet in-plane applied field (Sec. VI)
        W.small_pipe(nx=22, ny=22, nz=6, diameter=16.0, Ha=12.0, Rm=5e-3, n_mag=30, b0_kind="field",
                     b0_field=W.six_magnet_field(22, 22, 16.0), precision=precision, seed=6),
        # the paper's D3Q27 flow lattice (Sec. III.A, Table I)
        W.small_pipe(nx=24, ny=20, nz=8, diameter=15.0, Ha=15.0, Rm=2e-2, n_mag=40, flow_q=27,
                     precision=precision, seed=7),
        # the macroscopic scheme for tau >= 1 (Sec. V.G)
        W.small_pipe(nx=20, ny=22, nz=7, diameter=15.0, Re=1.0, Ha=5.0, Rm=5e-2, n_mag=50,
                     flow_scheme="macroscopic", precision=precision, seed=8),
    ]
    return ps[:n]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_members_match_single_instances(precision):
    ps = uneven(precision, n=8)
    steps = 6
    with Batch(ps) as B:
        info = B.info()
        assert info["count"] == len(ps) and info["max_n_mag"] == 270
        assert info["sweep_threads"] in (128, 256, 512)
        B.step(steps)
        got = [B.member(i).state() for i in range(len(ps))]
    for i, p in enumerate(ps):
        with Solver(dict(p, sweep_kernel="split")) as s:
            s.step(steps)
            want = s.state()
        for a, b in zip(got[i], want):
            assert rel(a, b) <= (1e-13 if precision == "fp64" else 1e-6), i


def test_batch_member_matches_oracle_fp64():
    ps = uneven("fp64", 3)
    with Batch(ps) as B:
        B.step(4)
        m = B.member(1)
        _, u, b = m.state()
        obs = m.observables()
    o = oracle.Oracle(ps[1])
    o.step(4)
    _, ou, ob = o.state()
    assert rel(u, ou) <= 1e-12 and rel(b, ob) <= 1e-12
    assert obs["step"] == 4


@pytest.mark.parametrize("k", [6, 7])  # D3Q27; the macroscopic scheme
def test_batch_variant_member_matches_oracle_fp64(k):
    ps = uneven("fp64", 8)
    with Batch([ps[0], ps[k]]) as B:
        B.step(4)
        rho, u, b = B.member(1).state()
    o = oracle.Oracle(ps[k])
    o.step(4)
    orho, ou, ob = o.state()
    assert rel(u, ou) <= 1e-12 and rel(b, ob) <= 1e-12
    assert np.abs(rho - orho).max() <= 1e-12


def test_batch_steps_in_chunks_equal_one_call():
    ps = uneven("fp32", 4)
    with Batch(ps) as A, Batch(ps) as B:
        A.step(5)
        for _ in range(5):
            B.step(1)
        for i in range(len(ps)):
            for a, b in zip(A.member(i).state(), B.member(i).state()):
                np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batched_workload_member_matches_oracle(precision):
    # a real member of the 64-pipe batched workload (seed 4): its smallest
    # pipe (D = 27, 35 x 35 x 126, tanh-ramped field, N_mag = 270) stepped in
    # a batch with the next smallest, against the oracle on every node
    ps = W.batched_pipes(precision=precision)
    order = sorted(range(len(ps)), key=lambda k: W.nodes(ps[k]))
    a, b = ps[order[0]], ps[order[1]]
    steps = 2
    with Batch([b, a]) as B:
        B.step(steps)
        rho, u, bb = B.member(1).state()
    o = oracle.Oracle(dict(a, precision="fp64"))
    o.step(steps)
    orho, ou, ob = o.state()
    tol = 1e-12 if precision == "fp64" else 1e-4
    assert rel(u, ou) <= tol and rel(bb, ob) <= tol, (rel(u, ou), rel(bb, ob))
    if precision == "fp64":
        assert np.abs(rho - orho).max() <= 1e-12


def grouped(precision="fp32"):
    # more planes than the device has CTA slots (217 against 152 SMs), so that
    # the group kernel splits them: 2-plane groups of the two 24 x 24 x 96
    # pipes, 1-plane groups of the 40 x 40 x 20 pipe, two unequal groups (2 and
    # 1 planes, each the other's both neighbours) of a 3-plane pipe, and one
    # group of every plane (2 planes)
    return [
        W.small_pipe(nx=24, ny=24, nz=96, diameter=16.0, Re=200.0, Ha=30.0, Rm=1e-3, precision=precision, seed=11),
        W.small_pipe(nx=24, ny=24, nz=96, diameter=18.0, Re=60.0, Ha=10.0, Rm=2e-3, b0_kind="tanh",
                     ramp_center=48.0, ramp_width=8.0, precision=precision, seed=16),
        W.small_pipe(nx=40, ny=40, nz=20, diameter=32.0, Re=80.0, Ha=50.0, Rm=5e-3, b0_kind="tanh",
                     ramp_center=10.0, ramp_width=4.0, precision=precision, seed=12),
        W.small_pipe(nx=24, ny=24, nz=3, diameter=18.0, Re=40.0, Ha=10.0, Rm=2e-2, n_mag=60, precision=precision,
                     seed=13),
        W.small_pipe(nx=20, ny=20, nz=2, diameter=14.0, n_mag=33, precision=precision, seed=14),
    ]


def test_resident_groups_match_single_instances():
    import torch

    ps = grouped()
    steps = 5
    with Batch(ps) as B:
        info = B.info()
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        assert info["resident_instances"] == len(ps)
        assert len(ps) < info["resident_groups"] <= sms
        assert info["launches_per_step"] == 4  # groups, force, flow, parity advance
        assert info["graph_steps"] > 1
        B.step(steps)
        got = [B.member(i).state() for i in range(len(ps))]
    for i, p in enumerate(ps):
        with Solver(dict(p, sweep_kernel="split")) as s:
            s.step(steps)
            want = s.state()
        for a, b in zip(got[i], want):
            assert rel(a, b) <= 1e-6, i


def test_resident_groups_and_marching_in_one_batch():
    # the same instances, half of them kept on the marching sweep, and one too
    # large for a group (a 96 x 96 plane): every member as when the batch holds
    # only its own kind
    ps = grouped()
    ps = [dict(p, sweep_kernel="split") if k % 2 else p for k, p in enumerate(ps)]
    big = W.small_pipe(nx=96, ny=96, nz=4, diameter=88.0, Re=500.0, Ha=50.0, Rm=1e-2, n_mag=40, seed=15)
    steps = 4
    with Batch(ps + [big]) as B:
        info = B.info()
        assert info["resident_instances"] == 3
        B.step(steps)
        mixed = [B.member(i).state() for i in range(len(ps) + 1)]
    for i, p in enumerate(ps + [big]):
        with Batch([p]) as A:
            A.step(steps)
            alone = A.member(0).state()
        for a, b in zip(mixed[i], alone):
            np.testing.assert_array_equal(a, b)


def test_resident_groups_chunked_steps_equal_single_steps():
    ps = grouped()[:2]
    with Batch(ps) as A, Batch(ps) as B:
        n = A.info()["graph_steps"] + 3  # one chunk graph and three single steps
        A.step(n)
        for _ in range(n):
            B.step(1)
        for i in range(len(ps)):
            for a, b in zip(A.member(i).state(), B.member(i).state()):
                np.testing.assert_array_equal(a, b)


def test_resident_groups_variants_match_single_instances():
    # the sweep variants the group kernel runs through the sweep weights: the
    # accelerated sweep (Sec. V.H), the time-resolved update (Sec. III.D, one
    # sweep per step), a single plane (both z neighbours are the plane itself),
    # and the six-magnet in-plane field split over several groups
    ps = [
        W.small_pipe(nx=24, ny=24, nz=40, diameter=16.0, Re=100.0, Ha=20.0, Rm=1e-3, alpha=0.75, n_mag=60, seed=31),
        W.small_pipe(nx=24, ny=22, nz=10, diameter=16.0, U0=0.05, Re=50.0, Ha=10.0, Rm=4.0, b0_kind="tanh",
                     ramp_center=5.0, ramp_width=2.0, perturb=0.0, mag_scheme=1, seed=32),
        W.small_pipe(nx=20, ny=20, nz=1, diameter=14.0, Re=40.0, Ha=10.0, Rm=1e-2, n_mag=30, seed=33),
        W.small_pipe(nx=40, ny=40, nz=12, diameter=30.0, Ha=12.0, Rm=5e-3, n_mag=40, b0_kind="field",
                     b0_field=W.six_magnet_field(40, 40, 30.0), seed=34),
    ]
    steps = 6
    with Batch(ps) as B:
        info = B.info()
        assert info["resident_instances"] == len(ps)
        B.step(steps)
        got = [B.member(i).state() for i in range(len(ps))]
    for i, p in enumerate(ps):
        with Solver(dict(p, sweep_kernel="split")) as s:
            s.step(steps)
            want = s.state()
        for a, b in zip(got[i], want):
            assert rel(a, b) <= 1e-6, i


def test_batch_two_phase_ib_member_matches_oracle_fp64():
    # a pipe whose ring (1131 markers per plane, D = 360) and shell are too
    # large for the staged corrector's shared memory in FP64, so the batch
    # corrects b after each sweep with the two-phase form (one thread per
    # marker, then one per shell node; two launches per sweep); the same pipe
    # alone takes the single-instance two-phase form
    big = W.small_pipe(nx=368, ny=368, nz=2, diameter=360.0, n_mag=4, precision="fp64", seed=21)
    small = W.small_pipe(nx=20, ny=20, nz=7, diameter=14.0, n_mag=4, precision="fp64", seed=22)
    steps = 2
    with Batch([small, big]) as B:
        info = B.info()
        # force, flow and parity advance, then per sweep the marching launch
        # and the two IB launches
        assert info["launches_per_step"] == 3 + 4 * 3, info["launches_per_step"]
        B.step(steps)
        rho, u, b = B.member(1).state()
    with Solver(big) as s:
        assert s.units["n_markers"] == 2 * 1131
        s.step(steps)
        want = s.state()
    for a, w in zip((rho, u, b), want):
        assert rel(a, w) <= 1e-13
    o = oracle.Oracle(big)
    o.step(steps)
    orho, ou, ob = o.state()
    assert rel(u, ou) <= 1e-12 and rel(b, ob) <= 1e-12, (rel(u, ou), rel(b, ob))
    assert np.abs(rho - orho).max() <= 1e-12
