"""The seeded synthetic workloads have the stated shapes, parameter ranges and
structure (host only; the generators hold no arithmetic of the method)."""
import math

import numpy as np

from paper_2211_09370_gb300 import workloads as W


def test_single_instance_workloads():
    h = W.hartmann_channel_2d()
    assert (h["dim"], h["nx"], h["ny"], h["geometry"], h["steps"]) == (2, 64, 32, "channel", 2000)
    assert (h["Re"], h["Ha"], h["Rm"], h["precision"], h["n_mag_cap"]) == (10.0, 10.0, 1e-2, "fp64", 0)
    p = W.pipe_64x64x128()
    assert (p["nx"], p["ny"], p["nz"], p["diameter"], p["steps"]) == (64, 64, 128, 56.0, 10000)
    assert (p["Re"], p["Ha"], p["Rm"], p["seed"], p["perturb"]) == (100.0, 20.0, 1e-3, 2211, 0.01)
    for rm in (1e-4, 1e-3, 1e-2, 1e-1, 1.0):
        r = W.pipe_ramp_96x96x512(Rm=rm)
        assert (r["nx"], r["ny"], r["nz"], r["diameter"], r["steps"]) == (96, 96, 512, 88.0, 20000)
        assert (r["Re"], r["Ha"], r["Rm"], r["b0_kind"]) == (500.0, 50.0, rm, "tanh")
        assert (r["ramp_center"], r["ramp_width"], r["force_amp"], r["force_period"]) == (256.0, 16.0, 0.2, 2000.0)


def test_batched_pipes_follow_their_recipe():
    ps = W.batched_pipes()
    assert len(ps) == 64
    D = np.array([p["diameter"] for p in ps])
    L = np.array([p["nz"] for p in ps])
    assert D.min() >= 24 and D.max() <= 80 and np.all(D == np.round(D))
    assert np.all(L >= 4 * D - 0.5) and np.all(L <= 8 * D + 0.5)
    assert all(p["nx"] == p["ny"] == int(p["diameter"]) + 8 for p in ps)
    Ha = np.array([p["Ha"] for p in ps])
    Re = np.array([p["Re"] for p in ps])
    Rm = np.array([p["Rm"] for p in ps])
    assert Ha.min() >= 0 and Ha.max() <= 100
    assert Re.min() >= 10 and Re.max() <= 1000 and Rm.min() >= 1e-4 and Rm.max() <= 1e-1
    kinds = [p["b0_kind"] for p in ps]
    assert set(kinds) == {"uniform", "tanh"} and 16 <= kinds.count("tanh") <= 48  # Bernoulli(1/2)
    for p in ps:
        if p["b0_kind"] == "tanh":
            assert p["ramp_center"] == p["nz"] / 2 and p["ramp_width"] == p["diameter"] / 4
    assert len({p["seed"] for p in ps}) == 64
    # seeded: the same list every time, another seed gives another list
    assert W.batched_pipes() == ps and W.batched_pipes(seed=5) != ps


def test_serving_requests_follow_their_recipe():
    rs = W.serving_requests()
    assert len(rs) == 256
    t = np.array([r["arrival_s"] for r in rs])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    # Poisson arrivals at 20/s: mean gap 1/20 s (256 gaps: within 4 standard errors)
    assert abs(gaps.mean() - 0.05) < 4 * 0.05 / math.sqrt(256)
    for r in rs:
        p = r["params"]
        D = int(p["diameter"])
        assert D in (16, 32, 48, 64, 96, 128)
        assert (p["nx"], p["ny"], p["nz"]) == (D + 8, D + 8, 6 * D)
        assert 0 <= p["Ha"] <= 80 and 10 <= p["Re"] <= 500 and 1e-4 <= p["Rm"] <= 1e-2
        assert r["tol"] == 1e-6
    assert {int(r["params"]["diameter"]) for r in rs} == {16, 32, 48, 64, 96, 128}
    assert W.serving_requests() == rs
