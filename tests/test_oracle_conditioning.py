"""The FP64 parity horizons are well conditioned: a one-ulp perturbation of the
initial velocity changes the oracle's own result by less than 1e-13 there, so
the 1e-12 GPU-versus-oracle bound tests arithmetic, not the flow's sensitivity.
"""
import numpy as np
import pytest

import oracle
from tests.parity_cases import DEGENERATE, FP64_CASES, MAC_CASES, Q27_CASES, degenerate, mac_case


def _sensitivity(p, steps, t0):
    a, b = oracle.Oracle(p), oracle.Oracle(p)
    rho, u, bb = b.state()
    rng = np.random.default_rng(0)
    b.set_state(rho, u * (1 + 1e-16 * rng.standard_normal(u.shape)), bb, t=t0)
    if t0:
        a.set_state(rho, u, bb, t=t0)
    a.step(steps)
    b.step(steps)
    _, ua, ba = a.state()
    _, ub, bbb = b.state()
    rel = lambda x, y: np.linalg.norm(x - y) / max(np.linalg.norm(y), 1e-300)  # noqa: E731
    return rel(ub, ua), rel(bbb, ba)


@pytest.mark.parametrize("name", sorted(FP64_CASES))
def test_fp64_parity_horizon_is_well_conditioned(name):
    p, steps, t0 = FP64_CASES[name]
    su, sb = _sensitivity(dict(p, precision="fp64"), steps, t0)
    assert su < 1e-13 and sb < 1e-13, (su, sb)


@pytest.mark.parametrize("name", sorted(Q27_CASES))
def test_d3q27_parity_horizon_is_well_conditioned(name):
    p, steps, t0 = Q27_CASES[name]
    su, sb = _sensitivity(dict(p, precision="fp64"), steps, t0)
    assert su < 1e-13 and sb < 1e-13, (su, sb)


@pytest.mark.parametrize("name", sorted(MAC_CASES))
def test_macroscopic_parity_horizon_is_well_conditioned(name):
    p, steps = mac_case(name, precision="fp64")
    su, sb = _sensitivity(p, steps, 0)
    assert su < 1e-13 and sb < 1e-13, (su, sb)


@pytest.mark.parametrize("case", sorted(DEGENERATE))
def test_degenerate_horizon_is_well_conditioned(case):
    p, steps = degenerate(case)
    su, sb = _sensitivity(dict(p, precision="fp64"), steps, 0)
    assert su < 1e-13 and sb < 1e-13, (su, sb)


@pytest.mark.parametrize("name", ["small_pipe", "smooth_pipe_long"])
def test_viscosity_scaled_ib_horizon_is_well_conditioned(name):
    # the same cases with lambda = nu / nu_ref = 2 (Sec. V.E)
    p, steps, t0 = FP64_CASES[name]
    nu = oracle.derive(dict(p, precision="fp64"))["nu"]
    su, sb = _sensitivity(dict(p, precision="fp64", nu_ref=nu / 2.0), steps, t0)
    assert su < 1e-13 and sb < 1e-13, (su, sb)
