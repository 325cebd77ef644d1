"""Write the oracle fixtures the GPU parity tests compare against.

Calls only the CPU oracle (``oracle/``) and the workload definitions; nothing
here touches the CUDA library.  Usage: ``python tests/golden/make_golden.py
[name ...]``; each fixture is an ``.npz`` beside this script with a SHA-256 of
its arrays stored inside.

Fixtures
  hartmann_2000   2-D Hartmann channel 64x32 (D2Q9 + D2Q5, N_mag = 465), all
                  fields after the workload's full 2000 steps from rest.
  pipe_64x64x128  3-D pipe 64x64x128 (D3Q19 + D3Q7, N_mag = 270, seed 2211,
                  1 % noise): 4096 sampled nodes after 2 steps.
  ramp_96x96x512  3-D pipe 96x96x512 in the tanh-ramped field with the
                  pulsating body force, Rm = 1e-2 (N_mag = 270), 1 % noise
                  (seed 7), clock started at t = 500: 4096 sampled nodes after
                  1 step.
  ramp_96x96x512_rm<Rm>
                  the same pipe at the other magnetic Reynolds numbers of the
                  workload's sweep, Rm = 1e-4, 1e-3, 1e-1 (N_mag = 270, 270,
                  176: 1 step) and Rm = 1 (N_mag = 18: 3 steps).
"""
from __future__ import annotations

import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2211_09370_gb300 import workloads as W  # noqa: E402

SAMPLE = 4096


def digest(arrays: dict) -> str:
    h = hashlib.sha256()
    for k in sorted(arrays):
        h.update(k.encode())
        h.update(np.ascontiguousarray(arrays[k]).tobytes())
    return h.hexdigest()


def save(name: str, arrays: dict):
    arrays = dict(arrays)
    arrays["sha256"] = np.array(digest(arrays))
    np.savez_compressed(os.path.join(HERE, name + ".npz"), **arrays)


def sample_nodes(n: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n, size=min(SAMPLE, n), replace=False))


def run_sampled(p: dict, steps: int, t0: int, seed: int):
    o = oracle.Oracle(p)
    if t0:
        rho, u, b = o.state()
        o.set_state(rho, u, b, t=t0)
    t = time.time()
    o.step(steps)
    rho, u, b = o.state()
    idx = sample_nodes(o.n, seed)
    fields = np.concatenate([rho.reshape(1, -1), u.reshape(3, -1), b.reshape(3, -1)])[:, idx]
    print(f"  {steps} steps in {time.time() - t:.1f}s", flush=True)
    return {"idx": idx, "fields": fields, "steps": np.array(steps), "t0": np.array(t0)}


def hartmann_2000():
    p = W.hartmann_channel_2d()
    o = oracle.Oracle(p)
    o.step(p["steps"])
    rho, u, b = o.state()
    return {"rho": rho, "u": u, "b": b, "steps": np.array(p["steps"])}


def pipe_64x64x128():
    return run_sampled(W.pipe_64x64x128(precision="fp64"), steps=2, t0=0, seed=1)


def ramp_96x96x512():
    return run_sampled(W.pipe_ramp_96x96x512(Rm=1e-2, precision="fp64", perturb=0.01, seed=7), steps=1, t0=500,
                       seed=2)


# the workload's magnetic Reynolds number sweep (1e-2 is ramp_96x96x512 itself)
RAMP_RM_STEPS = {"1e-4": 1, "1e-3": 1, "1e-1": 1, "1": 3}


def ramp_96x96x512_rm(rm: str):
    return lambda: run_sampled(W.pipe_ramp_96x96x512(Rm=float(rm), precision="fp64", perturb=0.01, seed=7),
                               steps=RAMP_RM_STEPS[rm], t0=500, seed=2)


FIXTURES = {"hartmann_2000": hartmann_2000, "pipe_64x64x128": pipe_64x64x128, "ramp_96x96x512": ramp_96x96x512}
FIXTURES.update({f"ramp_96x96x512_rm{rm}": ramp_96x96x512_rm(rm) for rm in RAMP_RM_STEPS})


def load(name: str) -> dict:
    with np.load(os.path.join(HERE, name + ".npz")) as z:
        d = {k: z[k] for k in z.files}
    want = str(d.pop("sha256"))
    if digest(d) != want:
        raise ValueError(f"fixture {name} fails its checksum")
    return d


if __name__ == "__main__":
    names = sys.argv[1:] or list(FIXTURES)
    for name in names:
        print(name, flush=True)
        t = time.time()
        save(name, FIXTURES[name]())
        print(f"  wrote {name}.npz in {time.time() - t:.1f}s", flush=True)
