"""Serving with continuous batching: results equal to solving each request
alone, admission under a device-memory budget, requests joining mid-flight."""
import numpy as np
import pytest

from paper_2211_09370_gb300 import workloads as W
from paper_2211_09370_gb300._lib import EBUDGET, ETIMEOUT, OK, Server, Solver

pytestmark = pytest.mark.gpu

GB = 1 << 30


def requests():
    return [
        W.small_pipe(nx=20, ny=20, nz=16, diameter=14.0, Re=20.0, Ha=30.0, Rm=1e-3, perturb=0.0,
                     init_kind="poiseuille", seed=1),
        W.small_pipe(nx=26, ny=26, nz=12, diameter=18.0, Re=50.0, Ha=40.0, Rm=1e-2, perturb=0.0,
                     init_kind="poiseuille", seed=2),
        W.small_pipe(nx=16, ny=18, nz=20, diameter=10.0, Re=10.0, Ha=20.0, Rm=1e-4, perturb=0.0,
                     init_kind="poiseuille", seed=3),
        W.small_pipe(nx=22, ny=22, nz=8, diameter=16.0, Re=30.0, Ha=35.0, Rm=3e-3, b0_dir=(0.6, 0.8, 0.0),
                     perturb=0.0, init_kind="poiseuille", seed=4),
    ]


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / nb if nb > 0 else np.linalg.norm(a)


def serve(reqs, tol, chunk, budget=8 * GB, max_running=0, late=()):
    with Server(budget, chunk_steps=chunk, max_running=max_running) as S:
        ids = [S.submit(p, tol=tol, max_steps=4000, keep_fields=True) for p in reqs]
        results, rounds = {}, 0
        late = list(late)
        while len(results) < len(reqs) + len(late) or rounds == 0:
            S.run()
            rounds += 1
            if rounds == 2:
                ids += [S.submit(p, tol=tol, max_steps=4000, keep_fields=True) for p in late]
            for r in S.poll():
                results[r["id"]] = r
            assert rounds < 500
        fields = {i: S.fields(i) for i in ids}
        stats = S.stats()
    return ids, results, fields, stats


def test_served_results_equal_alone_runs():
    reqs = requests()
    ids, res, fields, stats = serve(reqs[:3], tol=1e-4, chunk=25, late=reqs[3:])
    assert stats["rebuilds"] >= 2  # requests joined and left while others ran
    assert sum(res[i]["status"] == OK for i in ids) >= 3
    for i, p in zip(ids, reqs):
        r = res[i]
        assert r["status"] in (OK, ETIMEOUT), r
        if r["status"] == OK:
            assert r["obs"]["steady_residual"] < 1e-4
        with Solver(dict(p, sweep_kernel="split")) as s:
            s.step(r["steps"])
            want = s.state()
        for a, b in zip(fields[i], want):
            assert rel(a, b) <= 1e-6


def test_budget_admission_and_caps():
    reqs = requests()[:3]
    with Server(2 * GB, chunk_steps=20, max_running=1) as S:
        big = W.pipe_64x64x128(nz=8192)  # about 2.7 GB of FP32 state: above a 2 GB budget
        a = S.submit(big, tol=1e-6)
        b = S.submit(reqs[0], tol=1e-30, max_steps=40)  # cannot converge: hits the cap
        c = S.submit(reqs[1], tol=1e-30, max_steps=40)
        seen = {}
        for _ in range(20):
            nr, npd = S.run()
            assert nr <= 1
            for r in S.poll():
                seen[r["id"]] = r
            if len(seen) == 3:
                break
    assert seen[a]["status"] == EBUDGET
    assert seen[b]["status"] == ETIMEOUT and seen[b]["steps"] == 40
    assert seen[c]["status"] == ETIMEOUT and seen[c]["t_admit"] >= seen[b]["t_done"] - 1e-9
