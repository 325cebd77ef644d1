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


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-4)])
def test_served_result_matches_oracle(precision, tol):
    # a request served in a mix, stopped by its step cap after 3 flow steps,
    # against the oracle at the same step
    import oracle

    # (the oracle starts from rest with the seeded perturbation)
    reqs = [dict(p, init_kind="rest", perturb=0.01) for p in requests()]
    with Server(8 * GB, chunk_steps=3, precision=precision) as S:
        ids = [S.submit(dict(p, precision=precision), tol=1e-30, max_steps=3, keep_fields=True) for p in reqs[:3]]
        res = {}
        for _ in range(5):
            S.run()
            for r in S.poll():
                res[r["id"]] = r
            if len(res) == len(ids):
                break
        rho, u, b = S.fields(ids[2])
    assert all(r["status"] == ETIMEOUT and r["steps"] == 3 for r in res.values())
    o = oracle.Oracle(dict(reqs[2], precision="fp64"))
    o.step(3)
    orho, ou, ob = o.state()
    assert rel(u, ou) <= tol and rel(b, ob) <= tol, (rel(u, ou), rel(b, ob))


def test_smallest_first_admission():
    reqs = requests()
    big = W.small_pipe(nx=40, ny=40, nz=40, diameter=30.0, perturb=0.0, init_kind="poiseuille", seed=9)
    with Server(8 * GB, chunk_steps=5, max_running=1, admit="smallest") as S:
        a = S.submit(big, tol=1e-30, max_steps=5)
        b = S.submit(reqs[2], tol=1e-30, max_steps=5)  # 16 x 18 x 20: the smallest
        seen = {}
        for _ in range(10):
            S.run()
            for r in S.poll():
                seen[r["id"]] = r
            if len(seen) == 2:
                break
    assert seen[b]["t_done"] <= seen[a]["t_admit"] + 1e-9


def test_smallest_first_keeps_the_running_set_in_the_group_kernel():
    # 24 x 24 x 96 pipes take 12 groups each at the largest group size, so at
    # most floor(SMs / 12) of them run at once; the rest wait their turn
    import torch

    sms = torch.cuda.get_device_properties(0).multi_processor_count
    p = W.small_pipe(nx=24, ny=24, nz=96, diameter=16.0, Re=50.0, Ha=10.0, Rm=1e-3, perturb=0.0,
                     init_kind="poiseuille", seed=21)
    n = sms // 12 + 3
    with Server(8 * GB, chunk_steps=10, admit="smallest") as S:
        ids = [S.submit(dict(p, seed=21 + k), tol=1e-30, max_steps=20) for k in range(n)]
        most, seen = 0, {}
        for _ in range(20):
            nr, _ = S.run()
            most = max(most, nr)
            for r in S.poll():
                seen[r["id"]] = r
            if len(seen) == n:
                break
    assert most == sms // 12
    assert all(seen[i]["status"] == ETIMEOUT and seen[i]["steps"] == 20 for i in ids)
