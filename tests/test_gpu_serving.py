"""Continuous-batching request loop: admission by memory, resident state,
shared launches, and results independent of the mix."""
import time

import numpy as np
import pytest

import paper_1912_03278_gb300 as pkg
import workloads
from paper_1912_03278_gb300 import binding

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.build()


REQ = [
    dict(n_traj=12, seed=11, dim=2, L=(32, 32), beta=np.array([0.40, 0.44, 0.48, 0.52]), eps=0.08,
         n_md=6, n_chains=4),
    dict(n_traj=30, seed=12, dim=3, L=(8, 8, 8), beta=0.2217, h=0.05, eps=0.1, n_md=5, n_chains=8),
    dict(n_traj=7, seed=13, dim=2, L=(20, 12), beta=0.3, h=0.1, eps=0.1, n_md=4, n_chains=3),
    dict(n_traj=20, seed=14, dim=3, L=(12, 12, 12), beta=0.2, eps=0.1, n_md=4, n_chains=2,
         flip_every=4),
    dict(n_traj=5, seed=15, dim=2, L=(8, 8), beta=0.44, eps=0.1, n_md=10, n_chains=1,
         precision=pkg.ISING_PREC_PLAIN_FP64),
    # dense couplings on the tensor cores (served by its own launches)
    dict(n_traj=6, seed=16, kind="dense", J=workloads.dense_couplings(256, seed=5), beta=0.5,
         C=0.5 * 2.2 + 0.1, h=0.05, eps=0.05, n_md=4, n_chains=130,
         precision=pkg.ISING_PREC_BF16),
]


def _run(reqs, budget=8 << 30, quantum=4):
    srv = pkg.IsingServer(budget, quantum)
    try:
        ids = [srv.submit(**r) for r in reqs]
        srv.drain(120.0)
        return [srv.poll(i) for i in ids], srv.stats()
    finally:
        srv.close()


def test_result_same_alone_and_in_the_mix():
    mixed, stats = _run(REQ)
    assert stats["completed"] == len(REQ) and stats["rejected"] == 0
    assert stats["group_launches"] >= 1
    for i, r in enumerate(REQ):
        alone, _ = _run([r])
        assert mixed[i]["state"] == 2 and alone[0]["state"] == 2
        for key in ("m", "E", "abs_m", "acceptance", "mean_dH", "mean_exp_mdH", "n_meas"):
            assert mixed[i]["obs"][key] == alone[0]["obs"][key], (i, key)


def test_result_matches_a_direct_handle():
    r = dict(REQ[0])
    n, seed = r.pop("n_traj"), r.pop("seed")
    res, _ = _run([REQ[0], REQ[1]], quantum=5)
    sim = pkg.IsingHMC(**r)
    try:
        sim.trajectories(n, seed)
        o = sim.observables()
    finally:
        sim.close()
    for key in ("m", "E", "abs_m", "acceptance"):
        assert res[0]["obs"][key] == o[key]


def test_admission_by_memory_budget():
    cfg, _ = binding.make_config(**{k: v for k, v in REQ[1].items() if k not in ("n_traj", "seed")})
    one = binding.ising_hmc_estimate_bytes(cfg)
    reqs = [dict(REQ[1], seed=100 + i) for i in range(4)]
    srv = pkg.IsingServer(int(one * 1.5), 2)   # room for one at a time
    try:
        ids = [srv.submit(**r) for r in reqs]
        peak_active = 0
        t0 = time.time()
        while time.time() - t0 < 60:
            st = srv.stats()
            peak_active = max(peak_active, st["active"])
            assert st["bytes_in_use"] <= one * 1.5
            if st["completed"] == len(reqs):
                break
            time.sleep(0.002)
        assert srv.stats()["completed"] == len(reqs)
        assert peak_active == 1
        res = [srv.poll(i) for i in ids]
        assert all(r["state"] == 2 for r in res)
        assert all(r["queue"] >= 0 for r in res)
    finally:
        srv.close()


def test_oversized_request_rejected():
    srv = pkg.IsingServer(1 << 20, 2)
    try:
        rid = srv.submit(**dict(REQ[0], L=(512, 512)))   # 16 MB of state, budget 1 MB
        srv.drain(30.0)
        r = srv.poll(rid)
        assert r["state"] == 3 and r["status"] == binding.ISING_ENOMEM
    finally:
        srv.close()
