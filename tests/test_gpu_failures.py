"""Failure paths, made on the host (no device wait is ever driven to its limit
and nothing faults the GPU): an injected device-allocation failure at every
allocation of a handle's creation, an error bit planted in a handle's device
error word, and a server that keeps serving after a request's allocation
failed."""
import numpy as np
import pytest

import paper_1912_03278_gb300 as pkg
from paper_1912_03278_gb300 import binding

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.build()
    yield
    binding.ising_hmc_inject_alloc_failure(0)


KW = dict(dim=3, L=(8, 8, 8), beta=0.22, h=np.full(512, 0.05), eps=0.1, n_md=4, n_chains=3)


@pytest.mark.parametrize("kw", [KW, dict(kind="dense", J=None, beta=0.5, eps=0.1, n_md=4,
                                         n_chains=2, precision=binding.ISING_PREC_BF16)])
def test_every_allocation_failure_is_reported_and_cleaned_up(kw):
    if kw.get("kind") == "dense":
        import workloads
        kw = dict(kw, J=workloads.dense_couplings(256, seed=3))
    failures = successes = 0
    for k in range(1, 40):
        binding.ising_hmc_inject_alloc_failure(k)
        try:
            sim = pkg.IsingHMC(**kw)
        except pkg.IsingError as e:
            assert e.status == binding.ISING_ENOMEM, (k, e)
            failures += 1
            continue
        finally:
            binding.ising_hmc_inject_alloc_failure(0)
        # the k-th allocation was a temporary the creation can do without (the
        # dense Lanczos vectors fall back to the host), or k is beyond the
        # creation's allocations: the handle works
        successes += 1
        try:
            sim.trajectories(2, 5)
            assert np.all(np.isfinite(sim.records()[:, 0]))
        finally:
            sim.close()
    assert failures >= 5 and successes >= 1   # every state allocation was made to fail once
    with pkg.IsingHMC(**kw) as sim:   # nothing left behind that breaks the next handle
        sim.trajectories(1, 6)
        sim.sync()


def test_device_error_word_reports_timeout_and_handle_can_be_destroyed():
    sim = pkg.IsingHMC(**KW)
    try:
        sim.trajectories(1, 3)
        sim.sync()
        binding.ising_hmc_inject_device_error(sim.h, 1)   # a bounded wait gave up
        with pytest.raises(pkg.IsingError) as ei:
            sim.sync()
        assert ei.value.status == binding.ISING_ETIMEOUT
        with pytest.raises(pkg.IsingError) as ei:
            sim.observables()
        assert ei.value.status == binding.ISING_ETIMEOUT
        with pytest.raises(pkg.IsingError) as ei:
            binding.ising_hmc_inject_device_error(sim.h, 64)
        assert ei.value.status == binding.ISING_EINVAL
    finally:
        sim.close()
    other = pkg.IsingHMC(**KW)
    try:
        binding.ising_hmc_inject_device_error(other.h, 2)   # bounds check
        with pytest.raises(pkg.IsingError) as ei:
            other.sync()
        assert ei.value.status == binding.ISING_ECUDA
    finally:
        other.close()
    with pkg.IsingHMC(**KW) as fresh:   # the context is unaffected
        fresh.trajectories(1, 4)
        fresh.sync()


def test_server_rejects_a_request_whose_allocation_fails_and_keeps_serving():
    srv = pkg.IsingServer(int(4e9), 2)
    try:
        ok0 = srv.submit(3, 11, **{k: v for k, v in KW.items() if k != "h"}, h=0.05)
        srv.wait(ok0, 60.0)
        binding.ising_hmc_inject_alloc_failure(1)
        bad = srv.submit(3, 12, **{k: v for k, v in KW.items() if k != "h"}, h=0.05)
        res = srv.wait(bad, 60.0)
        assert res["state"] == 3 and res["status"] == binding.ISING_ENOMEM, res
        binding.ising_hmc_inject_alloc_failure(0)
        ok1 = srv.submit(3, 13, **{k: v for k, v in KW.items() if k != "h"}, h=0.05)
        srv.wait(ok1, 60.0)
        st = srv.stats()
        assert st["rejected"] >= 1 and st["completed"] >= 2
    finally:
        binding.ising_hmc_inject_alloc_failure(0)
        srv.close()
