"""GPU parity and statistics of the infinite-range (all-to-all) model of the
appendix: K_ij = 1/N for i != j, run by its own O(N) kernel (no matrix).

The oracle sees the same model as a dense coupling matrix
(workloads.infinite_range_couplings), so parity here checks the O(N) product
against the plain matrix-vector definition.  Tolerances are those of the FP32
lattice form: proposal psi 1e-5 relative, dH 1e-6 absolute against the
oracle's FP64 H on the GPU's own end points, accept decisions identical unless
within 1e-6 of the threshold.
"""
import numpy as np
import pytest

import oracle
import paper_1912_03278_gb300 as pkg
import workloads
from tests.stats_util import within
from tests.test_gpu_parity import one_trajectory_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.build()
    oracle.build()


# Variant by N (threads = min(256, quads rounded up to 32)): resident with 1,
# 2, 4 or 8 quads per thread up to N = 8192, streaming above; resident chains
# whose quads fill every thread (N = 128 m up to 4 quads per thread) run an
# instance without per-quad bounds checks.
@pytest.mark.parametrize("N", [
    1024,   # resident, 1 quad per thread, float4 quads, every thread full
    2048,   # resident, 2 quads per thread, every thread full
    4096,   # resident, 4 quads per thread, every thread full
    1001,   # resident, scalar loads, ragged last quad
    1001,   # resident, scalar loads, ragged last quad
    2000,   # resident, 2 quads per thread, ragged thread tail
    4000,   # resident, 4 quads per thread
    8190,   # resident, 8 quads per thread, scalar loads
    8193,   # streaming, scalar loads, one site in the last quad
    9000,   # streaming, float4 quads
    2,      # smallest model
    5,      # one full quad plus a single site
])
def test_one_trajectory(N):
    one_trajectory_parity(kind="infinite", n_sites=N, betas=(1.0, 0.7, 1.3), h=0.05, eps=0.1,
                          n_md=5)


def test_per_site_field_and_omelyan():
    N = 640
    h = workloads.dense_fields(N, sigma=0.2, seed=5)
    one_trajectory_parity(kind="infinite", n_sites=N, betas=(1.0, 0.9), h=h, eps=0.12, n_md=4,
                          integrator=1)


def test_antiferromagnetic_coupling():
    # J < 0: C must exceed beta*|J|*(N-1)/N
    one_trajectory_parity(kind="infinite", n_sites=300, Jnn=-1.0, betas=(0.8,), h=0.1, eps=0.1,
                          n_md=6)


def test_sign_flip_at_zero_field():
    rec = one_trajectory_parity(kind="infinite", n_sites=256, betas=(1.2, 1.0), h=0.0, eps=0.1,
                                n_md=4, flip_every=1, traj=0)
    assert np.all(rec[:, 7] == 1.0)   # S(-psi) = S(psi) at h = 0: always accepted


def test_sign_flip_with_field():
    one_trajectory_parity(kind="infinite", n_sites=255, betas=(1.2, 1.0), h=0.03, eps=0.1, n_md=4,
                          flip_every=1, traj=0)


def test_several_trajectories():
    one_trajectory_parity(kind="infinite", n_sites=512, betas=(1.0,), h=0.05, eps=0.1, n_md=4,
                          n_traj=3, traj=0)


def test_sign_flip_streaming_and_several_quads_per_thread():
    for N in (3001, 8500):
        one_trajectory_parity(kind="infinite", n_sites=N, betas=(1.1,), h=0.02, eps=0.1, n_md=3,
                              flip_every=1, traj=0, n_traj=2)


@pytest.mark.parametrize("N", [777, 3001, 8500])
def test_trajectory_split_is_bitwise_invariant(N):
    kw = dict(kind="infinite", n_sites=N, beta=np.array([1.0, 0.9]), h=0.02, eps=0.1, n_md=5,
              n_chains=2, flip_every=2)
    a = pkg.IsingHMC(**kw)
    b = pkg.IsingHMC(**kw)
    try:
        a.trajectories(5, 99)
        b.trajectories(3, 99)
        b.trajectories(2, 99)
        assert np.array_equal(a.state(), b.state())
        assert np.array_equal(a.chain_sums(), b.chain_sums())
    finally:
        a.close()
        b.close()


def test_chain_result_independent_of_batch_size():
    betas = np.array([0.9, 1.0, 1.1])
    a = pkg.IsingHMC(kind="infinite", n_sites=300, beta=betas, eps=0.1, n_md=5, n_chains=3)
    b = pkg.IsingHMC(kind="infinite", n_sites=300, beta=betas[:1], eps=0.1, n_md=5, n_chains=1)
    try:
        a.trajectories(4, 8)
        b.trajectories(4, 8)
        assert np.array_equal(a.state()[:1], b.state())
    finally:
        a.close()
        b.close()


def test_small_model_against_brute_force():
    """N = 13 (scalar path), beta = 1, h = 0.05: E, m and |m| of 512 chains
    within 3 standard errors of the exact sums over all 2^13 spin states."""
    N, beta, h, C = 13, 1.0, 0.05, 1.0
    bf = oracle.brute_force(oracle.Model(kind="dense", J=workloads.infinite_range_couplings(N), h=h,
                                         beta=beta, C=C))
    sim = pkg.IsingHMC(kind="infinite", n_sites=N, beta=beta, C=C, h=h, eps=0.25, n_md=4,
                       n_chains=512, n_therm=100)
    try:
        sim.trajectories(1100, 2)
        o = sim.observables()
        assert 0.5 < o["acceptance"] <= 1.0
        for key in ("E", "m", "abs_m"):
            assert within(o[key], bf[key], o[key + "_err"]), (key, o[key], bf[key], o[key + "_err"])
    finally:
        sim.close()


@pytest.mark.parametrize("N", [64, 400])
def test_energy_matches_appendix_exact_sum(N):
    """<beta eps> at the critical coupling beta*J = 1, h = 0, against the exact
    finite-N sum of the appendix (1024 chains, 300 measured trajectories each)."""
    beta = 1.0
    exact = oracle.infinite_range_energy(beta, 1.0, 0.0, N)
    sim = pkg.IsingHMC(kind="infinite", n_sites=N, beta=beta, C=1.0, eps=0.25, n_md=4,
                       n_chains=1024, n_therm=100)
    try:
        sim.trajectories(400, 4)
        o = sim.observables()
        assert 0.5 < o["acceptance"] <= 1.0
        assert within(o["E"], exact, o["E_err"]), (o["E"], exact, o["E_err"])
        assert within(o["m"], 0.0, o["m_err"]), (o["m"], o["m_err"])
        assert abs(o["mean_exp_mdH"] - 1.0) < 5 * o["exp_mdH_err"] + 1e-3
    finally:
        sim.close()
