"""Per-trajectory series recorded on the device: the recorded values are the
ones the measurement step sums, recording changes no result, and the capacity
bounds what is kept."""
import math

import numpy as np
import pytest

import paper_1912_03278_gb300 as pkg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.build()


@pytest.mark.parametrize("kw", [
    dict(dim=2, L=(8, 8), beta=np.array([0.4, 0.44, 0.5, 0.3]), h=0.02, eps=0.1, n_md=5,
         n_chains=4, flip_every=3),
    dict(kind="infinite", n_sites=300, beta=np.array([1.0, 0.9]), eps=0.1, n_md=4, n_chains=2),
    dict(dim=2, L=(6, 6), beta=np.array([0.44, 0.3]), eps=0.1, n_md=4, n_chains=2,
         precision=pkg.ISING_PREC_PLAIN_FP64),
])
def test_series_is_what_the_sums_add_and_changes_nothing(kw):
    a = pkg.IsingHMC(**kw)
    b = pkg.IsingHMC(**kw)
    try:
        a.series_enable(50)
        a.trajectories(30, 17)
        b.trajectories(30, 17)
        ser = a.series()
        sums = a.chain_sums()
        assert ser.shape == (kw["n_chains"], 30, 3)
        for c in range(kw["n_chains"]):
            for k, col in ((2, 0), (4, 1), (6, 2)):   # ISING_SUM_M, _E, _ABSM
                assert math.isclose(sums[c, k], math.fsum(ser[c, :, col]), rel_tol=1e-12,
                                    abs_tol=1e-12), (c, k)
        assert np.array_equal(a.state(), b.state())
        assert np.array_equal(sums, b.chain_sums())
    finally:
        a.close()
        b.close()


def test_capacity_and_disable():
    sim = pkg.IsingHMC(dim=2, L=(8, 8), beta=0.4, eps=0.1, n_md=4, n_chains=3)
    try:
        sim.series_enable(5)
        sim.trajectories(8, 1)
        assert sim.series().shape == (3, 5, 3)
        sim.trajectories(2, 1)
        assert sim.series().shape == (3, 5, 3)
        sim.series_enable(0)
        assert sim.series().shape == (3, 0, 3)
    finally:
        sim.close()


def test_tau_int_of_abs_m_grows_with_the_lattice():
    """Sec. 4 (Fig. 2): tau_int of |m| at the critical coupling grows with L
    (z ~ 2); 128 chains x 600 trajectories after 100 of thermalisation."""
    beta = math.log(1 + math.sqrt(2)) / 2
    taus = []
    for L in (8, 24):
        n_md = max(1, int(math.log(L * L)))
        sim = pkg.IsingHMC(dim=2, L=(L, L), beta=beta, C=5 * beta, eps=1 / (n_md * math.sqrt(beta)),
                           n_md=n_md, n_chains=128)
        try:
            sim.trajectories(100, 3)
            sim.series_enable(600)
            sim.trajectories(600, 3)
            r = pkg.binding.ising_gamma_method(sim.series()[:, :, 2])
            taus.append(r["tau_int"])
        finally:
            sim.close()
    assert taus[1] > 2.0 * taus[0], taus
