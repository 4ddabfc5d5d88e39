"""The device conjugate-gradient solve of A x = b (Sec. 2's A of one chain)
against the oracle's A and its own CG, and a closed form."""
import numpy as np
import pytest

import oracle
import paper_1912_03278_gb300 as pkg
import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.build()
    oracle.build()


@pytest.mark.parametrize("kw", [
    dict(kind="dense", J=workloads.dense_couplings(200, seed=5),
         precision=pkg.ISING_PREC_PLAIN_FP64),
    dict(dim=2, L=(8, 6)),
    dict(dim=3, L=(4, 5, 6)),
    dict(dim=1, L=(9,)),
    dict(kind="infinite", n_sites=300, Jnn=1.0),
    dict(kind="infinite", n_sites=301, Jnn=-1.0),
])
def test_solution_satisfies_the_oracles_A(kw):
    betas = np.array([0.4, 0.3])
    C = np.array([3.0, 2.5])   # above every bound here (lattice 2 d beta |J|; infinite beta |J|)
    sim = pkg.IsingHMC(beta=betas, C=C, n_chains=2, **kw)
    try:
        N = pkg.binding.load().ising_hmc_n_sites(sim.h)
        b = workloads.dense_fields(N, sigma=1.0, seed=3)
        x, it, res = sim.solve_A(b, chain=1)
    finally:
        sim.close()
    if kw.get("kind") == "infinite":
        model = oracle.Model(kind="dense", J=workloads.infinite_range_couplings(N, kw["Jnn"]),
                             beta=0.3, C=float(C[1]))
    elif kw.get("kind") == "dense":
        model = oracle.Model(kind="dense", J=kw["J"], beta=0.3, C=float(C[1]))
    else:
        model = oracle.Model(dim=kw["dim"], L=kw["L"], beta=0.3, C=float(C[1]))
    assert res <= 1e-13 and 0 < it < 10000
    Ax = oracle.apply_A(model, x)
    assert np.abs(Ax - b).max() <= 1e-11 * np.abs(b).max()
    xr, _ = oracle.cg_solve(model, b)
    np.testing.assert_allclose(x, xr, rtol=1e-9, atol=1e-11)


def test_uniform_right_hand_side_closed_form():
    """The constant vector is an eigenvector of K (2d neighbours): x = b / (C + 2d beta J)."""
    sim = pkg.IsingHMC(dim=2, L=(10, 10), beta=0.44, C=2.0, n_chains=1)
    try:
        x, it, res = sim.solve_A(np.full(100, 0.7))
    finally:
        sim.close()
    np.testing.assert_allclose(x, 0.7 / (2.0 + 4 * 0.44), rtol=1e-14)
    assert it <= 2


def test_tensor_core_dense_form_rejected():
    """The BF16 form keeps no FP64 couplings on the device: EINVAL."""
    J = workloads.dense_couplings(128, seed=1)
    sim = pkg.IsingHMC(kind="dense", J=J, beta=0.5, precision=pkg.ISING_PREC_BF16)
    try:
        with pytest.raises(pkg.IsingError) as ei:
            sim.solve_A(np.ones(128))
        assert ei.value.status == pkg.ISING_EINVAL
    finally:
        sim.close()
