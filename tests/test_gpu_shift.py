"""The default shift C (Sec. 2, spectrum bound and shift) is chosen inside the
library: a handle created without C reports, per chain, the bound that makes
A = beta*J*K + C*1 positive definite plus 0.1."""
import numpy as np
import pytest

import workloads
import paper_1912_03278_gb300 as pkg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.build()


def test_lattice_default_shift():
    betas = np.array([0.2, 0.3, 0.2217])
    with pkg.IsingHMC(dim=3, L=(6, 6, 6), beta=betas, Jnn=1.5, n_chains=3) as s:
        prm = s.params
        np.testing.assert_array_equal(prm[:, 0], betas)
        np.testing.assert_allclose(prm[:, 1], betas * 1.5 * 6 + 0.1, rtol=1e-15, atol=0)
        s.trajectories(1, 3)
        assert np.all(np.isfinite(s.records()[:, 0]))


def test_infinite_range_default_shift():
    N = 64
    with pkg.IsingHMC(kind="infinite", n_sites=N, beta=1.0, Jnn=1.0) as s:
        assert abs(s.params[0, 1] - (1.0 / N + 0.1)) < 1e-15
    with pkg.IsingHMC(kind="infinite", n_sites=N, beta=0.5, Jnn=-1.0) as s:
        assert abs(s.params[0, 1] - (0.5 * (N - 1) / N + 0.1)) < 1e-15


@pytest.mark.parametrize("N,prec", [(200, pkg.ISING_PREC_PLAIN_FP64), (512, pkg.ISING_PREC_BF16)])
def test_dense_default_shift_from_lanczos(N, prec):
    """No C given: the library's Lanczos estimate of lambda_min(J) sets
    C = beta |lambda_min| + 0.1 per chain (here against numpy's eigvalsh)."""
    J = workloads.dense_couplings(N, seed=1)
    lam = np.linalg.eigvalsh(J)[0]
    betas = np.array([0.5, 1.0])
    with pkg.IsingHMC(kind="dense", J=J, beta=betas, eps=0.1, n_md=4, n_chains=2,
                      precision=prec) as s:
        C = s.params[:, 1]
        np.testing.assert_allclose(C, betas * abs(lam) + 0.1, rtol=0, atol=1e-9)
        s.trajectories(1, 5)
        assert np.all(np.isfinite(s.records()[:, 0]))


def test_explicit_shift_kept_and_too_small_rejected():
    with pkg.IsingHMC(dim=2, L=(8, 8), beta=0.44, C=3.0) as s:
        assert s.params[0, 1] == 3.0
    with pytest.raises(pkg.IsingError) as ei:
        pkg.IsingHMC(dim=2, L=(8, 8), beta=0.44, C=4 * 0.44)
    assert ei.value.status == pkg.ISING_ENOTPD
