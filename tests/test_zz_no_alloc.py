"""The allocation-free energy entry point, for callers that cannot call
cudaMalloc (memory owned by an external pool or arena, allocation forbidden
after start-up, or work inside a region where an allocation would disturb the
caller's stream).  It must give the same FP64 action S(psi) and kinetic
energy as the regular handle-based path, and keep doing so on repeated calls
that reuse its fixed device scratch array.  Collected last so that a failure
here does not hide the other tests."""
import numpy as np
import pytest

import workloads
import paper_1912_03278_gb300 as pkg
from paper_1912_03278_gb300 import binding

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.build()
    return torch


@pytest.mark.parametrize("dim,L,with_p", [
    (2, (12, 10), True),
    (2, (12, 10), False),     # p = NULL: K must be exactly 0
    (3, (6, 5, 7), True),
    (1, (9,), True),
])
def test_energy_noalloc_matches_handle_path(torch_cuda, dim, L, with_p):
    """Two calls in a row (the second reuses the scratch array the first
    filled): S and K equal the handle path's S0 and K0 and the oracle's FP64
    values within 1e-6."""
    import oracle
    oracle.build()
    torch = torch_cuda
    beta, h0, n, seed, traj = 0.41, 0.07, 3, 21, 4
    C = 2 * dim * beta + 0.2
    N = int(np.prod(L))
    model = oracle.Model(dim=dim, L=L, beta=beta, C=C, h=h0)
    for call in range(2):
        psi = workloads.start_psi(n, N, scale=0.6 + 0.3 * call, seed=40 + call)
        # existing entry point: S0 and K0 of the trajectory record of a plain FP64 handle
        sim = pkg.IsingHMC(dim=dim, L=L, beta=beta, C=C, h=h0, eps=0.1, n_md=2, n_chains=n,
                           precision=pkg.ISING_PREC_PLAIN_FP64)
        try:
            sim.set_state(psi, next_traj=traj)
            sim.trajectories(1, seed)
            rec = sim.records()
            p0 = sim.momenta(seed, traj)
        finally:
            sim.close()
        dpsi = torch.tensor(psi, dtype=torch.float64, device="cuda")
        dp = torch.tensor(p0, dtype=torch.float64, device="cuda") if with_p else None
        out = torch.full((2 * n,), float("nan"), dtype=torch.float64, device="cuda")
        binding.ising_hmc_energy_noalloc(dim, L, beta, 1.0, C, h0, n, dpsi.data_ptr(),
                                         dp.data_ptr() if with_p else 0, out.data_ptr())
        torch.cuda.synchronize()
        res = out.cpu().numpy().reshape(n, 2)
        np.testing.assert_allclose(res[:, 0], rec[:, 4], rtol=0, atol=1e-6)   # S
        for c in range(n):
            assert abs(res[c, 0] - oracle.action(model, psi[c])) <= 1e-6
        if with_p:
            np.testing.assert_allclose(res[:, 1], rec[:, 3], rtol=0, atol=1e-6)   # K
            for c in range(n):
                assert abs(res[c, 1] - oracle.kinetic(p0[c])) <= 1e-6
        else:
            assert np.all(res[:, 1] == 0.0)


def test_energy_noalloc_rejects_too_many_chains(torch_cuda):
    torch = torch_cuda
    n = binding.ISING_NOALLOC_MAX_CHAINS + 1
    d = torch.zeros(n * 16, dtype=torch.float64, device="cuda")
    out = torch.zeros(2 * n, dtype=torch.float64, device="cuda")
    with pytest.raises(binding.IsingError) as ei:
        binding.ising_hmc_energy_noalloc(2, (4, 4), 0.4, 1.0, 2.0, 0.0, n, d.data_ptr(), 0,
                                         out.data_ptr())
    assert ei.value.status == binding.ISING_EINVAL
    assert "n_chains" in str(ei.value)
