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


def test_energy_noalloc_matches_handle_path(torch_cuda):
    torch = torch_cuda
    L, beta, C, h0, n, seed, traj = (12, 10), 0.41, 4 * 0.41 + 0.2, 0.07, 3, 21, 4
    N = L[0] * L[1]
    for call in range(2):
        psi = workloads.start_psi(n, N, scale=0.6 + 0.3 * call, seed=40 + call)
        # existing entry point: S0 and K0 of the trajectory record of a plain FP64 handle
        sim = pkg.IsingHMC(dim=2, L=L, beta=beta, C=C, h=h0, eps=0.1, n_md=2, n_chains=n,
                           precision=pkg.ISING_PREC_PLAIN_FP64)
        try:
            sim.set_state(psi, next_traj=traj)
            sim.trajectories(1, seed)
            rec = sim.records()
            p0 = sim.momenta(seed, traj)
        finally:
            sim.close()
        dpsi = torch.tensor(psi, dtype=torch.float64, device="cuda")
        dp = torch.tensor(p0, dtype=torch.float64, device="cuda")
        out = torch.full((2 * n,), float("nan"), dtype=torch.float64, device="cuda")
        binding.ising_hmc_energy_noalloc(2, L, beta, 1.0, C, h0, n, dpsi.data_ptr(),
                                         dp.data_ptr(), out.data_ptr())
        torch.cuda.synchronize()
        res = out.cpu().numpy().reshape(n, 2)
        np.testing.assert_allclose(res[:, 0], rec[:, 4], rtol=0, atol=1e-6)   # S
        np.testing.assert_allclose(res[:, 1], rec[:, 3], rtol=0, atol=1e-6)   # K


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
