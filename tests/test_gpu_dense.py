"""Dense couplings on the tensor cores: the BF16 tcgen05 GEMM behind the force."""
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


def to_bf16_bits(x):
    """Round FP32 to BF16 (nearest even) and return the 16-bit patterns."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32)
    r = (b + np.uint32(0x7FFF) + ((b >> np.uint32(16)) & np.uint32(1))) >> np.uint32(16)
    return r.astype(np.uint16)


def from_bf16_bits(b):
    return (b.astype(np.uint32) << np.uint32(16)).view(np.float32).astype(np.float64)


# 128-multiples run single-CTA 128 x 128 tiles, 256-multiples CTA-pair 256 x 256
# tiles; 4096 x 1280 has more pair tiles (80) than pairs fit on the GPU at once.
@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (256, 384, 512), (512, 256, 4096),
                                   (1024, 1024, 1024), (4096, 1280, 256)])
def test_tcgen05_bf16_gemm(M, N, K):
    g = np.random.default_rng(M + N + K)
    A = to_bf16_bits(g.standard_normal((M, K)))
    B = to_bf16_bits(g.standard_normal((N, K)))
    D = binding.ising_hmc_selftest_gemm(A, B)
    ref = from_bf16_bits(B) @ from_bf16_bits(A).T   # (N, M)
    err = np.abs(D - ref).max() / np.abs(ref).max()
    assert err < 1e-5, err   # FP32 accumulation over K terms


# ---------------------------------------------------------------- HMC with dense couplings
import oracle
import workloads
from tests.stats_util import within

BF16 = pkg.ISING_PREC_BF16


def _dense_parity(N, n_chains, samples, beta=0.5, n_md=8, eps=0.06, traj=2, seed=5, h=True,
                  psi_scale=0.4, prec=BF16, tol=2e-2, default_shift=False):
    J = workloads.dense_couplings(N, seed=1)
    hv = workloads.dense_fields(N, 0.1) if h else 0.0
    C = None if default_shift else beta * abs(np.linalg.eigvalsh(J)[0]) + 0.1
    psi0 = workloads.start_psi(n_chains, N, scale=psi_scale, seed=23).astype(np.float32).astype(np.float64)
    sim = pkg.IsingHMC(kind="dense", J=J, h=hv, beta=beta, C=C, eps=eps, n_md=n_md,
                       n_chains=n_chains, precision=prec)
    C = float(sim.params[0, 1])   # the library's choice when none was given
    try:
        sim.set_state(psi0, next_traj=traj)
        sim.trajectories(1, seed)
        rec = sim.records()
        ends = {c: (sim.chains(pkg.ISING_STATE_PSI_PROPOSAL, c, 1)[0],
                    sim.chains(pkg.ISING_STATE_P_END, c, 1)[0]) for c in samples}
        # the momenta call overwrites the stored end momenta: fetch those first
        got = {c: ends[c] + (sim.momenta(seed, traj, c, 1)[0],) for c in samples}
    finally:
        sim.close()
    model = oracle.Model(kind="dense", J=J, h=hv, beta=beta, C=C)
    for c in samples:
        prop, pend, p0 = got[c]
        ch = oracle.Chain(model, form=oracle.FORM_FP32, seed=seed, chain=c, psi0=psi0[c])
        ch.traj = traj
        r = ch.trajectory(eps, n_md)
        rel = np.abs(prop - r["psi_prop"]).max() / np.abs(r["psi_prop"]).max()
        assert rel <= tol, (c, rel)           # low-precision force
        H0 = oracle.kinetic(p0) + oracle.action(model, psi0[c])
        H1 = oracle.kinetic(pend) + oracle.action(model, prop)
        assert abs(rec[c, 0] - (H1 - H0)) <= 1e-6, (c, rec[c, 0], H1 - H0)   # FP64-accurate dH
        assert abs(rec[c, 4] - oracle.action(model, psi0[c])) <= 1e-6
        assert abs(rec[c, 1] - r["logu"]) <= 1e-14


def test_dense_bf16_parity_small_ragged_chains():
    _dense_parity(256, 130, samples=(0, 77, 129))


@pytest.mark.parametrize("prec,tol", [(BF16, 2e-2), (pkg.ISING_PREC_FP8, 0.1)])
def test_dense_parity_single_cta_tiles(prec, tol):
    """N = 384 and 100 chains are not multiples of 256: the forces and the
    action run on single-CTA 128 x 128 tiles instead of CTA pairs."""
    _dense_parity(384, 100, samples=(0, 57, 99), prec=prec, tol=tol)


@pytest.mark.parametrize("N,n_chains", [(4224, 130), (4352, 256)])
def test_dense_bf16_parity_beyond_exact_digit_range(N, n_chains):
    """N > 4096: the digit-plane product is no longer exact in the FP32
    accumulator, so the action's A psi runs on the double-float CUDA-core
    product instead; N = 4224 on single-CTA force tiles, N = 4352 on CTA pairs.
    C is the library's default shift."""
    _dense_parity(N, n_chains, samples=(0, n_chains - 1), n_md=6, eps=0.05, default_shift=True)


def test_dense_bf16_parity_config_size():
    """N = 4096 SK couplings, 1024 chains (the dense workload), sampled chains."""
    _dense_parity(4096, 1024, samples=(0, 1023), n_md=8, eps=0.05)


# FP8 E4M3 operands round to 3 mantissa bits (unit roundoff 2^-4): the force
# carries errors of a few per cent, so the proposal after a trajectory may sit
# up to ~10% (of max |psi|) from the exact one; dH is still exact to 1e-6.
FP8_TOL = 0.1


def test_dense_fp8_parity_small_ragged_chains():
    _dense_parity(256, 130, samples=(0, 77, 129), prec=pkg.ISING_PREC_FP8, tol=FP8_TOL)


def test_dense_fp8_parity_config_size():
    _dense_parity(4096, 1024, samples=(0, 1023), n_md=8, eps=0.05, prec=pkg.ISING_PREC_FP8,
                  tol=FP8_TOL)


def test_dense_bf16_statistics_small_against_brute_force():
    """N = 128 SK model is too large to enumerate; the same J distribution at
    N = 128 is checked against the plain FP64 form statistically instead."""
    N, beta = 128, 0.5
    J = workloads.dense_couplings(N, seed=3)
    hv = workloads.dense_fields(N, 0.1, seed=4)
    C = beta * abs(np.linalg.eigvalsh(J)[0]) + 0.1
    res = {}
    for prec, chains in ((BF16, 256), (pkg.ISING_PREC_PLAIN_FP64, 8)):
        sim = pkg.IsingHMC(kind="dense", J=J, h=hv, beta=beta, C=C, eps=0.1, n_md=6,
                           n_chains=chains, precision=prec, n_therm=50)
        try:
            sim.trajectories(350 if prec == BF16 else 300, 7)
            res[prec] = sim.observables()
        finally:
            sim.close()
    a, b = res[BF16], res[pkg.ISING_PREC_PLAIN_FP64]
    assert a["acceptance"] > 0.5
    for key in ("E", "m"):
        err = np.hypot(a[key + "_err"], b[key + "_err"])
        assert abs(a[key] - b[key]) <= 4 * err + 1e-3, (key, a[key], b[key], err)


def test_dense_fp8_statistics_against_plain_fp64():
    """The FP8 force only lowers the acceptance: the chain still samples the
    exact distribution (the action and dH are exact), so E and m agree with
    the plain FP64 form within the statistical errors."""
    N, beta = 128, 0.5
    J = workloads.dense_couplings(N, seed=3)
    hv = workloads.dense_fields(N, 0.1, seed=4)
    C = beta * abs(np.linalg.eigvalsh(J)[0]) + 0.1
    res = {}
    for prec, chains, eps in ((pkg.ISING_PREC_FP8, 256, 0.06), (pkg.ISING_PREC_PLAIN_FP64, 8, 0.1)):
        sim = pkg.IsingHMC(kind="dense", J=J, h=hv, beta=beta, C=C, eps=eps, n_md=6,
                           n_chains=chains, precision=prec, n_therm=50)
        try:
            sim.trajectories(350 if prec == pkg.ISING_PREC_FP8 else 300, 9)
            res[prec] = sim.observables()
        finally:
            sim.close()
    a, b = res[pkg.ISING_PREC_FP8], res[pkg.ISING_PREC_PLAIN_FP64]
    assert a["acceptance"] > 0.3
    for key in ("E", "m"):
        err = np.hypot(a[key + "_err"], b[key + "_err"])
        assert abs(a[key] - b[key]) <= 4 * err + 1e-3, (key, a[key], b[key], err)


def test_dense_forces_timing_aid_leaves_chains_untouched():
    """ising_hmc_dense_forces overwrites only working buffers: a trajectory
    after it is bitwise the trajectory without it."""
    N, B, beta = 256, 130, 0.5
    J = workloads.dense_couplings(N, seed=3)
    C = beta * abs(np.linalg.eigvalsh(J)[0]) + 0.1
    mk = lambda: binding.IsingHMC(kind="dense", J=J, beta=beta, C=C, eps=0.05, n_md=4, n_chains=B,
                                  precision=binding.ISING_PREC_BF16)
    a, b = mk(), mk()
    try:
        a.trajectories(2, 11)
        b.trajectories(2, 11)
        a.dense_forces(3)
        a.trajectories(1, 11)
        b.trajectories(1, 11)
        assert np.array_equal(a.state(), b.state())
        assert np.array_equal(a.records(), b.records())
    finally:
        a.close()
        b.close()


@pytest.mark.parametrize("prec", [BF16, pkg.ISING_PREC_FP8])
def test_dense_sign_flip_always_accepted_at_zero_field(prec):
    """Sec. 3 global flip in the tensor-core form: at h = 0, S(-psi) = S(psi),
    so every chain flips after its trajectory and the current configuration
    is exactly minus the one the Metropolis step kept."""
    N, B, beta, traj = 256, 130, 0.5, 3
    J = workloads.dense_couplings(N, seed=1)
    psi0 = workloads.start_psi(B, N, scale=0.4, seed=23).astype(np.float32).astype(np.float64)
    sim = pkg.IsingHMC(kind="dense", J=J, h=0.0, beta=beta, eps=0.05, n_md=4, n_chains=B,
                       precision=prec, flip_every=1)
    try:
        sim.set_state(psi0, next_traj=traj)
        sim.trajectories(1, 5)
        rec = sim.records()
        prop = sim.state(pkg.ISING_STATE_PSI_PROPOSAL)
        cur = sim.state(pkg.ISING_STATE_PSI)
    finally:
        sim.close()
    assert np.all(rec[:, 7] == 1.0)
    for c in range(B):
        kept = prop[c] if rec[c, 2] else psi0[c]
        assert np.array_equal(cur[c], -kept), c


def test_dense_sign_flip_samples_both_magnetisations():
    """Infinite-range couplings as a dense BF16 matrix (K_ij = 1/N) in the
    ordered phase, beta J = 1.5, with a small field h = 0.01: chains started at
    psi = 0 settle near +m or -m, and only the flip moves them between the two
    with the right weights; with flips every other trajectory <beta eps>
    matches the appendix's exact finite-N sum."""
    N, beta, h = 128, 1.5, 0.01
    J = workloads.infinite_range_couplings(N, 1.0)
    exact = oracle.infinite_range_energy(beta, 1.0, h, N)
    sim = pkg.IsingHMC(kind="dense", J=J, h=h, beta=beta, C=1.0, eps=0.15, n_md=6, n_chains=256,
                       n_therm=100, precision=BF16, flip_every=2)
    try:
        sim.trajectories(600, 3)
        o = sim.observables()
        rec = sim.records()
    finally:
        sim.close()
    assert o["acceptance"] > 0.5
    assert rec[:, 7].sum() > 0          # trajectory 599 was a flip trajectory
    assert within(o["E"], exact, o["E_err"]), (o["E"], exact, o["E_err"])
