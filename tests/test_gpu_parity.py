"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.

Tolerances (the contract of this library):
  * proposal psi after one trajectory from a common start:
      plain FP64 form: ||dpsi||_inf / ||psi||_inf <= 1e-10;  FP32 form: <= 1e-5
  * dH: plain FP64 form against the fully independent oracle trajectory, and
    FP32 form against the oracle's FP64 H evaluated on the GPU's own (psi, p)
    end points: |dH_gpu - dH_oracle| <= 1e-6 absolute
  * accept decisions identical unless |dH + log u| < 1e-6
  * observables of the resulting configuration: m, E within 1e-9 (FP64) or
    1e-6 (FP32); |m| identical up to spin decisions within 1e-6 of their
    threshold.
"""
import math

import numpy as np
import pytest

import oracle
import workloads
import paper_1912_03278_gb300 as pkg
from tests.stats_util import gamma_method, within

pytestmark = pytest.mark.gpu

FP32, FP64 = pkg.ISING_PREC_FP32, pkg.ISING_PREC_PLAIN_FP64


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.build()
    oracle.build()


def _oracle_model(kind, dim, L, J, h, beta, C, Jnn=1.0):
    if kind in ("dense", "infinite"):   # infinite: J is the all-to-all matrix
        return oracle.Model(kind="dense", J=J, h=h, beta=beta, C=C)
    return oracle.Model(dim=dim, L=L, Jnn=Jnn, h=h, beta=beta, C=C)


def _count_near_ties(model, psi, form, seed, chain, traj):
    """Sites whose spin decision lies within 1e-6 of its threshold."""
    _, a, t = oracle.action(model, psi, return_at=True)
    u = oracle.spin_uniforms(form, 0 if traj == 0xFFFFFFFF else seed, chain, traj, model.N)
    return int(np.sum(np.abs(u - (1 + t) / 2) < 1e-6))


def _parity_setup(kind="lattice", dim=2, L=(8, 8), J=None, h=0.0, betas=(0.44,), C=None,
                  eps=0.1, n_md=5, prec=FP32, integrator=0, flip_every=0, traj=3, seed=11,
                  psi_scale=0.5, n_traj=1, n_sites=0, Jnn=1.0, launch=None, split=None,
                  staging=None):
    """Create a handle at a common start state; returns the context of one
    parity case (the handle and everything the oracle needs)."""
    n_chains = len(betas)
    betas = np.asarray(betas, dtype=np.float64)
    if kind == "infinite":   # the oracle sees the same model as a dense matrix
        N = n_sites
        J = workloads.infinite_range_couplings(N, Jnn)
    else:
        N = int(np.prod(L[:dim])) if kind != "dense" else J.shape[0]
    if C is None:
        if kind in ("dense", "infinite"):
            C = betas * abs(np.linalg.eigvalsh(J)[0]) + 0.1
        else:
            C = betas * 2 * dim + 0.1
    C = np.broadcast_to(np.asarray(C, dtype=np.float64), (n_chains,)).copy()
    eps_c = np.broadcast_to(np.asarray(eps, dtype=np.float64), (n_chains,)).copy()
    psi0 = workloads.start_psi(n_chains, N, scale=psi_scale, seed=17)
    if prec == FP32:
        psi0 = psi0.astype(np.float32).astype(np.float64)
    sim = pkg.IsingHMC(kind=kind, dim=dim, L=L, J=None if kind == "infinite" else J,
                       n_sites=N if kind == "infinite" else 0, Jnn=Jnn, h=h, beta=betas, C=C,
                       eps=eps_c, n_md=n_md, n_chains=n_chains, precision=prec,
                       integrator=integrator, flip_every=flip_every)
    try:
        if launch is not None:
            sim.set_launch(*launch)
            assert sim.launch == tuple(launch)
        if split is not None:
            sim.set_chain_split(split)
            assert sim.chain_split == split
        if staging is not None:
            sim.set_staging(staging)
        sim.set_state(psi0, next_traj=traj)
        for k in range(n_traj - 1):
            sim.trajectories(1, seed)
    except BaseException:
        sim.close()
        raise
    return dict(sim=sim, kind=kind, dim=dim, L=L, J=J, h=h, betas=betas, C=C, eps=eps_c,
                n_md=n_md, prec=prec, integrator=integrator, flip_every=flip_every, traj=traj,
                seed=seed, n_traj=n_traj, Jnn=Jnn, N=N, psi0=psi0, n_chains=n_chains)


def _parity_before(ctx):
    sim = ctx["sim"]
    ctx["start_last"] = sim.state(pkg.ISING_STATE_PSI)
    ctx["sums_before"] = sim.chain_sums()


def _parity_after(ctx):
    """Read the GPU's results of the last trajectory, then release the handle."""
    sim = ctx["sim"]
    try:
        ctx["rec"] = sim.records()
        ctx["prop"] = sim.state(pkg.ISING_STATE_PSI_PROPOSAL)
        ctx["cur"] = sim.state(pkg.ISING_STATE_PSI)
        ctx["pend"] = sim.state(pkg.ISING_STATE_P_END)
        ctx["sums"] = sim.chain_sums() - ctx["sums_before"]
        ctx["p0"] = sim.momenta(ctx["seed"], ctx["traj"] + ctx["n_traj"] - 1)
    finally:
        sim.close()


def _parity_check(ctx):
    """Recompute every chain's trajectories with the oracle from the same start
    and compare element by element (tolerances in the module docstring)."""
    kind, dim, L, J, h, Jnn = ctx["kind"], ctx["dim"], ctx["L"], ctx["J"], ctx["h"], ctx["Jnn"]
    betas, C, eps_c, n_md = ctx["betas"], ctx["C"], ctx["eps"], ctx["n_md"]
    prec, integrator, flip_every = ctx["prec"], ctx["integrator"], ctx["flip_every"]
    traj, seed, n_traj, N, psi0 = ctx["traj"], ctx["seed"], ctx["n_traj"], ctx["N"], ctx["psi0"]
    rec, prop, cur, pend, sums, p0 = (ctx[k] for k in ("rec", "prop", "cur", "pend", "sums", "p0"))
    start_last = ctx["start_last"]
    form = oracle.FORM_FP32 if prec == FP32 else oracle.FORM_FP64
    for c in range(ctx["n_chains"]):
        model = _oracle_model(kind, dim, L, J, h, betas[c], C[c], Jnn)
        ch = oracle.Chain(model, form=form, seed=seed, chain=c, psi0=psi0[c])
        ch.traj = traj
        for k in range(n_traj):
            r = ch.trajectory(eps_c[c], n_md, integrator=integrator, flip_every=flip_every)
        scale = max(np.abs(r["psi_prop"]).max(), 1e-30)
        rel = np.abs(prop[c] - r["psi_prop"]).max() / scale
        tol_psi = 1e-5 if prec == FP32 else 1e-10
        assert rel <= tol_psi, ("psi proposal", c, rel)
        if prec == FP64:
            assert abs(rec[c, 0] - r["dH"]) <= 1e-6, ("dH", c, rec[c, 0], r["dH"])
        else:
            H0 = oracle.kinetic(p0[c]) + oracle.action(model, start_last[c])
            H1 = oracle.kinetic(pend[c]) + oracle.action(model, prop[c])
            assert abs(rec[c, 0] - (H1 - H0)) <= 1e-6, ("dH on GPU end points", c, rec[c, 0], H1 - H0)
            assert abs(rec[c, 0] - r["dH"]) <= max(1e-3, 1e-4 * abs(r["dH"]) * 10)
        assert abs(rec[c, 1] - r["logu"]) <= 1e-14
        if abs(r["dH"] + r["logu"]) >= 1e-6:
            assert bool(rec[c, 2]) == r["accepted"], ("accept", c)
        # observables of the current configuration (measured trajectory); a
        # configuration repeated after a rejection keeps its earlier spin draw
        last = traj + n_traj - 1
        if bool(rec[c, 2]) == r["accepted"] and not flip_every and (r["accepted"] or n_traj == 1):
            o_gpu = dict(m=sums[c, 2], E=sums[c, 4], abs_m=sums[c, 6])
            if prec == FP64:
                o_ref = ch.obs
                tol = 1e-9
            else:
                o_ref = oracle.measure(model, cur[c], form, seed if r["accepted"] else 0, c,
                                       last if r["accepted"] else 0xFFFFFFFF)
                tol = 1e-6
            assert abs(o_gpu["m"] - o_ref["m"]) <= tol, ("m", c)
            assert abs(o_gpu["E"] - o_ref["E"]) <= tol, ("E", c)
            ties = _count_near_ties(model, cur[c], form, seed, c,
                                    last if r["accepted"] else 0xFFFFFFFF)
            assert abs(o_gpu["abs_m"] - o_ref["abs_m"]) <= 2.0 * ties / N + 1e-12, ("|m|", c)
    return rec


def one_trajectory_parity(**kw):
    ctx = _parity_setup(**kw)
    try:
        _parity_before(ctx)
        ctx["sim"].trajectories(1, ctx["seed"])
    except BaseException:
        ctx["sim"].close()
        raise
    _parity_after(ctx)
    return _parity_check(ctx)


# ------------------------------------------------------------------ FP32 ----
@pytest.mark.parametrize("dim,L", [
    (2, (32, 32)),      # VEC=4, several planes
    (2, (12, 20)),      # rectangular
    (2, (10, 7)),       # scalar fallback (row not a multiple of 4)
    (2, (3, 3)),        # minimum extent
    (3, (8, 8, 8)),
    (3, (12, 6, 5)),    # vector path, ragged plane count
    (3, (5, 6, 7)),     # scalar fallback
    (1, (16,)),
    (1, (17,)),
])
def test_fp32_one_trajectory(dim, L):
    one_trajectory_parity(dim=dim, L=L, betas=(0.30, 0.44, 0.21), h=0.05, eps=0.08, n_md=6)


def test_fp32_per_site_field_and_long_trajectory():
    N = 16 * 16
    h = workloads.dense_fields(N, sigma=0.2, seed=5)
    one_trajectory_parity(dim=2, L=(16, 16), betas=(0.4, 0.45), h=h, eps=0.05, n_md=20)


def test_fp32_single_step_and_large_eps():
    one_trajectory_parity(dim=2, L=(8, 12), betas=(0.5,), eps=0.3, n_md=1)


def test_fp32_omelyan():
    one_trajectory_parity(dim=2, L=(16, 16), betas=(0.44, 0.3), eps=0.15, n_md=4, integrator=1)


def test_fp32_sign_flip_at_zero_field():
    rec = one_trajectory_parity(dim=2, L=(8, 8), betas=(0.6, 0.5), h=0.0, eps=0.1, n_md=4,
                                flip_every=1, traj=0)
    assert np.all(rec[:, 7] == 1.0)  # S(-psi) = S(psi) at h = 0: always accepted


def test_fp32_sign_flip_with_field():
    one_trajectory_parity(dim=2, L=(8, 8), betas=(0.6, 0.5), h=0.02, eps=0.1, n_md=4,
                          flip_every=1, traj=0)


def test_fp32_several_trajectories():
    one_trajectory_parity(dim=3, L=(6, 6, 6), betas=(0.22,), h=0.05, eps=0.1, n_md=4, n_traj=3,
                          traj=0)


# ------------------------------------ full-size layouts of the fused kernel ----
# A thread of the fused lattice kernel owns up to 4 vectors of a plane (a
# vector = 4 sites on rows that split into float4s, else 1 site).  These cases
# reach 2, 3 and 4 vectors per thread, ragged last vectors (vectors not a
# multiple of the thread count) and explicit launch shapes below the default
# thread count, on both the float4 and the scalar path.
@pytest.mark.parametrize("dim,L,launch", [
    (3, (48, 48, 4), None),        # 576 vectors / 256 threads: 3 each, the third ragged
    (3, (32, 32, 4), (64, 1)),     # 256 / 64: 4 each
    (3, (20, 12, 5), (32, 2)),     # 60 / 32: 2 each, ragged, ring depth 2
    (2, (1022, 6), None),          # scalar path, 1022 / 256: 4 each, ragged
    (2, (1001, 8), None),          # scalar path, odd row
    (2, (256, 8), (32, 1)),        # 64 / 32: 2 each
    (2, (1024, 6), (64, 1)),       # 256 / 64: 4 each (a row of the L = 1024 workload)
    (2, (1024, 5), (96, 4)),       # 256 / 96: 3 each, ragged, ring depth 4
])
def test_fp32_multi_vector_layouts(dim, L, launch):
    one_trajectory_parity(dim=dim, L=L, betas=(0.30, 0.44), h=0.05, eps=0.08, n_md=6,
                          launch=launch)


@pytest.mark.parametrize("L", [48, 64])
def test_fp32_3d_mixed_workload_sizes(L):
    """The two largest sizes of the mixed 3D workload (h = 0.05, beta = 0.2217,
    C = 6 beta + 0.1) at the default launch shape: 3 and 4 vectors per thread."""
    one_trajectory_parity(dim=3, L=(L, L, L), betas=(0.2217, 0.2217), h=0.05, eps=0.08, n_md=6)


def test_mixed_size_group_launch_against_oracle():
    """Members of different sizes and launch shapes advanced by one group
    launch; every chain of every member is checked against the oracle."""
    cases = [
        dict(dim=3, L=(48, 48, 4), betas=(0.2217,), h=0.05),
        dict(dim=2, L=(1001, 8), betas=(0.3, 0.44), h=0.02),
        dict(dim=3, L=(6, 5, 7), betas=(0.2,), h=0.0),
        dict(dim=2, L=(32, 32), betas=(0.4,), h=0.05, launch=(32, 1)),
        dict(dim=3, L=(16, 16, 16), betas=(0.2217, 0.25), h=0.05),
        dict(dim=3, L=(32, 32, 16), betas=(0.2217,), h=0.05, split=4),
        dict(dim=3, L=(24, 24, 12), betas=(0.23, 0.21), h=0.05, split=2),
    ]
    ctxs = []
    try:
        for c in cases:
            ctxs.append(_parity_setup(eps=0.08, n_md=6, **c))
        for c in ctxs:
            _parity_before(c)
        grp = pkg.IsingGroup([c["sim"] for c in ctxs])
        try:
            grp.trajectories(1, ctxs[0]["seed"])
            grp.sync()
            assert grp.launches == 1
        finally:
            grp.close()
    except BaseException:
        for c in ctxs:
            c["sim"].close()
        raise
    for c in ctxs:
        _parity_after(c)
    for c in ctxs:
        _parity_check(c)


# ------------------------------------------- chains split over a CTA cluster ----
# With a chain split over a cluster of CTAs every CTA streams a slab of planes
# and reads the planes beyond its slab's ends from the previous pass; the
# per-chain sums are added across the cluster in rank order.
@pytest.mark.parametrize("dim,L,split,extra", [
    (3, (48, 48, 8), 2, {}),                            # slabs of 4 planes, 3 vectors per thread
    (3, (20, 12, 10), 4, {}),                           # ragged slabs: 2, 3, 2, 3 planes
    (3, (64, 64, 16), 8, {}),                           # slabs of 2 planes, 4 vectors per thread
    (2, (1024, 16), 8, {}),                             # 2D rows: slabs of 2 rows
    (2, (1001, 12), 4, {}),                             # scalar path, ragged vectors, 3-row slabs
    (3, (8, 8, 8), 4, dict(integrator=1)),              # Omelyan
    (3, (16, 16, 16), 2, dict(launch=(64, 4))),         # explicit launch shape, depth 4
])
def test_fp32_split_chains(dim, L, split, extra):
    one_trajectory_parity(dim=dim, L=L, betas=(0.30, 0.2217), h=0.05, eps=0.08, n_md=6,
                          split=split, **extra)


def test_fp32_split_with_site_fields_flip_and_several_trajectories():
    N = 16 * 12 * 10
    h = workloads.dense_fields(N, sigma=0.2, seed=9)
    one_trajectory_parity(dim=3, L=(16, 12, 10), betas=(0.25, 0.2), h=h, eps=0.08, n_md=5,
                          n_traj=3, traj=0, split=4)
    rec = one_trajectory_parity(dim=3, L=(12, 12, 8), betas=(0.5, 0.45), h=0.0, eps=0.1, n_md=4,
                                flip_every=1, traj=0, split=2)
    assert np.all(rec[:, 7] == 1.0)  # S(-psi) = S(psi) at h = 0: always accepted


@pytest.mark.parametrize("split", [2, 4, 8])
def test_split_is_bitwise_in_psi_and_close_in_sums(split):
    """psi and p are computed by the same per-site arithmetic whatever the
    split, so the chains agree bit for bit; the per-chain sums differ only in
    how sites are grouped into per-thread partial sums (double-float energies:
    ~1e-12 relative; FP32 Kahan estimator sums: ~1e-7, inside the 1e-6 the
    FP32 observables are held to)."""
    kw = dict(dim=3, L=(24, 24, 16), beta=np.array([0.2217, 0.24, 0.2]), h=0.05, eps=0.09,
              n_md=6, n_chains=3, flip_every=2)
    a = pkg.IsingHMC(**kw)
    b = pkg.IsingHMC(**kw)
    try:
        b.set_chain_split(split)
        a.trajectories(6, 21)
        b.trajectories(4, 21)
        b.trajectories(2, 21)
        assert np.array_equal(a.state(), b.state())
        assert np.array_equal(a.state(pkg.ISING_STATE_P_END), b.state(pkg.ISING_STATE_P_END))
        ra, rb = a.records(), b.records()
        assert np.array_equal(ra[:, 2], rb[:, 2])
        np.testing.assert_allclose(rb[:, [0, 3, 4, 5, 6]], ra[:, [0, 3, 4, 5, 6]], rtol=1e-11,
                                   atol=1e-7)
        np.testing.assert_allclose(b.chain_sums(), a.chain_sums(), rtol=0, atol=1e-6)
    finally:
        a.close()
        b.close()


def test_invalid_splits_rejected():
    sim = pkg.IsingHMC(dim=3, L=(8, 8, 6), beta=0.22, eps=0.1, n_md=2)
    try:
        for bad in (3, 0, 16, 4):   # 4: 6 planes give slabs below two planes
            with pytest.raises(pkg.IsingError):
                sim.set_chain_split(bad)
        sim.set_chain_split(2)
        assert sim.chain_split == 2
    finally:
        sim.close()
    ring = pkg.IsingHMC(dim=1, L=(64,), beta=0.4, eps=0.1, n_md=2)
    try:
        with pytest.raises(pkg.IsingError):
            ring.set_chain_split(2)
    finally:
        ring.close()


@pytest.mark.parametrize("kw,split", [
    (dict(dim=2, L=(64, 36), beta=np.array([0.44, 0.4]), h=0.02, eps=0.08, n_md=5,
          n_chains=2, flip_every=2), 1),
    (dict(dim=3, L=(24, 24, 16), beta=np.array([0.2217, 0.24, 0.2]), h=0.05, eps=0.09,
          n_md=6, n_chains=3, flip_every=2), 1),
    (dict(dim=3, L=(24, 24, 16), beta=np.array([0.2217, 0.24, 0.2]), h=0.05, eps=0.09,
          n_md=6, n_chains=3, flip_every=2), 2),
])
def test_staging_modes_agree_bit_for_bit(kw, split):
    """Per-thread cp.async and bulk-copy staging put the same plane values in
    the same ring slots, so every result is identical, records included; the
    bulk mode also agrees with the oracle."""
    runs = []
    for mode in (pkg.ISING_STAGING_THREADS, pkg.ISING_STAGING_BULK):
        sim = pkg.IsingHMC(**kw)
        try:
            if split > 1:
                sim.set_chain_split(split)
            sim.set_staging(mode)
            assert sim.staging == mode
            sim.trajectories(3, 9)
            sim.trajectories(2, 9)
            runs.append((sim.state(), sim.state(pkg.ISING_STATE_P_END), sim.records(),
                         sim.chain_sums()))
        finally:
            sim.close()
    for x, y in zip(runs[0], runs[1]):
        assert np.array_equal(x, y)


def test_bulk_staging_one_trajectory_parity():
    """One trajectory with bulk staging forced on a small 2D lattice against
    the oracle (psi to 1e-5, dH to 1e-6)."""
    one_trajectory_parity(dim=2, L=(32, 12), betas=(0.44, 0.3), h=0.05, eps=0.1, n_md=4,
                          staging=pkg.ISING_STAGING_BULK)


def test_invalid_staging_rejected():
    sim = pkg.IsingHMC(dim=2, L=(30, 8), beta=0.4, eps=0.1, n_md=2)   # rows of 30 sites
    try:
        with pytest.raises(pkg.IsingError):
            sim.set_staging(pkg.ISING_STAGING_BULK)
        with pytest.raises(pkg.IsingError):
            sim.set_staging(7)
        sim.set_staging(pkg.ISING_STAGING_THREADS)
        assert sim.staging == pkg.ISING_STAGING_THREADS
    finally:
        sim.close()


# ------------------------------------------------------------ plain FP64 ----
@pytest.mark.parametrize("dim,L", [(2, (4, 4)), (3, (4, 5, 3)), (1, (9,)), (2, (16, 12))])
def test_fp64_one_trajectory(dim, L):
    one_trajectory_parity(dim=dim, L=L, betas=(0.44, 0.3), h=0.1, eps=0.1, n_md=10, prec=FP64)


def test_fp64_dense_with_fields():
    N = 48
    J = workloads.dense_couplings(N, seed=1)
    h = workloads.dense_fields(N, sigma=0.1)
    one_trajectory_parity(kind="dense", J=J, h=h, betas=(0.5, 0.8), eps=0.1, n_md=8, prec=FP64)


def test_fp64_omelyan_and_flip():
    one_trajectory_parity(dim=2, L=(6, 6), betas=(0.44,), h=0.03, eps=0.2, n_md=3, prec=FP64,
                          integrator=1, flip_every=1, traj=0)


def test_fp64_small_2d_sequence_stays_in_lockstep():
    """L=4, beta=0.44, eps=0.1, N_md=10, seed 0: 40 trajectories, step by step."""
    model = oracle.Model(dim=2, L=(4, 4), beta=0.44, C=4 * 0.44 + 0.1)
    sim = pkg.IsingHMC(dim=2, L=(4, 4), beta=0.44, C=4 * 0.44 + 0.1, eps=0.1, n_md=10,
                       precision=FP64)
    ch = oracle.Chain(model, form=oracle.FORM_FP64, seed=0)
    try:
        for k in range(40):
            sim.trajectories(1, 0)
            rec = sim.records()[0]
            r = ch.trajectory(0.1, 10)
            assert abs(rec[0] - r["dH"]) <= 1e-6, k
            assert bool(rec[2]) == r["accepted"], k
        np.testing.assert_allclose(sim.state()[0], ch.psi, atol=1e-9)
    finally:
        sim.close()


# --------------------------------------------------------- invariances ----
@pytest.mark.parametrize("prec", [FP32, FP64])
def test_trajectory_split_is_bitwise_invariant(prec):
    kw = dict(dim=2, L=(12, 12), beta=np.array([0.4, 0.45]), h=0.02, eps=0.1, n_md=5, n_chains=2,
              precision=prec, flip_every=2)
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


def test_checkpoint_resume_is_exact():
    kw = dict(dim=3, L=(6, 6, 6), beta=0.22, h=0.05, eps=0.1, n_md=5, n_chains=3, precision=FP32)
    a = pkg.IsingHMC(**kw)
    b = pkg.IsingHMC(**kw)
    try:
        a.trajectories(4, 5)
        psi, sums, k = a.state(), a.chain_sums(), a.traj_index
        a.trajectories(3, 5)
        b.set_state(psi, next_traj=k)
        pkg.ising_hmc_set_sums(b.h, sums)
        b.trajectories(3, 5)
        assert np.array_equal(a.state(), b.state())
        assert np.array_equal(a.chain_sums(), b.chain_sums())
    finally:
        a.close()
        b.close()


def test_chain_result_independent_of_batch_size():
    """Chain c's trajectory depends only on (seed, c, traj), not on the batch."""
    betas = np.array([0.3, 0.35, 0.4, 0.45])
    a = pkg.IsingHMC(dim=2, L=(16, 16), beta=betas, eps=0.1, n_md=5, n_chains=4)
    b = pkg.IsingHMC(dim=2, L=(16, 16), beta=betas[:2], eps=0.1, n_md=5, n_chains=2)
    try:
        a.trajectories(3, 8)
        b.trajectories(3, 8)
        assert np.array_equal(a.state()[:2], b.state())
    finally:
        a.close()
        b.close()


# --------------------------------------------------------- statistics ----
def test_fp64_small_2d_against_brute_force():
    """L=4 periodic, beta=0.44, C=4 beta+0.1, eps=0.1, N_md=10, FP64, 1 chain,
    20000 trajectories, seed 0: within 3 sigma (Gamma method) of enumeration."""
    model = oracle.Model(dim=2, L=(4, 4), beta=0.44, C=4 * 0.44 + 0.1)
    bf = oracle.brute_force(model)
    sim = pkg.IsingHMC(dim=2, L=(4, 4), beta=0.44, C=4 * 0.44 + 0.1, eps=0.1, n_md=10,
                       precision=FP64, n_therm=200)
    try:
        series = {"E": [], "abs_m": [], "m": []}
        prev = np.zeros(10)
        sim.trajectories(200, 0)
        for k in range(20000 - 200):
            sim.trajectories(1, 0)
            if k % 1 == 0:
                s = sim.chain_sums()[0]
                d = s - prev
                prev = s
                series["m"].append(d[2])
                series["E"].append(d[4])
                series["abs_m"].append(d[6])
        for key in series:
            mean, err, _ = gamma_method(series[key])
            assert within(mean, bf[key], err), (key, mean, bf[key], err)
    finally:
        sim.close()


def test_fp32_small_2d_many_chains_against_brute_force():
    model = oracle.Model(dim=2, L=(4, 4), beta=0.44, C=4 * 0.44 + 0.1)
    bf = oracle.brute_force(model)
    sim = pkg.IsingHMC(dim=2, L=(4, 4), beta=0.44, C=4 * 0.44 + 0.1, eps=0.1, n_md=10,
                       n_chains=512, n_therm=100)
    try:
        sim.trajectories(2100, 1)
        o = sim.observables()
        for key in ("E", "abs_m", "m"):
            assert within(o[key], bf[key], o[key + "_err"]), (key, o[key], bf[key], o[key + "_err"])
        assert within(o["mean_exp_mdH"], 1.0, o["exp_mdH_err"])
    finally:
        sim.close()


def test_fp32_2d_onsager_away_from_criticality():
    from tests.stats_util import onsager_energy
    beta = 0.30
    sim = pkg.IsingHMC(dim=2, L=(64, 64), beta=beta, eps=0.12, n_md=8, n_chains=256, n_therm=100)
    try:
        sim.trajectories(400, 3)
        o = sim.observables()
        assert within(o["E"], onsager_energy(beta), o["E_err"], floor=1e-3), o
        assert o["acceptance"] > 0.5
    finally:
        sim.close()


# ------------------------------------------------ full-size sampled parity ----
def test_full_size_2d_batch_sampled_parity():
    """The benchmark's launch: 2D L=1024, 16 betas x 256 chains, N_md=20, FP32.
    Two sampled chains are recomputed by the oracle from the same start."""
    import torch
    free, _ = torch.cuda.mem_get_info()
    L, n_md, eps = 1024, 20, 0.02
    betas = np.repeat(workloads.beta_sweep(), 256)
    n_chains = len(betas)
    if free < 16 * L * L * n_chains * 1.05:
        pytest.skip("not enough device memory for the full batch")
    C = workloads.lattice_C(betas, 2)
    sim = pkg.IsingHMC(dim=2, L=(L, L), beta=betas, C=C, eps=eps, n_md=n_md, n_chains=n_chains)
    seed, samples = 2024, (0, n_chains - 1)
    try:
        sim.trajectories(1, seed)
        rec = sim.records()
        got = {c: (sim.chains(pkg.ISING_STATE_PSI_PROPOSAL, c, 1)[0],
                   sim.chains(pkg.ISING_STATE_P_END, c, 1)[0]) for c in samples}
        p0 = {c: sim.momenta(seed, 0, c, 1)[0] for c in samples}
        assert np.all(np.isfinite(rec[:, 0]))
    finally:
        sim.close()
    for c in samples:
        model = oracle.Model(dim=2, L=(L, L), beta=betas[c], C=C[c])
        ch = oracle.Chain(model, form=oracle.FORM_FP32, seed=seed, chain=c)
        r = ch.trajectory(eps, n_md)
        prop, pend = got[c]
        rel = np.abs(prop - r["psi_prop"]).max() / np.abs(r["psi_prop"]).max()
        assert rel <= 1e-5, (c, rel)
        H0 = oracle.kinetic(p0[c]) + oracle.action(model, np.zeros(L * L))
        H1 = oracle.kinetic(pend) + oracle.action(model, prop)
        assert abs(rec[c, 0] - (H1 - H0)) <= 1e-6, (c, rec[c, 0], H1 - H0)


def test_fp32_action_large_arguments():
    """Arguments 2|a + h'| beyond the table's 36 (exp(-y) branch) and near 0."""
    one_trajectory_parity(dim=2, L=(16, 16), betas=(0.4, 0.3), C=8.0, psi_scale=2.5, h=0.3,
                          eps=0.01, n_md=3)


def test_fp32_action_matches_fp64_on_random_states():
    """Set arbitrary FP32 states; S of the current configuration equals the
    oracle's FP64 action within 1e-6 (double-float evaluation)."""
    L = 64
    for scale in (0.05, 0.7, 4.0):
        psi = workloads.start_psi(3, L * L, scale=scale, seed=31).astype(np.float32).astype(np.float64)
        sim = pkg.IsingHMC(dim=2, L=(L, L), beta=np.array([0.3, 0.44, 0.6]), h=0.07, eps=0.05,
                           n_md=2, n_chains=3)
        try:
            sim.set_state(psi, next_traj=0)
            sim.trajectories(1, 3)  # S0 in the record is the action of the set state
            rec = sim.records()
        finally:
            sim.close()
        for c, beta in enumerate((0.3, 0.44, 0.6)):
            model = oracle.Model(dim=2, L=(L, L), beta=beta, h=0.07)
            assert abs(rec[c, 4] - oracle.action(model, psi[c])) <= 1e-6, (scale, c)


@pytest.mark.parametrize("dim,L,n", [(2, (64, 64), 5), (2, (5, 7), 3)])   # 3*35 floats: not 16-byte
def test_set_state_native_from_pinned_device_and_pageable_memory(dim, L, n):
    """set_state_native reads a pinned host buffer with a copy kernel (16-byte
    words), anything else with cudaMemcpyAsync; every source gives the same
    chains as set_state from FP64 host memory, bit for bit."""
    import torch
    N = int(np.prod(L))
    psi = workloads.start_psi(n, N, scale=0.7, seed=3).astype(np.float32)
    kw = dict(dim=dim, L=L, beta=np.linspace(0.3, 0.45, n), h=0.02, eps=0.1, n_md=4, n_chains=n)
    ref = pkg.IsingHMC(**kw)
    try:
        ref.set_state(psi.astype(np.float64), next_traj=7)
        ref.trajectories(3, 19)
        want, want_sums = ref.state(), ref.chain_sums()
    finally:
        ref.close()
    pinned = torch.from_numpy(psi.ravel().copy()).pin_memory()
    dev = torch.from_numpy(psi.ravel().copy()).cuda()
    page = np.ascontiguousarray(psi.ravel())
    for src in (pinned.data_ptr(), dev.data_ptr(), page.ctypes.data):
        sim = pkg.IsingHMC(**kw)
        try:
            pkg.ising_hmc_set_state_native(sim.h, src, 7)
            back = torch.empty(n * N, dtype=torch.float32).pin_memory()
            pkg.ising_hmc_get_state_native(sim.h, back.data_ptr())
            assert np.array_equal(back.numpy(), psi.ravel())
            sim.trajectories(3, 19)
            assert np.array_equal(sim.state(), want)
            assert np.array_equal(sim.chain_sums(), want_sums)
        finally:
            sim.close()
