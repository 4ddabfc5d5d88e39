"""GPU checkerboard Metropolis-Hastings (the Sec. 4 comparator) against the
oracle's checkerboard form: spins and per-chain sums bit for bit (integer
spins and sums; every acceptance decision is taken in FP32 from the same
uniform and the same FP32-rounded probability on both sides), statistics
against exact enumeration."""
import math

import numpy as np
import pytest

import oracle
import paper_1912_03278_gb300 as pkg
from tests.stats_util import within

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.build()
    oracle.build()


def _oracle_chains(dim, L, betas, h, seed, n, n_therm, spins=None, sweep0=0):
    out_s, out_sums = [], []
    for c, b in enumerate(betas):
        model = oracle.Model(dim=dim, L=L, beta=float(b), h=h, C=2 * dim * float(b) + 0.1)
        s, sums = oracle.mh_checkerboard(model, seed=seed, chain=c, n=n, n_therm=n_therm,
                                         spins=None if spins is None else spins[c], sweep0=sweep0)
        out_s.append(s)
        out_sums.append(sums)
    return np.array(out_s), np.array(out_sums)


@pytest.mark.parametrize("dim,L,h", [
    (2, (32, 6), 0.02),     # rows a multiple of 32: 32 spins per word (multi-spin coding)
    (2, (64, 10), 0.0),
    (3, (32, 4, 6), 0.02),
    (3, (64, 8, 4), 0.03),
    (1, (64,), 0.1),
    (2, (16, 16), 0.0),     # rows a multiple of 8: one 8-byte word per thread
    (2, (24, 6), 0.03),
    (3, (8, 4, 6), 0.02),
    (1, (32,), 0.1),
    (2, (6, 10), 0.05),     # byte path: groups that cross rows
    (3, (4, 6, 8), 0.02),
    (1, (10,), 0.1),        # byte path, ragged last group
])
def test_sweeps_match_oracle_bitwise(dim, L, h):
    betas = np.array([0.3, 0.44, 0.6])
    sim = pkg.IsingMH(dim=dim, L=L, beta=betas, h=h, n_chains=3, n_therm=2)
    try:
        sim.sweeps(5, 21)
        s_gpu, sums_gpu = sim.spins(), sim.chain_sums()
    finally:
        sim.close()
    s_ref, sums_ref = _oracle_chains(dim, L, betas, h, 21, 5, 2)
    assert np.array_equal(s_gpu, s_ref)
    assert np.array_equal(sums_gpu, sums_ref)


@pytest.mark.parametrize("L", [(12, 8), (32, 8)])   # byte form, packed form
def test_split_and_resume_are_bitwise(L):
    kw = dict(dim=2, L=L, beta=np.array([0.4, 0.5]), h=0.01, n_chains=2, n_therm=1)
    a, b = pkg.IsingMH(**kw), pkg.IsingMH(**kw)
    try:
        a.sweeps(7, 3)
        b.sweeps(3, 3)
        mid = b.spins()
        b.sweeps(4, 3)
        assert np.array_equal(a.spins(), b.spins())
        assert np.array_equal(a.chain_sums(), b.chain_sums())
        # resume from stored spins at sweep 3
        c = pkg.IsingMH(**kw)
        c.set_spins(mid, next_sweep=3)
        c.sweeps(4, 3)
        assert np.array_equal(c.spins(), a.spins())
        c.close()
    finally:
        a.close()
        b.close()


def test_full_size_lattice_sampled_chains():
    """L = 1024, 64 chains, 2 sweeps (the benchmark's launch shape): chains 0 and 63
    against the oracle bit for bit."""
    betas = np.linspace(0.38, 0.5, 64)
    sim = pkg.IsingMH(dim=2, L=(1024, 1024), beta=betas, n_chains=64)
    try:
        sim.sweeps(2, 7)
        s = sim.spins()
        sums = sim.chain_sums()
    finally:
        sim.close()
    for c in (0, 63):
        model = oracle.Model(dim=2, L=(1024, 1024), beta=float(betas[c]), C=4 * betas[c] + 0.1)
        ref, rsums = oracle.mh_checkerboard(model, seed=7, chain=c, n=2)
        assert np.array_equal(s[c], ref), c
        assert np.array_equal(sums[c], rsums), c


def test_small_lattice_against_brute_force():
    """2D 4x4 at beta = 0.44, h = 0.05: 512 chains x 2000 measured sweeps; m, |m|, E
    within 3 standard errors of exact enumeration."""
    model = oracle.Model(dim=2, L=(4, 4), beta=0.44, h=0.05)
    bf = oracle.brute_force(model)
    sim = pkg.IsingMH(dim=2, L=(4, 4), beta=0.44, h=0.05, n_chains=512, n_therm=200)
    try:
        sim.sweeps(2200, 5)
        o = sim.observables()
    finally:
        sim.close()
    for key in ("m", "abs_m", "E"):
        assert within(o[key], bf[key], o[key + "_err"]), (key, o[key], bf[key], o[key + "_err"])
    assert 0.0 < o["acceptance"] < 1.0
