"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: each checks a closed form, an
identity, a brute-force enumeration, or a published known-answer vector, and
each is chosen so that a plausible mistake (dropped term, wrong sign, wrong
index, wrong step coefficient) fails at least one of them.  The planted-
mistake tests at the end show that for five such mistakes.
"""
import math

import numpy as np
import pytest
from scipy import stats

import oracle
import workloads
from tests.stats_util import BETA_C_2D, gamma_method, onsager_energy, within

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


# ---------------------------------------------------------------- Philox ----
# Known-answer vectors of Philox4x32-10 published with Salmon et al. (SC'11),
# the Random123 distribution's kat_vectors file: (counter, key) -> output.
PHILOX_KAT = [
    ((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
    ((0xFFFFFFFF,) * 4, (0xFFFFFFFF,) * 2, (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
    ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
     (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
]


@pytest.mark.parametrize("ctr,key,expect", PHILOX_KAT)
def test_philox_known_answers(ctr, key, expect):
    assert tuple(int(v) for v in oracle.philox(ctr, key)) == expect


def test_uniform_maps_exact_and_open():
    for x in (0, 1, 511, 512, 0xFFFFFFFF, 0x80000000):
        u = oracle.u23(x)
        assert 0.0 < u < 1.0
        assert float(np.float32(u)) == u  # exactly representable in FP32
    assert oracle.u23(0) == 2.0 ** -24
    assert oracle.u23(0xFFFFFFFF) == 1.0 - 2.0 ** -24
    assert oracle.u52(0, 0) == 2.0 ** -53
    assert oracle.u52(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 2.0 ** -53


@pytest.mark.parametrize("form", [oracle.FORM_FP64, oracle.FORM_FP32])
def test_momenta_are_standard_normal(form):
    N = 200_003  # ragged: not a multiple of 2 or 4
    p = oracle.momenta(form, seed=12345, chain=7, traj=3, N=N)
    assert abs(p.mean()) < 5 / math.sqrt(N)
    assert abs(p.var() - 1.0) < 5 * math.sqrt(2.0 / N)
    assert stats.kstest(p, "norm").pvalue > 1e-4
    # different counters give independent draws
    q = oracle.momenta(form, seed=12345, chain=8, traj=3, N=N)
    assert abs(np.corrcoef(p, q)[0, 1]) < 5 / math.sqrt(N)


def test_spin_uniforms_chi2():
    u = oracle.spin_uniforms(oracle.FORM_FP32, 9, 1, 2, 100_000)
    counts, _ = np.histogram(u, bins=50, range=(0, 1))
    assert stats.chisquare(counts).pvalue > 1e-4


# ------------------------------------------------------------ the model ----
@pytest.mark.parametrize("dim,L", [(1, (7,)), (2, (6, 5)), (3, (4, 5, 3))])
def test_apply_A_plane_wave_eigenvalues(dim, L):
    """On a periodic lattice cos(k.r) is an eigenvector of K with eigenvalue
    2 sum_d cos k_d, so A cos(k.r) = (C + 2 beta J sum_d cos k_d) cos(k.r)."""
    beta, J, C = 0.37, 1.3, 2.9
    model = oracle.Model(dim=dim, L=L, Jnn=J, beta=beta, C=C)
    coords = np.stack(np.meshgrid(*[np.arange(n) for n in L], indexing="ij"), -1)
    coords = coords.transpose(*range(dim - 1, -1, -1), dim).reshape(-1, dim)  # x fastest
    g = workloads.rng(5)
    for _ in range(4):
        n = np.array([g.integers(0, Ld) for Ld in L])
        k = 2 * np.pi * n / np.array(L)
        x = np.cos(coords @ k + 0.3)
        lam = C + 2 * beta * J * np.cos(k).sum()
        np.testing.assert_allclose(oracle.apply_A(model, x), lam * x, atol=1e-12)


def test_neighbor_lists_are_symmetric_and_distinct():
    model = oracle.Model(dim=3, L=(3, 4, 5))
    nbr = oracle.neighbors(model)
    for i in range(model.N):
        assert len(set(nbr[i])) == 6
        for j in nbr[i]:
            assert i in nbr[j]


def test_apply_A_dense_matches_matrix_product():
    N = 37
    J = workloads.dense_couplings(N, seed=4)
    h = workloads.dense_fields(N)
    model = oracle.Model(kind="dense", J=J, h=h, beta=0.7, C=2.1)
    x = workloads.rng(6).standard_normal(N)
    np.testing.assert_allclose(oracle.apply_A(model, x), 0.7 * J @ x + 2.1 * x, atol=1e-13)


def _models():
    N = 23
    J = workloads.dense_couplings(N, seed=8)
    h = workloads.dense_fields(N, sigma=0.3)
    return [
        oracle.Model(dim=2, L=(5, 4), beta=0.44, h=0.13),
        oracle.Model(dim=3, L=(3, 4, 3), beta=0.22, h=0.05),
        oracle.Model(dim=1, L=(9,), beta=0.8, h=-0.2),
        oracle.Model(kind="dense", J=J, h=h, beta=0.5),
    ]


@pytest.mark.parametrize("model", _models(), ids=["2d", "3d", "1d", "dense"])
def test_force_is_minus_gradient_of_action(model):
    psi = workloads.rng(11).standard_normal(model.N) * 0.7
    F = oracle.force(model, psi)
    step = 1e-5
    for i in range(0, model.N, max(1, model.N // 7)):
        e = np.zeros(model.N)
        e[i] = step
        fd = (oracle.action(model, psi + e) - oracle.action(model, psi - e)) / (2 * step)
        assert abs(-fd - F[i]) < 1e-7 * max(1.0, abs(F[i]))


def test_action_special_values():
    """S(0) = -N log 2cosh(h'); at h = 0, S(-psi) = S(psi)."""
    m = oracle.Model(dim=2, L=(4, 5), beta=0.4, h=0.3)
    assert abs(oracle.action(m, np.zeros(m.N)) + m.N * math.log(2 * math.cosh(0.4 * 0.3))) < 1e-12
    m0 = m.with_(h=0.0)
    psi = workloads.rng(1).standard_normal(m.N)
    assert abs(oracle.action(m0, psi) - oracle.action(m0, -psi)) < 1e-12


def test_action_large_argument_no_overflow():
    m = oracle.Model(dim=2, L=(3, 3), beta=0.5, C=50.0)
    psi = np.full(m.N, 40.0)
    S = oracle.action(m, psi)
    a = 50.0 * 40.0 + 0.5 * 4 * 40.0
    assert abs(S - m.N * (0.5 * 40.0 * a - a)) < 1e-9 * abs(S)


# ------------------------------------------------------ the integrators ----
@pytest.mark.parametrize("integ", ["leapfrog", "omelyan"])
def test_integrator_reversible(integ):
    m = oracle.Model(dim=2, L=(6, 6), beta=0.44, h=0.1)
    g = workloads.rng(3)
    psi0 = g.standard_normal(m.N) * 0.5
    p0 = g.standard_normal(m.N)
    f = oracle.leapfrog if integ == "leapfrog" else oracle.omelyan
    psi1, p1 = f(m, psi0, p0, 0.1, 10)
    psi2, p2 = f(m, psi1, -p1, 0.1, 10)
    assert np.abs(psi2 - psi0).max() < 1e-12
    assert np.abs(p2 + p0).max() < 1e-12


@pytest.mark.parametrize("integ", ["leapfrog", "omelyan"])
def test_energy_violation_scales_as_eps_squared(integ):
    """Second-order integrators: |dH| ~ eps^2 at fixed trajectory length."""
    m = oracle.Model(dim=2, L=(8, 8), beta=0.44, h=0.05)
    g = workloads.rng(4)
    psi0 = g.standard_normal(m.N) * 0.5
    p0 = g.standard_normal(m.N)
    f = oracle.leapfrog if integ == "leapfrog" else oracle.omelyan
    H0 = oracle.hamiltonian(m, psi0, p0)
    dH = []
    for n in (20, 40, 80):
        psi, p = f(m, psi0, p0, 1.0 / n, n)
        dH.append(abs(oracle.hamiltonian(m, psi, p) - H0))
    r1, r2 = dH[0] / dH[1], dH[1] / dH[2]
    assert 3.5 < r1 < 4.5 and 3.7 < r2 < 4.3, dH


def _omelyan_error_coefficients(lam, eps):
    """Leading error terms of one Omelyan step, read off the oracle's integrator.

    With a field h = 500 (h' = beta h = 100) the tanh in the force is exactly
    1 in FP64, so F = A(1 - psi) is linear, and on the uniform mode of a ring
    with C + 2 beta J = 1 the dynamics is a unit harmonic oscillator,
    q = psi - 1.
    The one-step map M (2x2, symplectic) is exp(eps J S) with S the quadratic
    form of the integrator's modified Hamiltonian
      H~ = p^2/2 + q^2/2 + eps^2 (a p^2 + b q^2) + O(eps^4),
    where a and b are the coefficients of the two nested Poisson brackets
    {T,{T,V}} = p^2 and {V,{V,T}} = q^2 (T = p^2/2, V = q^2/2).  Omelyan,
    Mryglod and Folk define the minimum-norm scheme as the lambda that
    minimises a^2 + b^2 (the norm of the eps^3 error of one step)."""
    m = oracle.Model(dim=1, L=(4,), Jnn=1.0, beta=0.2, C=0.6, h=500.0)
    cols = []
    for q0, p0 in ((1.0, 0.0), (0.0, 1.0)):
        psi, p = oracle.omelyan(m, np.ones(4) + q0, np.full(4, p0), eps, 1, lam)
        assert np.ptp(psi) == 0.0 and np.ptp(p) == 0.0   # stays on the uniform mode
        cols.append((psi[0] - 1.0, p[0]))
    M = np.array(cols).T
    assert abs(np.linalg.det(M) - 1.0) < 1e-13           # symplectic
    c = 0.5 * np.trace(M)
    s = math.sqrt(1.0 - c * c)
    K = (M - c * np.eye(2)) / s                           # M = cos(th) 1 + sin(th) K, K^2 = -1
    S = -(math.atan2(s, c) / eps) * np.array([[0.0, 1.0], [-1.0, 0.0]]) @ K
    assert abs(S[0, 1]) < 1e-8                            # time-reversible: no q p term
    return (S[1, 1] - 1.0) / (2 * eps ** 2), (S[0, 0] - 1.0) / (2 * eps ** 2)


def test_omelyan_lambda_is_the_minimum_norm_value():
    """The lambda of the oracle's Omelyan scheme (and of its HMC trajectory)
    is the one that minimises the norm of the scheme's leading error terms,
    measured on the oracle's own integrator, not typed in."""
    eps = 0.01
    lams = np.linspace(0.10, 0.30, 9)
    ab = np.array([_omelyan_error_coefficients(l, eps) for l in lams])
    # the eps^2 terms are polynomials in lambda of degree <= 2 (a product of
    # three exponentials with coefficients linear in lambda); fit, then minimise
    pa = np.polyfit(lams, ab[:, 0], 2)
    pb = np.polyfit(lams, ab[:, 1], 2)
    assert np.abs(np.polyval(pa, lams) - ab[:, 0]).max() < 1e-5
    assert np.abs(np.polyval(pb, lams) - ab[:, 1]).max() < 1e-5
    grid = np.linspace(0.10, 0.30, 200_001)
    norm = np.polyval(pa, grid) ** 2 + np.polyval(pb, grid) ** 2
    lam_star = grid[np.argmin(norm)]
    lam_oracle = oracle.omelyan.__defaults__[0]
    assert abs(lam_star - lam_oracle) < 2e-4, (lam_star, lam_oracle)
    # at lambda* the norm is well below that of neighbouring choices
    n_star = np.min(norm)
    for other in (0.15, 1.0 / 6.0, 0.25):
        assert np.polyval(pa, other) ** 2 + np.polyval(pb, other) ** 2 > 1.3 * n_star
    # the HMC trajectory's Omelyan path uses that same lambda
    model = oracle.Model(dim=2, L=(6, 6), beta=0.44, h=0.05)
    psi0 = workloads.rng(21).standard_normal(model.N) * 0.5
    ch = oracle.Chain(model, form=oracle.FORM_FP64, seed=4, chain=2, psi0=psi0)
    ch.traj = 5
    r = ch.trajectory(0.1, 6, integrator=1)
    p0 = oracle.momenta(oracle.FORM_FP64, 4, 2, 5, model.N)
    want, _ = oracle.omelyan(model, psi0, p0, 0.1, 6, lam_oracle)
    assert np.abs(r["psi_prop"] - want).max() < 1e-13
    off, _ = oracle.omelyan(model, psi0, p0, 0.1, 6, lam_oracle + 1e-3)
    assert np.abs(r["psi_prop"] - off).max() > 1e-6


def test_leapfrog_single_step_by_hand():
    """One step, n_md = 1: p += e/2 F(psi); psi += e p; p += e/2 F(psi')."""
    m = oracle.Model(dim=2, L=(3, 4), beta=0.3, h=0.2)
    g = workloads.rng(9)
    psi = g.standard_normal(m.N)
    p = g.standard_normal(m.N)
    eps = 0.37
    ph = p + 0.5 * eps * oracle.force(m, psi)
    psi1 = psi + eps * ph
    p1 = ph + 0.5 * eps * oracle.force(m, psi1)
    a, b = oracle.leapfrog(m, psi, p, eps, 1)
    np.testing.assert_allclose(a, psi1, atol=1e-14)
    np.testing.assert_allclose(b, p1, atol=1e-14)


# ------------------------------------------------------- exact results ----
def test_brute_force_ring_matches_transfer_matrix():
    N, J, h, beta = 12, 1.0, 0.15, 0.6
    m = oracle.Model(dim=1, L=(N,), Jnn=J, beta=beta, h=h)
    bf = oracle.brute_force(m)
    assert abs(bf["logZ"] - oracle.ring_logZ(beta, J, h, N)) < 1e-11
    d = 1e-5
    E = -beta * (oracle.ring_logZ(beta + d, J, h, N) - oracle.ring_logZ(beta - d, J, h, N)) / (
        2 * d) / N
    mag = (oracle.ring_logZ(beta, J, h + d, N) - oracle.ring_logZ(beta, J, h - d, N)) / (
        2 * d) / (beta * N)
    assert abs(bf["E"] - E) < 1e-8
    assert abs(bf["m"] - mag) < 1e-8


def test_brute_force_free_spins():
    N = 10
    h = workloads.dense_fields(N, sigma=0.5, seed=3)
    m = oracle.Model(kind="dense", J=np.zeros((N, N)), h=h, beta=0.9, C=0.5)
    bf = oracle.brute_force(m)
    assert abs(bf["m"] - np.tanh(0.9 * h).mean()) < 1e-13
    assert abs(bf["E"] + (0.9 * h * np.tanh(0.9 * h)).mean()) < 1e-13


@pytest.mark.parametrize("N,J", [(7, 1.0), (12, -0.5)])
def test_infinite_range_spectrum(N, J):
    """K = (11^T - 1)/N: eigenvalues -1/N (N-1 times) and (N-1)/N, the bounds the
    library's positive-definiteness check for the all-to-all model uses."""
    lam = np.linalg.eigvalsh(workloads.infinite_range_couplings(N, J))
    expect = np.sort(np.r_[np.full(N - 1, -J / N), J * (N - 1) / N])
    np.testing.assert_allclose(lam, expect, atol=1e-12)


def test_infinite_range_matches_brute_force():
    N = 12
    for beta, h in ((1.0, 0.0), (0.7, 0.2), (1.5, -0.1)):
        m = oracle.Model(kind="dense", J=workloads.infinite_range_couplings(N), h=h, beta=beta)
        assert abs(oracle.infinite_range_energy(beta, 1.0, h, N) - oracle.brute_force(m)["E"]) < 1e-12


def test_onsager_closed_form():
    """beta_c = ln(1+sqrt 2)/2 and u(beta_c) = -sqrt(2) J (Onsager 1944)."""
    assert abs(BETA_C_2D - 0.44068679350977) < 1e-12
    b = BETA_C_2D * (1 + 1e-7)  # k = 1 exactly at beta_c; approach the limit
    assert abs(onsager_energy(b) / b + math.sqrt(2)) < 1e-4
    # the leading term of the finite-size form quoted with Fig. 1 is this limit
    lead = -math.log(1 + math.sqrt(2)) * (math.sqrt(2) / 2)
    assert abs(lead - onsager_energy(b)) < 1e-4


# ------------------------------------------------ HMC against exact sums ----
def _hmc_stats(model, n, eps, n_md, form=oracle.FORM_FP64, seed=0, n_therm=500, flip_every=0,
               integrator=0):
    c = oracle.Chain(model, form=form, seed=seed)
    series = {k: [] for k in ("E", "abs_m", "m", "expmdH")}
    acc = 0
    for k in range(n):
        r = c.trajectory(eps, n_md, integrator=integrator, measure=k >= n_therm,
                         flip_every=flip_every)
        if k >= n_therm:
            o = c.obs
            series["E"].append(o["E"])
            series["abs_m"].append(o["abs_m"])
            series["m"].append(o["m"])
            series["expmdH"].append(math.exp(-r["dH"]))
            acc += r["accepted"]
    out = {k: gamma_method(v) for k, v in series.items()}
    out["acceptance"] = acc / (n - n_therm)
    return out


@pytest.mark.slow
def test_hmc_small_2d_matches_brute_force():
    """L=4 periodic square lattice at beta=0.44 (N=16; 2^16 states), eps=0.1, N_md=10."""
    model = oracle.Model(dim=2, L=(4, 4), beta=0.44, C=4 * 0.44 + 0.1)
    bf = oracle.brute_force(model)
    st = _hmc_stats(model, 20000, 0.1, 10)
    for key in ("E", "abs_m", "m"):
        mean, err, _ = st[key]
        assert within(mean, bf[key], err), (key, mean, bf[key], err)
    mean, err, _ = st["expmdH"]
    assert within(mean, 1.0, err)  # Creutz: <exp(-dH)> = 1


@pytest.mark.slow
def test_hmc_dense_sk_with_fields_matches_brute_force():
    N = 10
    J = workloads.dense_couplings(N, seed=21)
    h = workloads.dense_fields(N, sigma=0.3, seed=22)
    model = oracle.Model(kind="dense", J=J, h=h, beta=0.8)
    bf = oracle.brute_force(model)
    st = _hmc_stats(model, 12000, 0.25, 4)
    for key in ("E", "abs_m", "m"):
        mean, err, _ = st[key]
        assert within(mean, bf[key], err), (key, mean, bf[key], err)


@pytest.mark.slow
def test_hmc_infinite_range_matches_appendix():
    N = 16
    beta = 1.0
    model = oracle.Model(kind="dense", J=workloads.infinite_range_couplings(N), beta=beta)
    exact = oracle.infinite_range_energy(beta, 1.0, 0.0, N)
    st = _hmc_stats(model, 12000, 1.0 / 2, 2)
    mean, err, _ = st["E"]
    assert within(mean, exact, err), (mean, exact, err)


def test_hmc_free_spins_closed_form():
    """K = 0: <m> = mean tanh(beta h_i), <beta eps> = -mean beta h_i tanh(beta h_i)."""
    N = 8
    h = workloads.dense_fields(N, sigma=0.6, seed=5)
    model = oracle.Model(kind="dense", J=np.zeros((N, N)), h=h, beta=1.0, C=1.0)
    st = _hmc_stats(model, 6000, 0.3, 4)
    mean, err, _ = st["m"]
    assert within(mean, np.tanh(h).mean(), err)
    mean, err, _ = st["E"]
    assert within(mean, -(h * np.tanh(h)).mean(), err)


@pytest.mark.slow
def test_hmc_with_sign_flip_and_field():
    model = oracle.Model(dim=2, L=(4, 4), beta=0.6, h=0.02)
    bf = oracle.brute_force(model)
    st = _hmc_stats(model, 12000, 0.1, 10, flip_every=5)
    for key in ("E", "m"):
        mean, err, _ = st[key]
        assert within(mean, bf[key], err), (key, mean, bf[key], err)


@pytest.mark.slow
def test_hmc_fp32_form_draws_and_omelyan_match_brute_force():
    model = oracle.Model(dim=2, L=(3, 4), beta=0.5, h=0.1)
    bf = oracle.brute_force(model)
    st = _hmc_stats(model, 10000, 0.2, 5, form=oracle.FORM_FP32, integrator=1)
    for key in ("E", "abs_m", "m"):
        mean, err, _ = st[key]
        assert within(mean, bf[key], err), (key, mean, bf[key], err)


@pytest.mark.slow
def test_observables_independent_of_C():
    """The shift C changes only the sampling, not the results (Sec. 4)."""
    res = []
    for C in (4 * 0.44 + 1e-3, 4 * 0.44 + 1.0):
        model = oracle.Model(dim=2, L=(4, 4), beta=0.44, C=C)
        res.append(_hmc_stats(model, 10000, 0.1, 10, seed=3)["E"])
    (m1, e1, _), (m2, e2, _) = res
    assert within(m1, m2, math.hypot(e1, e2))


def test_virial_identity():
    """<psi . grad S> = N in the psi ensemble."""
    model = oracle.Model(dim=2, L=(4, 4), beta=0.3, h=0.1)
    c = oracle.Chain(model, seed=4)
    vals = []
    for k in range(3000):
        c.trajectory(0.15, 7)
        if k >= 200:
            psi = c.psi
            vals.append(-psi @ oracle.force(model, psi))
    mean, err, _ = gamma_method(vals)
    assert within(mean, model.N, err)


@pytest.mark.slow
def test_onsager_energy_away_from_criticality():
    beta = 0.30
    model = oracle.Model(dim=2, L=(16, 16), beta=beta)
    st = _hmc_stats(model, 6000, 0.2, 5, n_therm=300)
    mean, err, _ = st["E"]
    assert within(mean, onsager_energy(beta), err, floor=2e-3), (mean, onsager_energy(beta), err)


@pytest.mark.slow
def test_metropolis_hastings_matches_brute_force():
    model = oracle.Model(dim=2, L=(4, 4), beta=0.44)
    bf = oracle.brute_force(model)
    r = oracle.mh_run(model, seed=5, n=40000, n_therm=500, series=True)
    n = r["n_meas"]
    mean_am, err_am, _ = gamma_method(r["abs_m"][500:])
    assert within(mean_am, bf["abs_m"], err_am)
    E = r["sum_E"] / n
    varE = r["sum_E2"] / n - E * E
    assert within(E, bf["E"], 4 * math.sqrt(varE / n))  # loose: tau_E small


# --------------------------------------- checkerboard Metropolis-Hastings ----
def test_checkerboard_mh_beta_zero_flips_every_spin():
    """beta = 0: every proposal has p = 1, so one sweep negates every spin."""
    model = oracle.Model(dim=2, L=(6, 4), beta=0.0, C=1.0)
    s0 = np.where(workloads.rng(4).random(24) < 0.5, 1, -1).astype(np.int8)
    s, sums = oracle.mh_checkerboard(model, seed=3, n=1, spins=s0)
    assert np.array_equal(s, -s0)
    assert sums[1] == 1.0   # flipped fraction


def test_checkerboard_mh_strong_field_aligns_in_one_sweep():
    """h = 50: from all -1 colour 0 flips (its neighbours are all -1), then colour 1
    (its neighbours now all +1); from all +1 nothing flips."""
    model = oracle.Model(dim=3, L=(4, 4, 4), beta=1.0, h=50.0, C=7.0)
    s, _ = oracle.mh_checkerboard(model, seed=1, n=1, spins=-np.ones(64, np.int8))
    assert np.all(s == 1)
    s, sums = oracle.mh_checkerboard(model, seed=1, n=3, spins=np.ones(64, np.int8))
    assert np.all(s == 1) and sums[1] == 0.0


def test_checkerboard_mh_colour_order_does_not_matter():
    """The same sweep with each colour's sites visited in reverse order (a plain
    loop here, from the oracle's Philox and acceptance probability) gives the
    same spins: the property that lets a GPU update a colour in parallel."""
    L0, L1, beta, J, h, seed = 6, 4, 0.5, 1.0, 0.1, 9
    model = oracle.Model(dim=2, L=(L0, L1), beta=beta, h=h)
    nbr = oracle.neighbors(model)
    s0 = np.where(workloads.rng(8).random(L0 * L1) < 0.5, 1, -1).astype(np.int8)
    s = s0.copy()
    for k in range(3):
        for c in (0, 1):
            for i in reversed(range(L0 * L1)):
                if ((i % L0) + (i // L0)) % 2 != c:
                    continue
                nb = int(sum(s[j] for j in nbr[i]))
                j = i // 2
                w = oracle.philox((j // 4, 2 * k + c, 0, oracle.PURPOSE_MH),
                                  (seed & 0xffffffff, seed >> 32))
                u = np.float32(oracle.u23(w[j % 4]))
                if u < np.float32(oracle.mh_accept_prob(beta, J, h, int(s[i]), nb)):
                    s[i] = -s[i]
    ref, _ = oracle.mh_checkerboard(model, seed=seed, n=3, spins=s0)
    assert np.array_equal(s, ref)


@pytest.mark.parametrize("dim,L,beta,h", [(2, (4, 4), 0.44, 0.05), (2, (4, 4), 0.3, 0.0),
                                         (1, (12,), 0.7, 0.1)])
def test_checkerboard_mh_matches_brute_force(dim, L, beta, h):
    """64 independent chains (chain index in the Philox counter), 2500 sweeps
    each after 200 of thermalisation: m, |m| and E within 3 standard errors of
    the exact sums over all spin states.  (On a ring at h = 0 local Metropolis
    is not ergodic -- a flip between unlike neighbours costs nothing and is
    always taken -- in site order as in checkerboard order, so 1D runs with a
    field.)"""
    model = oracle.Model(dim=dim, L=L, beta=beta, h=h)
    bf = oracle.brute_force(model)
    per = {k: [] for k in ("m", "abs_m", "E")}
    for c in range(64):
        _, sums = oracle.mh_checkerboard(model, seed=11, chain=c, n=2700, n_therm=200)
        per["m"].append(sums[2] / sums[0])
        per["E"].append(sums[4] / sums[0])
        per["abs_m"].append(sums[6] / sums[0])
    for key, v in per.items():
        v = np.asarray(v)
        assert within(v.mean(), bf[key], v.std(ddof=1) / math.sqrt(len(v))), (key, v.mean(), bf[key])


# ---------------------------------------- the paper's own parametrisation ----
def test_pform_is_the_ns_form_under_the_map():
    """P form (Sec. 2-3 as printed) vs NS form: with C = J' C_p, eps_ns = eps_p/sqrt(J'),
    psi_ns = psi_p/sqrt(J') - A^-1 h' and equal momenta, trajectories coincide."""
    beta, Cp, h = 0.4, 4 + 1e-5, 0.15
    base = oracle.Model(dim=2, L=(5, 4), beta=beta, h=h)
    Jp = beta * 1.0
    ns = base.with_(C=Jp * Cp)
    g = workloads.rng(12)
    psip = g.standard_normal(ns.N)
    p = g.standard_normal(ns.N)
    Ainv_h, it = oracle.cg_solve(ns, np.full(ns.N, beta * h))
    assert it >= 0
    to_ns = lambda x: x / math.sqrt(Jp) - Ainv_h
    # actions differ by a constant
    d1 = oracle.pform_action(base, Cp, psip) - oracle.action(ns, to_ns(psip))
    d2 = oracle.pform_action(base, Cp, 2 * psip) - oracle.action(ns, to_ns(2 * psip))
    assert abs(d1 - d2) < 1e-10
    # forces: F_p = F_ns / sqrt(J')
    np.testing.assert_allclose(oracle.pform_force(base, Cp, psip),
                               oracle.force(ns, to_ns(psip)) / math.sqrt(Jp), atol=1e-12)
    # trajectories
    eps_p = 0.1
    a_p, b_p = oracle.pform_leapfrog(base, Cp, psip, p, eps_p, 8)
    a_n, b_n = oracle.leapfrog(ns, to_ns(psip), p, eps_p / math.sqrt(Jp), 8)
    np.testing.assert_allclose(to_ns(a_p), a_n, atol=1e-11)
    np.testing.assert_allclose(b_p, b_n, atol=1e-11)


def test_constant_field_closed_form_of_hKh():
    """Constant h on a regular lattice: h'.Kt^-1 h' = N h0'^2 / (n0 + C_p) (Sec. 2)."""
    beta, Cp, h = 0.5, 4.3, 0.2
    m = oracle.Model(dim=2, L=(6, 5), beta=1.0, Jnn=1.0, C=Cp)  # A = K + C_p
    hp = np.full(m.N, beta * h)
    x, it = oracle.cg_solve(m, hp)
    assert it >= 0
    assert abs(hp @ x - m.N * (beta * h) ** 2 / (4 + Cp)) < 1e-12


# -------------------------------------------------------- planted mistakes ----
def _planted(flag):
    path = oracle.build(extra_flags=("-D" + flag,))
    return oracle._load(path)


def test_planted_neighbor_mistake_is_caught(monkeypatch):
    monkeypatch.setattr(oracle, "_lib", _planted("OR_PLANT_NEIGHBOR"))
    with pytest.raises(AssertionError):
        test_apply_A_plane_wave_eigenvalues(2, (6, 5))


def test_planted_force_sign_mistake_is_caught(monkeypatch):
    monkeypatch.setattr(oracle, "_lib", _planted("OR_PLANT_FORCE_SIGN"))
    with pytest.raises(AssertionError):
        test_force_is_minus_gradient_of_action(_models()[0])


def test_planted_action_mistake_is_caught(monkeypatch):
    monkeypatch.setattr(oracle, "_lib", _planted("OR_PLANT_ACTION"))
    with pytest.raises(AssertionError):
        test_force_is_minus_gradient_of_action(_models()[0])


def test_planted_leapfrog_mistake_is_caught(monkeypatch):
    monkeypatch.setattr(oracle, "_lib", _planted("OR_PLANT_LEAPFROG"))
    with pytest.raises(AssertionError):
        test_integrator_reversible("leapfrog")


def test_planted_omelyan_lambda_mistake_is_caught(monkeypatch):
    monkeypatch.setattr(oracle, "_lib", _planted("OR_PLANT_OMELYAN"))
    with pytest.raises(AssertionError):
        test_omelyan_lambda_is_the_minimum_norm_value()
