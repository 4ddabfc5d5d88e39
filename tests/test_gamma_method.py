"""The library's Gamma method (host code, no GPU) against processes whose
integrated autocorrelation time is known in closed form."""
import math

import numpy as np
import pytest

from paper_1912_03278_gb300 import binding
from tests.stats_util import gamma_method


@pytest.fixture(scope="module")
def lib():
    import paper_1912_03278_gb300 as pkg
    pkg.build()
    return binding.load()


def _ar1(rho, n, reps, seed):
    """x_t = rho x_{t-1} + sqrt(1 - rho^2) xi_t, stationary start: unit variance,
    autocorrelation rho^t, tau_int = (1 + rho) / (2 (1 - rho))."""
    g = np.random.default_rng(seed)
    x = np.empty((reps, n))
    x[:, 0] = g.standard_normal(reps)
    xi = g.standard_normal((reps, n)) * math.sqrt(1 - rho * rho)
    for t in range(1, n):
        x[:, t] = rho * x[:, t - 1] + xi[:, t]
    return x


@pytest.mark.parametrize("rho", [0.0, 0.5, 0.9])
def test_ar1_tau_int(lib, rho):
    x = _ar1(rho, 20000, 8, seed=int(rho * 10) + 1)
    r = binding.ising_gamma_method(x)
    exact = (1 + rho) / (2 * (1 - rho))
    assert abs(r["tau_int"] - exact) <= 3 * r["tau_err"] + 0.02 * exact, (r, exact)
    # error of the mean: sqrt(2 tau_int var / N) with var = 1
    assert abs(r["err"] / math.sqrt(2 * exact / x.size) - 1) < 0.1
    assert abs(r["mean"]) < 4 * r["err"]


def test_agrees_with_the_test_suites_gamma_method(lib):
    x = _ar1(0.8, 50000, 1, seed=3)[0]
    r = binding.ising_gamma_method(x)
    mean, err, tau = gamma_method(x)
    assert r["mean"] == pytest.approx(mean, rel=1e-12)
    assert r["tau_int"] == pytest.approx(tau, rel=0.05)
    assert r["err"] == pytest.approx(err, rel=0.05)


def test_constant_series_and_invalid_input(lib):
    r = binding.ising_gamma_method(np.full(100, 2.5))
    assert r["mean"] == 2.5 and r["err"] == 0.0 and r["tau_int"] == 0.5
    with pytest.raises(binding.IsingError):
        binding.ising_gamma_method(np.zeros(1))
    with pytest.raises(binding.IsingError):
        binding.ising_gamma_method(np.zeros(10), S=0.0)
