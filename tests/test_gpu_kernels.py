"""Device functions the trajectories rely on, against FP64 references."""
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


def test_tanh_absolute_error_and_symmetry():
    g = np.random.default_rng(0)
    x = np.concatenate([np.linspace(-30, 30, 2_000_001), g.standard_normal(1_000_000) * 3,
                        np.array([0.0, -0.0, 1e-30, -1e-30, 88.0, -88.0, 1e4, -1e4])]).astype(np.float32)
    t = binding.ising_hmc_selftest(binding.ISING_SELFTEST_TANH, x)
    ref = np.tanh(x.astype(np.float64))
    err = np.abs(t.astype(np.float64) - ref)
    assert err.max() < 3e-7, err.max()
    assert np.all(np.abs(t) <= 1.0)
    tn = binding.ising_hmc_selftest(binding.ISING_SELFTEST_TANH, -x)
    assert np.array_equal(tn, -t)
    assert np.all(np.isfinite(t))


def test_log1pexp_double_float_accuracy():
    g = np.random.default_rng(1)
    y = np.concatenate([np.linspace(0, 40, 400_001), g.uniform(0, 60, 200_000),
                        np.array([0.0, 1 / 32, 35.999, 36.0, 36.001, 700.0])])
    # inputs representable as a double-float (hi + lo of two FP32 numbers),
    # which is how the action hands them to the function
    hi = y.astype(np.float32).astype(np.float64)
    y = hi + (y - hi).astype(np.float32).astype(np.float64)
    out = binding.ising_hmc_selftest(binding.ISING_SELFTEST_LOG1PEXP, y)
    ref = np.log1p(np.exp(-y))
    # 1e-11 per site: rounding errors of varying sign add up to about 1e-8
    # over a million sites, far inside the 1e-6 that dH is held to
    assert np.abs(out - ref).max() < 1e-11, np.abs(out - ref).max()
