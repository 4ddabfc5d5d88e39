"""Error analysis for Markov-chain time series (test infrastructure).

gamma_method follows Wolff, "Monte Carlo errors with less errors" (2004):
the integrated autocorrelation time with automatic windowing, S = 1.5.
"""
import math

import numpy as np


def gamma_method(x, S=1.5):
    """Return (mean, error, tau_int) of a scalar series."""
    x = np.asarray(x, dtype=np.float64)
    n = len(x)
    mean = x.mean()
    d = x - mean
    var = d.var()
    if var == 0.0 or n < 4:
        return mean, 0.0, 0.5
    # autocorrelation by FFT
    f = np.fft.rfft(d, n=2 * n)
    acf = np.fft.irfft(f * np.conj(f))[:n] / np.arange(n, 0, -1)
    rho = acf / acf[0]
    tau = 0.5
    W_opt = n // 2
    for W in range(1, n // 2):
        tau = 0.5 + rho[1:W + 1].sum()
        if tau <= 0.5:
            W_opt = W
            tau = 0.5
            break
        t = S / math.log((2 * tau + 1) / (2 * tau - 1))
        g = math.exp(-W / t) - t / math.sqrt(W * n)
        if g < 0:
            W_opt = W
            break
    tau = max(0.5 + rho[1:W_opt + 1].sum(), 0.5)
    err = math.sqrt(2.0 * tau * var / n)
    return mean, err, tau


def within(a, b, sigma, k=3.0, floor=0.0):
    return abs(a - b) <= k * sigma + floor


def onsager_energy(beta, J=1.0):
    """Infinite square lattice, beta*u per site (Onsager 1944):
    u = -J coth(2bJ) [1 + (2/pi)(2 tanh^2(2bJ) - 1) K(k)], k = 2 sinh(2bJ)/cosh^2(2bJ)."""
    from scipy.special import ellipk
    b = beta * J
    k = 2.0 * math.sinh(2 * b) / math.cosh(2 * b) ** 2
    u = -J / math.tanh(2 * b) * (1.0 + 2.0 / math.pi * (2.0 * math.tanh(2 * b) ** 2 - 1.0)
                                  * ellipk(k * k))
    return beta * u


BETA_C_2D = 0.5 * math.log(1.0 + math.sqrt(2.0))
