"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module holds no arithmetic of the method: it only draws the model's
inputs (couplings, fields, start configurations, parameter sweeps) from
numpy's seeded generator and lists the workload shapes.  Both the oracle
tests and the GPU tests take their inputs from here.

Workloads follow the paper's experiments (Sec. 4): periodic square and
simple-cubic lattices with nearest-neighbour J = 1, and dense all-to-all
couplings (Sec. 2 allows a full coupling matrix in place of J K).
"""
from __future__ import annotations

import math

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence(seed))


def dense_couplings(N: int, seed: int = 1) -> np.ndarray:
    """Symmetric J with J_ij ~ Normal(0, 1/N) for i < j and J_ii = 0 (SK-type)."""
    g = rng(seed)
    upper = np.triu(g.standard_normal((N, N)) / math.sqrt(N), k=1)
    return upper + upper.T


def dense_fields(N: int, sigma: float = 0.1, seed: int = 2) -> np.ndarray:
    """Per-site fields h_i ~ Normal(0, sigma^2)."""
    return rng(seed).standard_normal(N) * sigma


def infinite_range_couplings(N: int, J: float = 1.0) -> np.ndarray:
    """All-to-all J/N off the diagonal (the paper's appendix model)."""
    Jm = np.full((N, N), J / N)
    np.fill_diagonal(Jm, 0.0)
    return Jm


def start_psi(n_chains: int, N: int, scale: float = 0.5, seed: int = 3) -> np.ndarray:
    """Random start configurations psi ~ Normal(0, scale^2), shape (n_chains, N)."""
    return rng(seed).standard_normal((n_chains, N)) * scale


def beta_sweep(lo: float = 0.38, hi: float = 0.50, n: int = 16) -> np.ndarray:
    """The 2D beta sweep around the Onsager point."""
    return np.linspace(lo, hi, n)


def lattice_C(beta, dim: int, J: float = 1.0, margin: float = 0.1):
    """Shift in NS units for a periodic lattice: beta*|J|*2*dim + margin."""
    return np.asarray(beta) * abs(J) * 2 * dim + margin


def n_md_default(N: int) -> int:
    """Steps per unit trajectory, floor(ln N) (Sec. 4)."""
    return max(1, int(math.floor(math.log(N))))


# Workload shapes (sites per chain x chains).
CONFIG_SMALL_2D = dict(dim=2, L=4, beta=0.44, h=0.0, eps=0.1, n_md=10, n_chains=1,
                       n_traj=20000, seed=0)
CONFIG_2D = dict(dim=2, Ls=(256, 1024), betas=beta_sweep(), chains_per_beta=256, n_md=20)
CONFIG_3D = dict(dim=3, Ls=(16, 24, 32, 48, 64), beta=0.2217, h=0.05, chains_per_size=64)
CONFIG_DENSE = dict(N=4096, B=1024, beta=0.5, h_sigma=0.1, J_seed=1)
