"""GB300-native Hybrid Monte Carlo for the Ising model in its Hubbard-
Stratonovich auxiliary-field form (arXiv:1912.03278).

The compute path is the CUDA library ``lib/libising_hmc.so`` (C ABI in
``include/ising_hmc.h``); :mod:`.binding` marshals arguments to it.
"""
from .binding import *  # noqa: F401,F403
from .binding import IsingGroup, IsingHMC, IsingError, IsingMH, IsingServer, load, make_config  # noqa: F401


def build(force: bool = False) -> str:
    from .builder import build as _build
    return _build(force=force)
