"""Host-side checks of the C ABI that need no GPU: the library builds, loads and
exports every entry point declared in include/ising_hmc.h; the Python binding
mirrors the header's structures; invalid configurations are rejected before
any device work."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import paper_1912_03278_gb300 as pkg
from paper_1912_03278_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ising_hmc.h")


@pytest.fixture(scope="module")
def lib():
    pkg.build()
    return pkg.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ising_\w+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    out = subprocess.run(["nm", "-D", "--defined-only", binding.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (ising_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert hasattr(lib, n)


def declared_all():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ising_\w+)\s*\(", src)))


def test_binding_covers_every_entry_point(lib):
    for n in declared_all():
        assert hasattr(binding, n) or n in ("ising_hmc_n_sites", "ising_hmc_n_chains",
                                            "ising_hmc_last_create_error"), n


def _struct_size_from_c(name):
    """Compile a tiny host program against the header to get sizeof/offsets."""
    import tempfile
    code = """
#include <stdio.h>
#include <stddef.h>
#include "ising_hmc.h"
int main(void) {
  printf("%%zu %%zu %%zu %%zu\\n", sizeof(%s), offsetof(ising_hmc_config, n_md),
         offsetof(ising_hmc_config, stream), sizeof(ising_obs));
  return 0;
}
""" % name
    d = tempfile.mkdtemp()
    src = os.path.join(d, "t.c")
    exe = os.path.join(d, "t")
    open(src, "w").write(code)
    subprocess.check_call(["gcc", "-I", os.path.dirname(HEADER), src, "-o", exe])
    return [int(x) for x in subprocess.check_output([exe]).split()]


def test_ctypes_structs_match_header():
    size, off_nmd, off_stream, obs_size = _struct_size_from_c("ising_hmc_config")
    assert ctypes.sizeof(binding.ising_hmc_config) == size
    assert binding.ising_hmc_config.n_md.offset == off_nmd
    assert binding.ising_hmc_config.stream.offset == off_stream
    assert ctypes.sizeof(binding.ising_obs) == obs_size


@pytest.mark.parametrize("kw,status", [
    (dict(dim=2, L=(2, 4)), binding.ISING_EINVAL),          # L < 3 would double the bonds
    (dict(dim=4, L=(4, 4)), binding.ISING_EINVAL),
    (dict(dim=2, L=(4, 4), n_chains=0), binding.ISING_EINVAL),
    (dict(dim=2, L=(4, 4), n_md=0), binding.ISING_EINVAL),
    (dict(dim=2, L=(4, 4), beta=0.44, C=4 * 0.44), binding.ISING_ENOTPD),  # C must exceed 2d beta J
    (dict(dim=2, L=(4, 4), eps=-0.1), binding.ISING_EINVAL),
    (dict(dim=2, L=(4, 4), precision=binding.ISING_PREC_BF16), binding.ISING_EINVAL),
    # infinite-range model: N >= 2, FP32 form only, C above the exact spectrum bound
    (dict(kind="infinite", n_sites=1), binding.ISING_EINVAL),
    (dict(kind="infinite", n_sites=64, precision=binding.ISING_PREC_PLAIN_FP64),
     binding.ISING_EINVAL),
    (dict(kind="infinite", n_sites=64, beta=1.0, C=0.99 / 64), binding.ISING_ENOTPD),
    (dict(kind="infinite", n_sites=64, Jnn=-1.0, beta=1.0, C=0.98), binding.ISING_ENOTPD),
    (dict(kind="crystal", n_sites=64), binding.ISING_EINVAL),
])
def test_invalid_configurations_rejected(lib, kw, status):
    if kw.get("kind") not in (None, "lattice", "dense", "infinite"):
        with pytest.raises(ValueError):
            binding.make_config(**kw)
        return
    cfg, keep = binding.make_config(**kw)
    with pytest.raises(binding.IsingError) as ei:
        binding.ising_hmc_create(cfg)
    assert ei.value.status == status
    assert len(binding.load().ising_hmc_last_create_error()) > 0


@pytest.mark.parametrize("kw", [
    dict(dim=2, L=(5, 4)),                   # odd extent: no checkerboard
    dict(dim=2, L=(2, 4)),                   # extent below 4
    dict(dim=4, L=(4, 4)),
    dict(dim=2, L=(4, 4), n_chains=0),
    dict(dim=2, L=(4, 4), n_chains=70000),
    dict(dim=2, L=(4, 4), h=np.zeros(16)),    # per-site field
    dict(dim=2, L=(4, 4), beta=-0.1),
])
def test_mh_invalid_configurations_rejected(lib, kw):
    cfg, keep = binding.make_config(**kw)
    out = ctypes.c_void_p()
    st = binding.load().ising_mh_create(ctypes.byref(cfg), ctypes.byref(out))
    assert st == binding.ISING_EINVAL and not out.value
    assert len(binding.load().ising_mh_last_error(None)) > 0


def test_dense_not_positive_definite_rejected(lib):
    import workloads
    J = workloads.dense_couplings(40, seed=3)
    lam = np.linalg.eigvalsh(J)[0]
    cfg, keep = binding.make_config(kind="dense", J=J, beta=0.5, C=0.5 * abs(lam) * 0.99,
                                    precision=binding.ISING_PREC_PLAIN_FP64)
    with pytest.raises(binding.IsingError) as ei:
        binding.ising_hmc_create(cfg)
    assert ei.value.status == binding.ISING_ENOTPD


def test_dense_asymmetric_rejected(lib):
    J = np.zeros((5, 5))
    J[0, 1] = 0.3
    cfg, keep = binding.make_config(kind="dense", J=J, beta=0.5, C=1.0,
                                    precision=binding.ISING_PREC_PLAIN_FP64)
    with pytest.raises(binding.IsingError) as ei:
        binding.ising_hmc_create(cfg)
    assert ei.value.status == binding.ISING_EINVAL


def test_estimate_bytes(lib):
    cfg, keep = binding.make_config(dim=2, L=(1024, 1024), n_chains=4096)
    assert binding.ising_hmc_estimate_bytes(cfg) >= 16 * 1024 * 1024 * 4096
    # infinite range: three psi buffers and p in FP32, no coupling matrix
    cfg, keep = binding.make_config(kind="infinite", n_sites=4096, n_chains=4864)
    est = binding.ising_hmc_estimate_bytes(cfg)
    assert 16 * 4096 * 4864 <= est < 17 * 4096 * 4864
