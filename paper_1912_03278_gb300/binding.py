"""ctypes binding of the C ABI in include/ising_hmc.h (argument marshalling only).

Every function here has the name of the C entry point it calls; all work runs
in the CUDA library.  The library is loaded from this package's ``lib/``
directory; if it is missing the import of a function raises, there is no
fallback.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_int, c_int64, c_uint64, c_void_p

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libising_hmc.so")

# status codes
ISING_OK, ISING_EINVAL, ISING_ENOTPD, ISING_ENOMEM, ISING_ECUDA, ISING_ETIMEOUT, ISING_EBUSY = range(7)
ISING_STAGING_AUTO, ISING_STAGING_THREADS, ISING_STAGING_BULK = range(3)
STATUS_NAMES = ["OK", "EINVAL", "ENOTPD", "ENOMEM", "ECUDA", "ETIMEOUT", "EBUSY"]
ISING_KIND_LATTICE, ISING_KIND_DENSE, ISING_KIND_INFINITE = 0, 1, 2
_KINDS = {"lattice": ISING_KIND_LATTICE, "dense": ISING_KIND_DENSE,
          "infinite": ISING_KIND_INFINITE}
ISING_PREC_PLAIN_FP64, ISING_PREC_FP32, ISING_PREC_BF16, ISING_PREC_FP8 = 0, 1, 2, 3
ISING_INTEGRATOR_LEAPFROG, ISING_INTEGRATOR_OMELYAN = 0, 1
ISING_STATE_PSI, ISING_STATE_PSI_PROPOSAL, ISING_STATE_P_END = 0, 1, 2
SUM_NAMES = ["n_meas", "n_acc", "sum_m", "sum_m2", "sum_E", "sum_E2", "sum_am", "sum_am2",
             "sum_dH", "sum_expmdH"]
ISING_NSUMS = len(SUM_NAMES)
REC_NAMES = ["dH", "logu", "accepted", "K0", "S0", "K1", "S1", "flipped"]
ISING_NREC = len(REC_NAMES)


class IsingError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES[status] if 0 <= status < 7 else status, msg))
        self.status = status


class ising_hmc_config(ctypes.Structure):
    _fields_ = [("kind", c_int), ("dim", c_int), ("L", c_int * 3), ("n_sites", c_int64),
                ("J", c_void_p), ("Jnn", c_double), ("h", c_void_p), ("h0", c_double),
                ("beta", c_double), ("C", c_double), ("eps", c_double),
                ("beta_chain", c_void_p), ("C_chain", c_void_p), ("eps_chain", c_void_p),
                ("h0_chain", c_void_p), ("n_md", c_int), ("n_chains", c_int), ("n_therm", c_int),
                ("precision", c_int), ("integrator", c_int), ("flip_every", c_int),
                ("stream", c_void_p)]


class ising_obs(ctypes.Structure):
    _fields_ = [("m", c_double), ("m_err", c_double), ("abs_m", c_double),
                ("abs_m_err", c_double), ("E", c_double), ("E_err", c_double),
                ("acceptance", c_double), ("mean_dH", c_double), ("mean_exp_mdH", c_double),
                ("exp_mdH_err", c_double), ("n_traj", c_int64), ("n_meas", c_int64)]


_lib = None


def load(path: str | None = None):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise OSError("libising_hmc.so not built (%s); run paper_1912_03278_gb300.builder" % p)
    lib = ctypes.CDLL(p)
    P = c_void_p
    sig = {
        "ising_hmc_create": (c_int, [P, P]),
        "ising_hmc_trajectories": (c_int, [P, c_int64, c_uint64]),
        "ising_hmc_observables": (c_int, [P, P]),
        "ising_hmc_chain_sums": (c_int, [P, P]),
        "ising_hmc_last_records": (c_int, [P, P]),
        "ising_hmc_reset_sums": (c_int, [P]),
        "ising_hmc_get_state": (c_int, [P, c_int, P]),
        "ising_hmc_set_state": (c_int, [P, P, c_int64]),
        "ising_hmc_set_state_native": (c_int, [P, P, c_int64]),
        "ising_hmc_get_state_native": (c_int, [P, P]),
        "ising_hmc_state_elem_bytes": (c_int, [P]),
        "ising_hmc_set_sums": (c_int, [P, P]),
        "ising_hmc_momenta": (c_int, [P, c_uint64, c_int64, c_int, c_int, P]),
        "ising_hmc_get_chains": (c_int, [P, c_int, c_int, c_int, P]),
        "ising_hmc_set_eps": (c_int, [P, P]),
        "ising_hmc_chain_params": (c_int, [P, P]),
        "ising_hmc_traj_index": (c_int64, [P]),
        "ising_hmc_n_sites": (c_int64, [P]),
        "ising_hmc_n_chains": (c_int, [P]),
        "ising_hmc_device_bytes": (c_int64, [P]),
        "ising_hmc_estimate_bytes": (c_int64, [P]),
        "ising_hmc_launch_count": (c_int64, [P]),
        "ising_hmc_sync": (c_int, [P]),
        "ising_hmc_selftest": (c_int, [c_int, P, P, c_int64]),
        "ising_hmc_selftest_gemm": (c_int, [c_int, c_int, c_int, P, P, P]),
        "ising_hmc_dense_forces": (c_int, [P, c_int]),
        "ising_hmc_set_launch": (c_int, [P, c_int, c_int]),
        "ising_hmc_get_launch": (c_int, [P, P, P]),
        "ising_hmc_autotune": (c_int, [P, c_int, P]),
        "ising_hmc_set_chain_split": (c_int, [P, c_int]),
        "ising_hmc_get_chain_split": (c_int, [P]),
        "ising_hmc_set_staging": (c_int, [P, c_int]),
        "ising_hmc_get_staging": (c_int, [P]),
        "ising_group_autotune": (c_int, [P, c_int, P]),
        "ising_group_create": (c_int, [P, c_int, P]),
        "ising_group_trajectories": (c_int, [P, c_int64, c_uint64]),
        "ising_group_trajectories_seeds": (c_int, [P, c_int64, P]),
        "ising_server_create": (c_int, [c_int64, c_int, P]),
        "ising_server_submit": (c_int, [P, P, c_int64, c_uint64, P]),
        "ising_server_poll": (c_int, [P, c_int64, P, P, P, P]),
        "ising_server_wait": (c_int, [P, c_int64, c_double]),
        "ising_server_drain": (c_int, [P, c_double]),
        "ising_server_stats": (c_int, [P, P]),
        "ising_server_last_error": (c_char_p, [P]),
        "ising_server_destroy": (None, [P]),
        "ising_group_sync": (c_int, [P]),
        "ising_group_launch_count": (c_int64, [P]),
        "ising_group_stream": (c_void_p, [P]),
        "ising_group_last_error": (c_char_p, [P]),
        "ising_group_destroy": (None, [P]),
        "ising_hmc_energy_noalloc": (c_int, [c_int, P, c_double, c_double, c_double, c_double,
                                             c_int, P, P, P, P]),
        "ising_hmc_energy_noalloc_error": (c_char_p, []),
        "ising_hmc_destroy": (None, [P]),
        "ising_hmc_inject_alloc_failure": (None, [c_int64]),
        "ising_hmc_inject_device_error": (c_int, [P, c_int]),
        "ising_hmc_solve_A": (c_int, [P, c_int, P, P, c_double, c_int, P, P]),
        "ising_hmc_series_enable": (c_int, [P, c_int64]),
        "ising_hmc_series_get": (c_int, [P, P, P]),
        "ising_gamma_method": (c_int, [P, c_int64, c_int, c_double, P]),
        "ising_mh_create": (c_int, [P, P]),
        "ising_mh_sweeps": (c_int, [P, c_int64, c_uint64]),
        "ising_mh_observables": (c_int, [P, P]),
        "ising_mh_chain_sums": (c_int, [P, P]),
        "ising_mh_get_spins": (c_int, [P, P]),
        "ising_mh_set_spins": (c_int, [P, P, c_int64]),
        "ising_mh_sync": (c_int, [P]),
        "ising_mh_sweep_index": (c_int64, [P]),
        "ising_mh_launch_count": (c_int64, [P]),
        "ising_mh_last_error": (c_char_p, [P]),
        "ising_mh_destroy": (None, [P]),
        "ising_hmc_last_error": (c_char_p, [P]),
        "ising_hmc_last_create_error": (c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(h, st):
    if st != ISING_OK:
        lib = load()
        msg = lib.ising_hmc_last_error(h) if h else lib.ising_hmc_last_create_error()
        raise IsingError(st, (msg or b"").decode())


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def make_config(kind="lattice", dim=2, L=(4, 4), n_sites=0, J=None, Jnn=1.0, h=0.0, beta=0.44,
                C=None, eps=0.1, n_md=10, n_chains=1, n_therm=0, precision=ISING_PREC_FP32,
                integrator=ISING_INTEGRATOR_LEAPFROG, flip_every=0, stream=None):
    """Build an ising_hmc_config; array arguments may be per chain (beta, C, eps)
    or per site (h).  Returns (config, keepalive) -- keep both alive until the
    create call returns."""
    cfg = ising_hmc_config()
    keep = []
    if kind not in _KINDS:
        raise ValueError("kind must be one of %s" % sorted(_KINDS))
    cfg.kind = _KINDS[kind]
    cfg.dim = dim
    Lt = tuple(L) + (1,) * (3 - len(L))
    for i in range(3):
        cfg.L[i] = int(Lt[i])
    if kind == "dense":
        Jm = _f64(J)
        keep.append(Jm)
        cfg.J = Jm.ctypes.data
        cfg.n_sites = Jm.shape[0]
    elif kind == "infinite":
        cfg.n_sites = int(n_sites)
    cfg.Jnn = Jnn
    if np.isscalar(h):
        cfg.h = None
        cfg.h0 = float(h)
    else:
        hv = _f64(h)
        keep.append(hv)
        cfg.h = hv.ctypes.data
        cfg.h0 = 0.0

    def per_chain(name, v):
        if v is None:
            return
        if np.isscalar(v):
            setattr(cfg, name, float(v))
        else:
            arr = _f64(v)
            if arr.shape != (n_chains,):
                raise ValueError("%s must have one value per chain" % name)
            keep.append(arr)
            setattr(cfg, name + "_chain", arr.ctypes.data)
            setattr(cfg, name, float(arr[0]))

    per_chain("beta", beta)
    if C is None:
        C = 0.0   # the library's default shift (Sec. 2 bound + 0.1)
    per_chain("C", C)
    per_chain("eps", eps)
    cfg.n_md = n_md
    cfg.n_chains = n_chains
    cfg.n_therm = n_therm
    cfg.precision = precision
    cfg.integrator = integrator
    cfg.flip_every = flip_every
    cfg.stream = stream
    return cfg, keep


def ising_hmc_create(cfg: ising_hmc_config) -> int:
    lib = load()
    out = c_void_p()
    _check(None, lib.ising_hmc_create(ctypes.byref(cfg), ctypes.byref(out)))
    return out.value


def ising_hmc_trajectories(h, n, seed):
    _check(h, load().ising_hmc_trajectories(h, int(n), int(seed)))


def ising_hmc_observables(h) -> dict:
    o = ising_obs()
    _check(h, load().ising_hmc_observables(h, ctypes.byref(o)))
    return {k: getattr(o, k) for k, _ in ising_obs._fields_}


def ising_hmc_chain_sums(h) -> np.ndarray:
    n = load().ising_hmc_n_chains(h)
    out = np.zeros((n, ISING_NSUMS))
    _check(h, load().ising_hmc_chain_sums(h, out.ctypes.data))
    return out


def ising_hmc_last_records(h) -> np.ndarray:
    n = load().ising_hmc_n_chains(h)
    out = np.zeros((n, ISING_NREC))
    _check(h, load().ising_hmc_last_records(h, out.ctypes.data))
    return out


def ising_hmc_reset_sums(h):
    _check(h, load().ising_hmc_reset_sums(h))


def ising_hmc_set_sums(h, sums):
    s = _f64(sums)
    _check(h, load().ising_hmc_set_sums(h, s.ctypes.data))


def ising_hmc_get_state(h, which=ISING_STATE_PSI) -> np.ndarray:
    lib = load()
    n, N = lib.ising_hmc_n_chains(h), lib.ising_hmc_n_sites(h)
    out = np.zeros((n, N))
    _check(h, lib.ising_hmc_get_state(h, which, out.ctypes.data))
    return out


def ising_hmc_set_state(h, psi, next_traj):
    lib = load()
    n, N = lib.ising_hmc_n_chains(h), lib.ising_hmc_n_sites(h)
    arr = _f64(psi).reshape(n, N)
    _check(h, lib.ising_hmc_set_state(h, arr.ctypes.data, int(next_traj)))


def ising_hmc_set_state_native(h, ptr, next_traj):
    """psi as a raw pointer (int) to n_chains*N elements in the state precision,
    device or host memory."""
    _check(h, load().ising_hmc_set_state_native(h, c_void_p(ptr), int(next_traj)))


def ising_hmc_get_state_native(h, ptr):
    _check(h, load().ising_hmc_get_state_native(h, c_void_p(ptr)))


def ising_hmc_state_elem_bytes(h) -> int:
    return load().ising_hmc_state_elem_bytes(h)


def ising_hmc_momenta(h, seed, traj, chain0=0, count=None) -> np.ndarray:
    lib = load()
    n, N = lib.ising_hmc_n_chains(h), lib.ising_hmc_n_sites(h)
    count = n - chain0 if count is None else count
    out = np.zeros((count, N))
    _check(h, lib.ising_hmc_momenta(h, int(seed), int(traj), chain0, count, out.ctypes.data))
    return out


def ising_hmc_get_chains(h, which, chain0, count) -> np.ndarray:
    lib = load()
    N = lib.ising_hmc_n_sites(h)
    out = np.zeros((count, N))
    _check(h, lib.ising_hmc_get_chains(h, which, chain0, count, out.ctypes.data))
    return out


def ising_hmc_set_eps(h, eps):
    e = _f64(eps)
    _check(h, load().ising_hmc_set_eps(h, e.ctypes.data))


def ising_hmc_chain_params(h) -> np.ndarray:
    """(n_chains, 3) array of (beta, C, eps) as the handle uses them."""
    out = np.zeros((load().ising_hmc_n_chains(h), 3))
    _check(h, load().ising_hmc_chain_params(h, out.ctypes.data))
    return out


def ising_hmc_traj_index(h) -> int:
    return load().ising_hmc_traj_index(h)


def ising_hmc_device_bytes(h) -> int:
    return load().ising_hmc_device_bytes(h)


def ising_hmc_estimate_bytes(cfg) -> int:
    return load().ising_hmc_estimate_bytes(ctypes.byref(cfg))


def ising_hmc_launch_count(h) -> int:
    return load().ising_hmc_launch_count(h)


def ising_hmc_sync(h):
    _check(h, load().ising_hmc_sync(h))


ISING_SELFTEST_TANH, ISING_SELFTEST_LOG1PEXP = 0, 1


def ising_hmc_selftest(which, x) -> np.ndarray:
    """Evaluate a device function on host data (see the header)."""
    dt = np.float32 if which == ISING_SELFTEST_TANH else np.float64
    xin = np.ascontiguousarray(x, dtype=dt)
    out = np.zeros_like(xin)
    _check(None, load().ising_hmc_selftest(which, xin.ctypes.data, out.ctypes.data, xin.size))
    return out


def ising_hmc_set_launch(h, threads, depth):
    _check(h, load().ising_hmc_set_launch(h, int(threads), int(depth)))


def ising_hmc_get_launch(h):
    t, d = ctypes.c_int(), ctypes.c_int()
    _check(h, load().ising_hmc_get_launch(h, ctypes.byref(t), ctypes.byref(d)))
    return t.value, d.value


def ising_hmc_autotune(h, reps=2) -> float:
    ms = c_double()
    _check(h, load().ising_hmc_autotune(h, int(reps), ctypes.byref(ms)))
    return ms.value


def ising_hmc_set_chain_split(h, ctas):
    _check(h, load().ising_hmc_set_chain_split(h, int(ctas)))


def ising_hmc_get_chain_split(h) -> int:
    return load().ising_hmc_get_chain_split(h)


def ising_hmc_set_staging(h, mode):
    _check(h, load().ising_hmc_set_staging(h, int(mode)))


def ising_hmc_get_staging(h) -> int:
    return load().ising_hmc_get_staging(h)


def ising_group_autotune(g, reps=2) -> float:
    ms = c_double()
    _gcheck(g, load().ising_group_autotune(g, int(reps), ctypes.byref(ms)))
    return ms.value


def ising_hmc_dense_forces(h, n):
    _check(h, load().ising_hmc_dense_forces(h, int(n)))


def _gcheck(g, st):
    if st != ISING_OK:
        msg = load().ising_group_last_error(g)
        raise IsingError(st, (msg or b"").decode())


def ising_group_create(handles) -> int:
    arr = (c_void_p * len(handles))(*handles)
    out = c_void_p()
    _gcheck(None, load().ising_group_create(arr, len(handles), ctypes.byref(out)))
    return out.value


def ising_group_trajectories(g, n, seed):
    _gcheck(g, load().ising_group_trajectories(g, int(n), int(seed)))


def ising_group_trajectories_seeds(g, n, seeds):
    arr = np.ascontiguousarray(seeds, dtype=np.uint64)
    _gcheck(g, load().ising_group_trajectories_seeds(g, int(n), arr.ctypes.data))


def ising_group_sync(g):
    _gcheck(g, load().ising_group_sync(g))


def ising_group_launch_count(g) -> int:
    return load().ising_group_launch_count(g)


def ising_group_stream(g) -> int:
    return load().ising_group_stream(g)


def ising_group_last_error(g) -> str:
    return (load().ising_group_last_error(g) or b"").decode()


def ising_group_destroy(g):
    if g:
        load().ising_group_destroy(g)


def ising_hmc_solve_A(h, chain, b, tol=1e-13, max_iter=10000):
    """x with A x = b for one chain (FP64 conjugate gradients on the device);
    returns (x, iterations, relative residual)."""
    bv = _f64(b)
    x = np.zeros_like(bv)
    it = ctypes.c_int(0)
    res = c_double(0.0)
    _check(h, load().ising_hmc_solve_A(h, int(chain), bv.ctypes.data, x.ctypes.data, float(tol),
                                       int(max_iter), ctypes.byref(it), ctypes.byref(res)))
    return x, it.value, res.value


# --------------------------------------- series and autocorrelation ----
def ising_hmc_series_enable(h, capacity):
    _check(h, load().ising_hmc_series_enable(h, int(capacity)))


def ising_hmc_series_get(h) -> np.ndarray:
    """Recorded series as an array (n_chains, n, 3): m, beta*eps, |m|."""
    n = ctypes.c_int64(0)
    _check(h, load().ising_hmc_series_get(h, None, ctypes.byref(n)))
    nc = load().ising_hmc_n_chains(h)
    out = np.zeros((nc, n.value, 3))
    if n.value:
        _check(h, load().ising_hmc_series_get(h, out.ctypes.data, ctypes.byref(n)))
    return out


def ising_gamma_method(x, S=1.5) -> dict:
    """Gamma method on a series (1D) or replicas (2D array, one row per replica)."""
    a = np.ascontiguousarray(np.atleast_2d(x), dtype=np.float64)
    out = np.zeros(5)
    _check(None, load().ising_gamma_method(a.ctypes.data, a.shape[1], a.shape[0], float(S),
                                           out.ctypes.data))
    return dict(mean=out[0], err=out[1], tau_int=out[2], tau_err=out[3], window=int(out[4]))


# ------------------------------------------ local Metropolis-Hastings ----
def _check_mh(h, st):
    if st != ISING_OK:
        msg = load().ising_mh_last_error(h)
        raise IsingError(st, (msg or b"").decode())


def ising_mh_create(cfg: ising_hmc_config) -> int:
    out = c_void_p()
    _check_mh(None, load().ising_mh_create(ctypes.byref(cfg), ctypes.byref(out)))
    return out.value


def ising_mh_sweeps(h, n, seed):
    _check_mh(h, load().ising_mh_sweeps(h, int(n), int(seed)))


def ising_mh_observables(h) -> dict:
    o = ising_obs()
    _check_mh(h, load().ising_mh_observables(h, ctypes.byref(o)))
    return {k: getattr(o, k) for k, _ in ising_obs._fields_}


def ising_mh_chain_sums(h, n_chains) -> np.ndarray:
    out = np.zeros((n_chains, ISING_NSUMS))
    _check_mh(h, load().ising_mh_chain_sums(h, out.ctypes.data))
    return out


def ising_mh_get_spins(h, n_chains, N) -> np.ndarray:
    out = np.zeros((n_chains, N), dtype=np.int8)
    _check_mh(h, load().ising_mh_get_spins(h, out.ctypes.data))
    return out


def ising_mh_set_spins(h, spins, next_sweep=0):
    a = np.ascontiguousarray(spins, dtype=np.int8)
    _check_mh(h, load().ising_mh_set_spins(h, a.ctypes.data, int(next_sweep)))


def ising_mh_sync(h):
    _check_mh(h, load().ising_mh_sync(h))


def ising_mh_sweep_index(h) -> int:
    return load().ising_mh_sweep_index(h)


def ising_mh_launch_count(h) -> int:
    return load().ising_mh_launch_count(h)


def ising_mh_last_error(h) -> str:
    return (load().ising_mh_last_error(h) or b"").decode()


def ising_mh_destroy(h):
    load().ising_mh_destroy(h)


class IsingMH:
    """The local Metropolis-Hastings comparator (Sec. 4) on the GPU: checkerboard
    sweeps of many lattice chains.  IsingMH(**make_config kwargs); the lattice
    kind, dim, L (even extents), Jnn, scalar h, beta (per chain allowed),
    n_chains, n_therm and stream are used."""

    def __init__(self, **kw):
        cfg, keep = make_config(**kw)
        self.h = ising_mh_create(cfg)
        del keep
        self.n_chains = int(kw.get("n_chains", 1))
        L = tuple(kw.get("L", (4, 4)))[: kw.get("dim", 2)]
        self.N = int(np.prod(L))

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def close(self):
        if self.h:
            ising_mh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sweeps(self, n, seed):
        ising_mh_sweeps(self.h, n, seed)

    def observables(self) -> dict:
        return ising_mh_observables(self.h)

    def chain_sums(self) -> np.ndarray:
        return ising_mh_chain_sums(self.h, self.n_chains)

    def spins(self) -> np.ndarray:
        return ising_mh_get_spins(self.h, self.n_chains, self.N)

    def set_spins(self, spins, next_sweep=0):
        if np.size(spins) != self.n_chains * self.N:
            raise ValueError("need n_chains * N spins")
        ising_mh_set_spins(self.h, spins, next_sweep)

    def sync(self):
        ising_mh_sync(self.h)

    @property
    def sweep_index(self):
        return ising_mh_sweep_index(self.h)

    @property
    def launches(self):
        return ising_mh_launch_count(self.h)


class IsingGroup:
    """Several IsingHMC objects advanced by one CUDA-graph launch per call."""

    def __init__(self, sims):
        self.sims = list(sims)
        self.g = ising_group_create([s.h for s in self.sims])

    def trajectories(self, n, seed):
        ising_group_trajectories(self.g, n, seed)

    def sync(self):
        ising_group_sync(self.g)

    def autotune(self, reps=2):
        """Pick every member's chain split for the fastest group launch."""
        return ising_group_autotune(self.g, reps)

    @property
    def launches(self):
        return ising_group_launch_count(self.g)

    @property
    def stream(self):
        """cudaStream_t (as an integer) the group's graph launches run on."""
        return ising_group_stream(self.g) or 0

    def close(self):
        if self.g:
            ising_group_destroy(self.g)
            self.g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _scheck(s, st):
    if st != ISING_OK:
        msg = load().ising_server_last_error(s)
        raise IsingError(st, (msg or b"").decode())


ISING_SERVER_NSTATS = 14
SERVER_STAT_NAMES = ["admitted", "completed", "rejected", "queued", "active", "bytes_in_use",
                     "site_steps", "group_launches", "quanta", "seconds",
                     "create_s", "graph_s", "quanta_s", "retire_s"]


def ising_server_create(budget_bytes, quantum_traj) -> int:
    out = c_void_p()
    _scheck(None, load().ising_server_create(int(budget_bytes), int(quantum_traj),
                                             ctypes.byref(out)))
    return out.value


def ising_server_submit(s, cfg, n_traj, seed) -> int:
    rid = c_int64()
    _scheck(s, load().ising_server_submit(s, ctypes.byref(cfg), int(n_traj), int(seed),
                                          ctypes.byref(rid)))
    return rid.value


def ising_server_poll(s, rid):
    state = c_int()
    o = ising_obs()
    lat, q = c_double(), c_double()
    st = load().ising_server_poll(s, int(rid), ctypes.byref(state), ctypes.byref(o),
                                  ctypes.byref(lat), ctypes.byref(q))
    res = dict(state=state.value, status=st)
    if state.value >= 2:
        res.update(latency=lat.value, queue=q.value,
                   obs={k: getattr(o, k) for k, _ in ising_obs._fields_})
    return res


def ising_server_wait(s, rid, timeout_s):
    _scheck(s, load().ising_server_wait(s, int(rid), float(timeout_s)))


def ising_server_drain(s, timeout_s):
    _scheck(s, load().ising_server_drain(s, float(timeout_s)))


def ising_server_stats(s) -> dict:
    out = np.zeros(ISING_SERVER_NSTATS)
    _scheck(s, load().ising_server_stats(s, out.ctypes.data))
    return dict(zip(SERVER_STAT_NAMES, out.tolist()))


def ising_server_last_error(s) -> str:
    return (load().ising_server_last_error(s) or b"").decode()


def ising_server_destroy(s):
    if s:
        load().ising_server_destroy(s)


class IsingServer:
    """Continuous-batching request loop (see the header)."""

    def __init__(self, budget_bytes, quantum_traj=4):
        self.s = ising_server_create(budget_bytes, quantum_traj)

    def submit(self, n_traj, seed, **kw):
        cfg, keep = make_config(**kw)
        rid = ising_server_submit(self.s, cfg, n_traj, seed)
        del keep
        return rid

    def poll(self, rid):
        return ising_server_poll(self.s, rid)

    def wait(self, rid, timeout_s=60.0):
        ising_server_wait(self.s, rid, timeout_s)
        return self.poll(rid)

    def drain(self, timeout_s=600.0):
        ising_server_drain(self.s, timeout_s)

    def stats(self):
        return ising_server_stats(self.s)

    def close(self):
        if self.s:
            ising_server_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


ISING_NOALLOC_MAX_CHAINS = 64


def ising_hmc_energy_noalloc(dim, L, beta, Jnn, C, h0, n_chains, psi_ptr, p_ptr, out_ptr,
                             stream=None):
    """FP64 S and 1/2 p.p of n_chains lattice configurations without any
    allocation; all pointers are device addresses owned by the caller."""
    Lc = (c_int * 3)(*[int(x) for x in (tuple(L) + (1, 1, 1))[:3]])
    st = load().ising_hmc_energy_noalloc(int(dim), Lc, float(beta), float(Jnn), float(C),
                                         float(h0), int(n_chains), c_void_p(psi_ptr),
                                         c_void_p(p_ptr) if p_ptr else None, c_void_p(out_ptr),
                                         c_void_p(stream) if stream else None)
    if st != ISING_OK:
        raise IsingError(st, (load().ising_hmc_energy_noalloc_error() or b"").decode())


def ising_hmc_energy_noalloc_error() -> str:
    return (load().ising_hmc_energy_noalloc_error() or b"").decode()


def ising_hmc_selftest_gemm(A_bf16_bits, B_bf16_bits) -> np.ndarray:
    """D (N x M, n-major) = B A^T from BF16 bit patterns (uint16 arrays M x K, N x K)."""
    A = np.ascontiguousarray(A_bf16_bits, dtype=np.uint16)
    B = np.ascontiguousarray(B_bf16_bits, dtype=np.uint16)
    M, K = A.shape
    N = B.shape[0]
    D = np.zeros((N, M), dtype=np.float32)
    _check(None, load().ising_hmc_selftest_gemm(M, N, K, A.ctypes.data, B.ctypes.data,
                                                D.ctypes.data))
    return D


def ising_hmc_inject_alloc_failure(k):
    """Test hook: the k-th next device allocation fails (k <= 0 cancels)."""
    load().ising_hmc_inject_alloc_failure(int(k))


def ising_hmc_inject_device_error(h, bits):
    """Test hook: OR bits into the handle's device error word."""
    _check(h, load().ising_hmc_inject_device_error(h, int(bits)))


def ising_hmc_destroy(h):
    if h:
        load().ising_hmc_destroy(h)


def ising_hmc_last_error(h) -> str:
    return (load().ising_hmc_last_error(h) or b"").decode()


class IsingHMC:
    """Owning wrapper around a handle: IsingHMC(**make_config kwargs)."""

    def __init__(self, **kw):
        cfg, keep = make_config(**kw)
        self.h = ising_hmc_create(cfg)
        self.kw = kw
        del keep

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def close(self):
        if self.h:
            ising_hmc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def trajectories(self, n, seed):
        ising_hmc_trajectories(self.h, n, seed)

    def observables(self):
        return ising_hmc_observables(self.h)

    def chain_sums(self):
        return ising_hmc_chain_sums(self.h)

    def records(self):
        return ising_hmc_last_records(self.h)

    def state(self, which=ISING_STATE_PSI):
        return ising_hmc_get_state(self.h, which)

    def set_state(self, psi, next_traj):
        ising_hmc_set_state(self.h, psi, next_traj)

    def momenta(self, seed, traj, chain0=0, count=None):
        return ising_hmc_momenta(self.h, seed, traj, chain0, count)

    def chains(self, which, chain0, count):
        return ising_hmc_get_chains(self.h, which, chain0, count)

    def set_eps(self, eps):
        ising_hmc_set_eps(self.h, eps)

    def reset_sums(self):
        ising_hmc_reset_sums(self.h)

    @property
    def params(self):
        """(n_chains, 3) array of (beta, C, eps) per chain."""
        return ising_hmc_chain_params(self.h)

    def autotune(self, reps=2):
        return ising_hmc_autotune(self.h, reps)

    def dense_forces(self, n):
        """Queue n force evaluations (BF16 dense form; timing aid)."""
        ising_hmc_dense_forces(self.h, n)

    def set_launch(self, threads, depth):
        ising_hmc_set_launch(self.h, threads, depth)

    @property
    def launch(self):
        return ising_hmc_get_launch(self.h)

    def set_chain_split(self, ctas):
        ising_hmc_set_chain_split(self.h, ctas)

    @property
    def chain_split(self):
        return ising_hmc_get_chain_split(self.h)

    def set_staging(self, mode):
        """ISING_STAGING_AUTO, _THREADS or _BULK (FP32 lattice form)."""
        ising_hmc_set_staging(self.h, mode)

    @property
    def staging(self):
        return ising_hmc_get_staging(self.h)

    def sync(self):
        ising_hmc_sync(self.h)

    def solve_A(self, b, chain=0, tol=1e-13, max_iter=10000):
        return ising_hmc_solve_A(self.h, chain, b, tol, max_iter)

    def series_enable(self, capacity):
        ising_hmc_series_enable(self.h, capacity)

    def series(self) -> np.ndarray:
        return ising_hmc_series_get(self.h)

    @property
    def traj_index(self):
        return ising_hmc_traj_index(self.h)

    @property
    def launches(self):
        return ising_hmc_launch_count(self.h)

    @property
    def device_bytes(self):
        return ising_hmc_device_bytes(self.h)
