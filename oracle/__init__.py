"""FP64 CPU oracle of the HS-field HMC for the Ising model (arXiv:1912.03278).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg import this module; the product package never
does.  The arithmetic lives in ``ising_oracle.c`` (plain C, FP64); this file
only compiles it with gcc and marshals numpy arrays through ctypes.

Parity status: every C function is pinned by a CPU test (see the header
``ising_oracle.h`` for which pin covers which function).
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess
from ctypes import POINTER, c_double, c_int, c_int64, c_uint32, c_uint64, c_void_p

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ising_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libising_oracle.so")

FORM_FP64 = 0
FORM_FP32 = 1
PURPOSE_MOM, PURPOSE_ACC, PURPOSE_SPIN, PURPOSE_FLIP, PURPOSE_MH = 1, 2, 3, 4, 5


def build(force: bool = False, extra_flags=()) -> str:
    """Compile the oracle into a shared library next to its source."""
    out = _LIB_PATH if not extra_flags else os.path.join(
        _HERE, "libising_oracle_%s.so"
        % hashlib.sha1(" ".join(extra_flags).encode()).hexdigest()[:8])
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", *extra_flags,
               _SRC, "-o", out, "-lm", "-lpthread"]
        subprocess.check_call(cmd)
    return out


class _Model(ctypes.Structure):
    _fields_ = [("kind", c_int), ("dim", c_int), ("L", c_int * 3), ("N", c_int64),
                ("J", c_void_p), ("Jnn", c_double), ("h", c_void_p), ("h0", c_double),
                ("beta", c_double), ("C", c_double)]


class _Obs(ctypes.Structure):
    _fields_ = [("m", c_double), ("E", c_double), ("abs_m", c_double), ("abs_mt", c_double),
                ("E_cond", c_double)]


class _Chain(ctypes.Structure):
    _fields_ = [("psi", c_void_p), ("S", c_double), ("obs", _Obs), ("traj", c_uint32),
                ("n_meas", c_double), ("n_acc", c_double), ("n_traj", c_double),
                ("sum_m", c_double), ("sum_m2", c_double), ("sum_E", c_double),
                ("sum_E2", c_double), ("sum_am", c_double), ("sum_am2", c_double),
                ("sum_dH", c_double), ("sum_expmdH", c_double), ("sum_Econd", c_double),
                ("sum_amt", c_double)]


class _Rec(ctypes.Structure):
    _fields_ = [("dH", c_double), ("logu", c_double), ("K0", c_double), ("S0", c_double),
                ("K1", c_double), ("S1", c_double), ("accepted", c_int)]


def _load(path=None):
    lib = ctypes.CDLL(path or build())
    P = c_void_p
    sig = {
        "or_philox4x32_10": (None, [P, P, P]),
        "or_u23": (c_double, [c_uint32]),
        "or_u52": (c_double, [c_uint32, c_uint32]),
        "or_momenta": (None, [c_int, c_uint64, c_uint32, c_uint32, c_int64, P]),
        "or_accept_uniform": (c_double, [c_uint64, c_uint32, c_uint32]),
        "or_spin_uniforms": (None, [c_int, c_uint64, c_uint32, c_uint32, c_int64, P]),
        "or_num_sites": (c_int64, [P]),
        "or_neighbors": (None, [P, P]),
        "or_apply_A": (None, [P, P, P]),
        "or_action": (c_double, [P, P, P, P]),
        "or_force": (None, [P, P, P]),
        "or_kinetic": (c_double, [c_int64, P]),
        "or_leapfrog": (None, [P, P, P, c_double, c_int]),
        "or_omelyan": (None, [P, P, P, c_double, c_int, c_double]),
        "or_measure": (None, [P, P, c_int, c_uint64, c_uint32, c_uint32, P]),
        "or_chain_init": (None, [P, P, c_int, c_uint64, c_uint32]),
        "or_trajectory": (None, [P, P, c_int, c_uint64, c_uint32, c_double, c_int, c_int, c_int,
                                 c_int, P, P, P]),
        "or_hmc_run": (None, [P, P, c_int, c_uint64, c_uint32, c_double, c_int, c_int, c_int,
                              c_int64, c_int64, P, P]),
        "or_hmc_run_chains": (None, [P, c_int, c_int, c_uint64, P, P, P, c_int, c_int64, c_int64,
                                     c_int, P]),
        "or_brute_force": (None, [P, P]),
        "or_ring_logZ": (c_double, [c_double, c_double, c_double, c_int64]),
        "or_infinite_range_energy": (c_double, [c_double, c_double, c_double, c_int64]),
        "or_mh_accept_prob": (ctypes.c_float, [c_double, c_double, c_double, c_int, c_int]),
        "or_mh_checkerboard": (None, [P, c_uint64, c_uint32, c_int64, c_int64, c_int64, P, P]),
        "or_mh_run": (None, [P, c_uint64, c_int64, c_int64, P, P]),
        "or_pform_action": (c_double, [P, c_double, P]),
        "or_pform_force": (None, [P, c_double, P, P]),
        "or_pform_leapfrog": (None, [P, c_double, P, P, c_double, c_int]),
        "or_cg_solve": (c_int, [P, P, P, c_double, c_int]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = _load()
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Model:
    """An Ising model in the NS parametrisation A = beta*J*K + C*1.

    kind='lattice': dim, L (tuple), Jnn; kind='dense': J (N x N symmetric).
    h: scalar h0 or per-site array.  The instance keeps its arrays alive for
    the C side.
    """

    def __init__(self, kind="lattice", dim=2, L=(4, 4, 1), Jnn=1.0, J=None, h=0.0, beta=0.44,
                 C=None):
        self.kind = kind
        self.dim = dim
        self.L = tuple(L) + (1,) * (3 - len(L))
        self.Jnn = float(Jnn)
        self.beta = float(beta)
        self._J = None if J is None else _f64(J)
        if np.isscalar(h):
            self._h = None
            self.h0 = float(h)
        else:
            self._h = _f64(h)
            self.h0 = 0.0
        if kind == "dense":
            self.N = self._J.shape[0]
        else:
            self.N = int(np.prod(self.L[:dim]))
        if C is None:
            if kind == "dense":
                lam = np.linalg.eigvalsh(self._J)[0]
                C = self.beta * abs(lam) + 0.1
            else:
                C = self.beta * abs(self.Jnn) * 2 * dim + 0.1
        self.C = float(C)

    @property
    def h(self):
        return np.full(self.N, self.h0) if self._h is None else self._h

    def struct(self, beta=None, C=None):
        m = _Model()
        m.kind = 1 if self.kind == "dense" else 0
        m.dim = self.dim
        for i in range(3):
            m.L[i] = self.L[i]
        m.N = self.N
        m.J = None if self._J is None else self._J.ctypes.data
        m.Jnn = self.Jnn
        m.h = None if self._h is None else self._h.ctypes.data
        m.h0 = self.h0
        m.beta = self.beta if beta is None else beta
        m.C = self.C if C is None else C
        return m

    def with_(self, **kw):
        args = dict(kind=self.kind, dim=self.dim, L=self.L, Jnn=self.Jnn, J=self._J,
                    h=self.h0 if self._h is None else self._h, beta=self.beta, C=self.C)
        args.update(kw)
        return Model(**args)


def philox(ctr, key):
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def u23(x):
    return lib().or_u23(int(x))


def u52(a, b):
    return lib().or_u52(int(a), int(b))


def momenta(form, seed, chain, traj, N):
    p = np.zeros(N)
    lib().or_momenta(form, seed, chain, traj, N, _ptr(p))
    return p


def accept_uniform(seed, chain, traj):
    return lib().or_accept_uniform(seed, chain, traj)


def spin_uniforms(form, seed, chain, traj, N):
    u = np.zeros(N)
    lib().or_spin_uniforms(form, seed, chain, traj, N, _ptr(u))
    return u


def neighbors(model: Model):
    nbr = np.zeros(model.N * 2 * model.dim, dtype=np.int64)
    m = model.struct()
    lib().or_neighbors(ctypes.byref(m), _ptr(nbr))
    return nbr.reshape(model.N, 2 * model.dim)


def apply_A(model: Model, x):
    x = _f64(x)
    y = np.zeros(model.N)
    m = model.struct()
    lib().or_apply_A(ctypes.byref(m), _ptr(x), _ptr(y))
    return y


def action(model: Model, psi, return_at=False):
    psi = _f64(psi)
    a = np.zeros(model.N)
    t = np.zeros(model.N)
    m = model.struct()
    S = lib().or_action(ctypes.byref(m), _ptr(psi), _ptr(a), _ptr(t))
    return (S, a, t) if return_at else S


def force(model: Model, psi):
    psi = _f64(psi)
    F = np.zeros(model.N)
    m = model.struct()
    lib().or_force(ctypes.byref(m), _ptr(psi), _ptr(F))
    return F


def kinetic(p):
    p = _f64(p)
    return lib().or_kinetic(len(p), _ptr(p))


def hamiltonian(model: Model, psi, p):
    return kinetic(p) + action(model, psi)


def leapfrog(model: Model, psi, p, eps, n_md):
    psi = _f64(psi).copy()
    p = _f64(p).copy()
    m = model.struct()
    lib().or_leapfrog(ctypes.byref(m), _ptr(psi), _ptr(p), eps, n_md)
    return psi, p


def omelyan(model: Model, psi, p, eps, n_md, lam=0.1931833275037836):
    psi = _f64(psi).copy()
    p = _f64(p).copy()
    m = model.struct()
    lib().or_omelyan(ctypes.byref(m), _ptr(psi), _ptr(p), eps, n_md, lam)
    return psi, p


def measure(model: Model, psi, form, seed, chain, traj):
    psi = _f64(psi)
    o = _Obs()
    m = model.struct()
    lib().or_measure(ctypes.byref(m), _ptr(psi), form, seed, chain, traj, ctypes.byref(o))
    return dict(m=o.m, E=o.E, abs_m=o.abs_m, abs_mt=o.abs_mt, E_cond=o.E_cond)


class Chain:
    """One HMC Markov chain driven by the oracle (Sec. 3 algorithm)."""

    def __init__(self, model: Model, form=FORM_FP64, seed=0, chain=0, psi0=None):
        self.model = model
        self.form = form
        self.seed = seed
        self.chain = chain
        self._psi = np.zeros(model.N) if psi0 is None else _f64(psi0).copy()
        self._m = model.struct()
        self._c = _Chain()
        self._c.psi = self._psi.ctypes.data
        lib().or_chain_init(ctypes.byref(self._m), ctypes.byref(self._c), form, seed, chain)

    @property
    def psi(self):
        return self._psi.copy()

    @property
    def traj(self):
        return self._c.traj

    @traj.setter
    def traj(self, v):
        self._c.traj = v

    @property
    def S(self):
        return self._c.S

    @property
    def obs(self):
        o = self._c.obs
        return dict(m=o.m, E=o.E, abs_m=o.abs_m, abs_mt=o.abs_mt, E_cond=o.E_cond)

    def trajectory(self, eps, n_md, integrator=0, measure=True, flip_every=0):
        rec = _Rec()
        prop = np.zeros(self.model.N)
        pend = np.zeros(self.model.N)
        lib().or_trajectory(ctypes.byref(self._m), ctypes.byref(self._c), self.form, self.seed,
                            self.chain, eps, n_md, integrator, int(measure), flip_every,
                            ctypes.byref(rec), _ptr(prop), _ptr(pend))
        return dict(dH=rec.dH, logu=rec.logu, K0=rec.K0, S0=rec.S0, K1=rec.K1, S1=rec.S1,
                    accepted=bool(rec.accepted), psi_prop=prop, p_end=pend)

    def run(self, n, eps, n_md, n_therm=0, integrator=0, flip_every=0, records=False,
            series=False):
        recs = (_Rec * n)() if records else None
        ser = np.zeros(n) if series else None
        lib().or_hmc_run(ctypes.byref(self._m), ctypes.byref(self._c), self.form, self.seed,
                         self.chain, eps, n_md, integrator, flip_every, n, n_therm,
                         recs, None if ser is None else _ptr(ser))
        out = {}
        if records:
            out["dH"] = np.array([r.dH for r in recs])
            out["logu"] = np.array([r.logu for r in recs])
            out["accepted"] = np.array([r.accepted for r in recs], dtype=bool)
        if series:
            out["abs_m"] = ser
        return out

    def sums(self):
        c = self._c
        return dict(n_meas=c.n_meas, n_acc=c.n_acc, n_traj=c.n_traj, sum_m=c.sum_m,
                    sum_m2=c.sum_m2, sum_E=c.sum_E, sum_E2=c.sum_E2, sum_am=c.sum_am,
                    sum_am2=c.sum_am2, sum_dH=c.sum_dH, sum_expmdH=c.sum_expmdH,
                    sum_Econd=c.sum_Econd, sum_amt=c.sum_amt)


def run_chains(model: Model, n_chains, form, seed, eps, n_md, n, n_therm=0, beta=None, C=None,
               n_threads=1):
    """Independent chains in POSIX threads; returns an (n_chains, 10) array of sums."""
    eps_a = _f64(np.broadcast_to(eps, (n_chains,)))
    beta_a = None if beta is None else _f64(np.broadcast_to(beta, (n_chains,)))
    C_a = None if C is None else _f64(np.broadcast_to(C, (n_chains,)))
    out = np.zeros((n_chains, 10))
    m = model.struct()
    lib().or_hmc_run_chains(ctypes.byref(m), n_chains, form, seed, _ptr(eps_a),
                            None if beta_a is None else _ptr(beta_a),
                            None if C_a is None else _ptr(C_a), n_md, n, n_therm, n_threads,
                            _ptr(out))
    return out


def brute_force(model: Model):
    out = np.zeros(5)
    m = model.struct()
    lib().or_brute_force(ctypes.byref(m), _ptr(out))
    return dict(logZ=out[0], m=out[1], abs_m=out[2], E=out[3], m2=out[4])


def ring_logZ(beta, J, h, N):
    return lib().or_ring_logZ(beta, J, h, N)


def infinite_range_energy(beta, J, h, N):
    return lib().or_infinite_range_energy(beta, J, h, N)


def mh_run(model: Model, seed, n, n_therm=0, series=False):
    out = np.zeros(6)
    ser = np.zeros(n) if series else None
    m = model.struct()
    lib().or_mh_run(ctypes.byref(m), seed, n, n_therm, _ptr(out),
                    None if ser is None else _ptr(ser))
    res = dict(n_meas=out[0], sum_am=out[1], sum_am2=out[2], sum_E=out[3], sum_E2=out[4],
               acceptance=out[5])
    if series:
        res["abs_m"] = ser
    return res


def mh_checkerboard(model: Model, seed, chain=0, n=1, n_therm=0, spins=None, sweep0=0):
    """Checkerboard local Metropolis-Hastings (Sec. 4 comparator).  Returns the
    spins (int8, starting from `spins` or all +1) and the ISING_SUM_* sums."""
    N = model.N
    s = np.ones(N, dtype=np.int8) if spins is None else np.ascontiguousarray(spins, dtype=np.int8).copy()
    sums = np.zeros(10)
    m = model.struct()
    lib().or_mh_checkerboard(ctypes.byref(m), seed, chain, sweep0, n, n_therm, s.ctypes.data,
                             _ptr(sums))
    return s, sums


def mh_accept_prob(beta, J, h, s, nb):
    return lib().or_mh_accept_prob(beta, J, h, s, nb)


def pform_action(model: Model, Cp, psip):
    psip = _f64(psip)
    m = model.struct()
    return lib().or_pform_action(ctypes.byref(m), Cp, _ptr(psip))


def pform_force(model: Model, Cp, psip):
    psip = _f64(psip)
    F = np.zeros(model.N)
    m = model.struct()
    lib().or_pform_force(ctypes.byref(m), Cp, _ptr(psip), _ptr(F))
    return F


def pform_leapfrog(model: Model, Cp, psip, p, eps, n_md):
    psip = _f64(psip).copy()
    p = _f64(p).copy()
    m = model.struct()
    lib().or_pform_leapfrog(ctypes.byref(m), Cp, _ptr(psip), _ptr(p), eps, n_md)
    return psip, p


def cg_solve(model: Model, b, tol=1e-14, max_iter=10000):
    b = _f64(b)
    x = np.zeros(model.N)
    m = model.struct()
    it = lib().or_cg_solve(ctypes.byref(m), _ptr(b), _ptr(x), tol, max_iter)
    return x, it
