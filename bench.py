"""Throughput benchmark: leapfrog site-steps/s of the HS-field HMC.

Workload (the paper's 2D periodic square lattice, Sec. 4): L = 256 and
L = 1024, nearest-neighbour J = 1, h = 0, beta swept over 16 values in
[0.38, 0.50] with 256 independent chains per beta (4096 chains per L),
C = 4 beta + 0.1, N_md = 20 leapfrog steps, eps tuned per beta for ~80%
acceptance during an untimed equilibration phase.  FP32 state and force, FP64
action, dH and Metropolis test.

One step = one full trajectory (momenta, N_md leapfrog steps, action, dH,
accept, measurement) of every chain of both lattices.  A site-step is one psi
component of one chain advanced one leapfrog step.

Reported next to it: the plain FP64 form (one chain per launch, unfused) on
the same GPU, the dominant kernel's HBM roofline fraction, an end-to-end
number through the public C ABI with host buffers, and the FP64 CPU oracle on
the host cores.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "leapfrog site-steps/s chosen vs plain form, same GPU; %roofline; serve p50/p99"
UNIT = "site-steps/s"
LS = (256, 1024)
N_MD = 20
EPS0 = {256: 0.10, 1024: 0.05}   # tuner start: acceptance at fixed eps falls with N (<dH> ~ N eps^4)
TARGET_ACC = 0.80


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--chains-per-beta", type=int, default=256)
    ap.add_argument("--L", type=str, default="256,1024")
    ap.add_argument("--tune-rounds", type=int, default=6)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-dense", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-integrators", action="store_true")
    ap.add_argument("--no-infinite", action="store_true")
    ap.add_argument("--no-mh", action="store_true")
    ap.add_argument("--no-autocorr", action="store_true")
    ap.add_argument("--serve-seconds", type=float, default=8.0)
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def replica_seed(rank):
    """Seed of rank `rank`'s chains: replicas run independent Markov chains."""
    return 1234 + 7919 * rank


def job_rate(units_local, elapsed_local, ws, device=None):
    """Whole-job throughput of `ws` replicas that each processed `units_local`
    units in `elapsed_local` seconds: all units over the slowest rank's time
    (max over ranks; no collective when ws == 1).  Returns (rate, max time)."""
    elapsed = float(elapsed_local)
    if ws > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([elapsed], dtype=torch.float64,
                         device=device if device is not None else "cpu")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed = float(t.item())
    return units_local * ws / elapsed, elapsed


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = max(smax, float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def measured_peaks_all():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


STAGING_NAMES = {0: "auto", 1: "threads", 2: "bulk"}

TRAFFIC_SOURCES = ("fused_lattice_impl.cuh", "fused_lattice_2d.cu", "df32.cuh",
                   "device_common.cuh", "mbarrier.cuh")


def traffic_source_sha():
    """Hash of the kernel sources a committed traffic figure was measured on."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_1912_03278_gb300", "csrc")
    data = b"".join(open(os.path.join(csrc, f), "rb").read() for f in TRAFFIC_SOURCES)
    return hashlib.sha256(data).hexdigest()[:16]


def traffic_record(kernel, workload, depth=None):
    """DRAM bytes per launch from a committed ncu summary (for the launch's
    ring depth where one was captured), if it matches the current kernel
    source."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
        rec = d.get(kernel, {}).get(workload)
        if rec and rec.get("source_sha") == traffic_source_sha():
            by_depth = rec.get("bytes_per_launch_by_depth", {})
            if depth is not None and str(depth) in by_depth:
                return by_depth[str(depth)]
            return rec.get("bytes_per_launch")
    except (OSError, ValueError):
        pass
    return None


# ---------------------------------------------------------------- reference ----
def cpu_sample_rate(n_threads, L=1024, n_traj=1, seed=5):
    """FP64 oracle, one chain per thread, one trajectory each: site-steps/s."""
    import oracle
    betas = workloads.beta_sweep()
    b = betas[np.arange(n_threads) % len(betas)]
    model = oracle.Model(dim=2, L=(L, L), beta=float(b[0]))
    t0 = time.perf_counter()
    oracle.run_chains(model, n_threads, oracle.FORM_FP32, seed, eps=EPS0.get(L, 0.02), n_md=N_MD,
                      n=n_traj, beta=b, C=workloads.lattice_C(b, 2), n_threads=n_threads)
    dt = time.perf_counter() - t0
    return n_threads * L * L * N_MD * n_traj / dt, dt


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        cpu_sample_rate(cores, L=256)
    t0 = time.perf_counter()
    work = 0.0
    for _ in range(args.steps):
        r, dt = cpu_sample_rate(cores, L=1024)
        work += r * dt
    el = time.perf_counter() - t0
    val = work / el
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "2D periodic square lattice, L=1024 sample of the L=256/1024 "
                               "16-beta x 256-chain batch, N_md=20", "parallelism": "host threads"},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "%d chains (one per core) of L=1024, 1 trajectory each per step"
                                   % cores},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- our arm ----
BETA_C = 0.5 * math.log(1.0 + math.sqrt(2.0))   # Onsager's critical coupling (J = 1)


def onsager_u(beta):
    """Energy per site of the infinite square lattice (J = 1, h = 0), Onsager's
    closed form: u = -coth(2b) [1 + (2/pi)(2 tanh^2(2b) - 1) K(k)], k =
    2 sinh(2b)/cosh^2(2b), K the complete elliptic integral of the first kind."""
    from scipy.special import ellipk
    b2 = 2.0 * beta
    k = 2.0 * math.sinh(b2) / math.cosh(b2) ** 2
    return -(1.0 / math.tanh(b2)) * (1.0 + (2.0 / math.pi) * (2.0 * math.tanh(b2) ** 2 - 1.0)
                                     * float(ellipk(k * k)))


def hot_start(pkg, sims, seed, betas, C, batch=256):
    """Start every chain from spins s = +-1 dressed with the HS field's exact
    conditional fluctuation: given s, phi = A psi ~ N(A s, A) (Sec. 2,
    Eq. did_HS_trafo), i.e. psi = s + A^{-1/2} xi with xi ~ N(0, 1).  Spins
    are drawn at random for beta <= beta_c and all +1 above it (the phase each
    chain equilibrates to, so off-critical chains become stationary within a
    few dozen trajectories).  On the periodic square lattice A = beta J K + C
    is circulant, so A^{-1/2} is applied in Fourier space (eigenvalues
    C + 2 beta J (cos kx + cos ky)).  Set-up only (torch on the device,
    before any timed region)."""
    import torch
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    betas = np.asarray(betas, dtype=np.float64)
    C = np.asarray(C, dtype=np.float64)
    for L, sim in sims.items():
        n_chains = pkg.binding.load().ising_hmc_n_chains(sim.h)
        k = torch.arange(L, device="cuda", dtype=torch.float64) * (2.0 * math.pi / L)
        lam_k = 2.0 * (torch.cos(k)[:, None] + torch.cos(k[: L // 2 + 1])[None, :])
        psi = torch.empty(n_chains, L, L, device="cuda", dtype=torch.float32)
        for c0 in range(0, n_chains, batch):
            c1 = min(n_chains, c0 + batch)
            b = torch.tensor(betas[c0:c1], device="cuda")[:, None, None]
            c = torch.tensor(C[c0:c1], device="cuda")[:, None, None]
            xi = torch.randn(c1 - c0, L, L, device="cuda", generator=g, dtype=torch.float32)
            f = torch.fft.rfft2(xi)
            f *= (c + b * lam_k[None]).rsqrt().to(torch.float32)
            spins = torch.randint(0, 2, (c1 - c0, L, L), device="cuda", generator=g,
                                  dtype=torch.int8).to(torch.float32).mul_(2.0).sub_(1.0)
            ordered = torch.tensor(betas[c0:c1] > BETA_C, device="cuda")[:, None, None]
            spins = torch.where(ordered, torch.ones_like(spins), spins)
            psi[c0:c1] = spins + torch.fft.irfft2(f, s=(L, L))
            del xi, f, spins
        torch.cuda.synchronize()
        pkg.ising_hmc_set_state_native(sim.h, psi.data_ptr(), 0)
        del psi


def tune_eps(sims, betas_per_chain, rounds, seed, therm=6, lo_acc=0.75, hi_acc=0.90, checks=8):
    """Step-size tuning during equilibration only (frozen afterwards).  For a
    second-order integrator the mean energy violation grows as eps^4 and the
    acceptance is erfc(sqrt(<dH>)/2).  Each round runs one trajectory at the
    new step sizes to settle, then estimates the acceptance per beta group
    from the mean of min(1, exp(-dH)) over two more, converts it to an
    effective <dH> and proposes eps * (0.128 / <dH>)^(1/4) (0.128 gives 80%),
    clamped to [0.85, 1] (the chains still relax while the tuner runs and
    their acceptance drifts down, so early readings would push eps up; a
    large step can also push chains into states they leave only slowly: the
    action is not convex); a proposal outside the
    group's bracket of step sizes measured above / below 80% is replaced by
    the bracket's geometric mean.  Last, each group's step is nudged by 8%
    until its measured acceptance lies in [lo_acc, hi_acc] on two checks in a
    row (at most `checks`)."""
    from scipy.special import erfcinv
    target = 4.0 * erfcinv(TARGET_ACC) ** 2
    ub = np.unique(betas_per_chain)
    trace = {}

    def measure(sim, s0, n=2):
        acc = np.zeros(len(betas_per_chain))
        for m in range(n):
            sim.trajectories(1, s0 + m)
            dH = sim.records()[:, 0]
            acc += np.minimum(1.0, np.exp(-np.clip(dH, -50, 50)))
        return acc / n

    for L, sim in sims.items():
        eps = np.full(len(betas_per_chain), EPS0.get(L, 0.05))
        lo = {b: None for b in ub}
        hi = {b: None for b in ub}
        sim.trajectories(therm, seed + 999)
        trace[str(L)] = []
        for r in range(rounds):
            sim.set_eps(eps)
            sim.trajectories(1, seed + 1000 + 10 * r)
            pacc = measure(sim, seed + 1001 + 10 * r)
            trace[str(L)].append(round(float(pacc.mean()), 3))
            for b in ub:
                sel = betas_per_chain == b
                e = float(eps[sel][0])
                a = float(np.clip(pacc[sel].mean(), 1e-3, 1 - 1e-6))
                if a >= TARGET_ACC:
                    lo[b] = e if lo[b] is None else max(lo[b], e)
                else:
                    hi[b] = e if hi[b] is None else min(hi[b], e)
                eff = 4.0 * erfcinv(a) ** 2
                prop = e * float(np.clip((target / eff) ** 0.25, 0.85, 1.0))
                if lo[b] is not None and hi[b] is not None and not lo[b] < prop < hi[b]:
                    prop = math.sqrt(lo[b] * hi[b])
                eps[sel] = prop
        for b in ub:
            sel = betas_per_chain == b
            eps[sel] = lo[b] if lo[b] is not None else 0.9 * hi[b]
        in_band = 0
        for k in range(checks):
            sim.set_eps(eps)
            sim.trajectories(1, seed + 2000 + 10 * k)
            pacc = measure(sim, seed + 2001 + 10 * k)
            trace[str(L)].append(round(float(pacc.mean()), 3))
            done = True
            for b in ub:
                sel = betas_per_chain == b
                a = float(pacc[sel].mean())
                if a < lo_acc:
                    eps[sel] *= 0.92
                    done = False
                elif a > hi_acc:
                    eps[sel] *= 1.08
                    done = False
            in_band = in_band + 1 if done else 0
            if in_band >= 2:
                break
        sim.set_eps(eps)
        sim._eps = eps.copy()
        trace[str(L)].append([round(float(eps.min()), 4), round(float(eps.max()), 4)])
    return trace


def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    import paper_1912_03278_gb300 as pkg
    pkg.build()
    stream = torch.cuda.Stream()
    Ls = tuple(int(x) for x in args.L.split(","))
    betas = np.repeat(workloads.beta_sweep(), args.chains_per_beta)
    n_chains = len(betas)
    C = workloads.lattice_C(betas, 2)
    sims = {}
    for L in Ls:
        sims[L] = pkg.IsingHMC(dim=2, L=(L, L), beta=betas, C=C, eps=EPS0.get(L, 0.02), n_md=N_MD,
                               n_chains=n_chains, precision=pkg.ISING_PREC_FP32,
                               stream=stream.cuda_stream)
    seed = replica_seed(rank)
    # launch shape (threads per CTA, ring depth) per lattice size from the
    # library's autotuner (a temporary handle, before any state is set)
    tuned_launch = {}
    if not args.no_autotune:
        for L in Ls:
            ms = sims[L].autotune(reps=2)
            tuned_launch[str(L)] = dict(zip(("threads", "depth"), sims[L].launch), ms=ms,
                                        staging=STAGING_NAMES[sims[L].staging])
    hot_start(pkg, sims, seed, betas, C)
    tune_trace = tune_eps(sims, betas, args.tune_rounds, seed)
    for L in Ls:
        sims[L].reset_sums()

    def step(k):
        for L in Ls:
            sims[L].trajectories(1, seed)

    for k in range(args.warmup):
        step(k)
    for s in sims.values():
        s.sync()
    big = max(Ls)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    launches0 = sum(s.launches for s in sims.values())
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for k in range(args.steps):
            for L in Ls:
                if L == big:
                    ev[k][0].record(stream)
                sims[L].trajectories(1, seed)
                if L == big:
                    ev[k][1].record(stream)
        t_end.record(stream)
        torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    elapsed = t_start.elapsed_time(t_end) / 1e3
    launches = sum(s.launches for s in sims.values()) - launches0
    big_ms = [a.elapsed_time(b) for a, b in ev]
    obs = {L: sims[L].observables() for L in Ls}
    value, elapsed = job_rate(sum(L * L for L in Ls) * n_chains * N_MD * args.steps, elapsed, ws,
                              device="cuda")

    # dominant kernel: one launch = one trajectory of all chains of the largest lattice
    alg_bytes = 16.0 * N_MD * big * big * n_chains
    dur = float(np.mean(big_ms)) / 1e3
    peak, peak_kind = measured_peaks()
    achieved = alg_bytes / dur / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_kind,
                "traffic": traffic_record("fused_lattice_kernel", "2d_L%d_B%d" % (big, n_chains),
                                          sims[big].launch[1]),
                "kernel": "fused_lattice_kernel", "algorithmic_bytes_per_launch": alg_bytes,
                "ms_per_launch": dur * 1e3}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "2D periodic square lattice L=%s, 16 betas in [0.38,0.50] x %d "
                                   "chains, J=1, h=0, C=4beta+0.1, N_md=%d, eps tuned to ~80%% "
                                   "acceptance; FP32 force and state, FP64 action/dH/accept"
                                   % ("+".join(map(str, Ls)), args.chains_per_beta, N_MD),
                       "global_batch": n_chains * len(Ls) * ws, "parallelism": "replicas",
                       "l2": "inputs larger than L2 (state %.1f GB)"
                             % (16 * sum(L * L for L in Ls) * n_chains / 1e9)},
            "acceptance": {str(L): obs[L]["acceptance"] for L in Ls},
            "tuning": tune_trace,
            "launch_shape": tuned_launch or {str(L): sims[L].launch for L in Ls},
            "roofline": roofline,
            "gpu_launches": int(launches)}

    if rank == 0:
        line["clocks"] = clk.summary()
        if not args.no_plain:
            cmp = {str(L): acceptance_compare(pkg, L, betas, C, sims[L], stream) for L in Ls}
            # plain-form time for one step's work (every chain of every size)
            work = {L: float(L * L) * n_chains * N_MD for L in Ls}
            plain_rate = sum(work.values()) / sum(work[L] / cmp[str(L)]["plain_rate"] for L in Ls)
            line["plain_form"] = {"value": plain_rate, "unit": UNIT, "dtype": "f64",
                                  "by_L": cmp}
            line["speedup_vs_plain"] = value / ws / plain_rate
        if 256 in sims:
            line["onsager"] = onsager_sweep(pkg, stream, sims[256], betas)
        if not args.no_e2e:
            line["e2e"] = e2e_rate(pkg, sims, Ls, n_chains, seed, stream)
        if not args.no_integrators:
            line["integrators"] = integrator_compare(pkg, sims[big], betas, stream, L=big)
    for s in sims.values():
        s.close()
    sims = {}
    if rank == 0:
        if not args.no_mixed:
            line["mixed_3d"] = mixed_3d_rate(pkg)
        if not args.no_dense:
            line["dense"] = dense_rate(pkg, stream)
        if not args.no_infinite:
            line["infinite"] = infinite_rate(pkg, stream)
        if not args.no_mh:
            line["mh"] = mh_rate(pkg, stream, big, betas, float(np.mean(big_ms)))
        if not args.no_autocorr:
            line["autocorr"] = autocorr_run(pkg, stream)
        if not args.no_serve:
            line["serve"] = serve_run(pkg, args.serve_seconds)
        if not args.no_cpu:
            import oracle
            oracle.build()
            cores = os.cpu_count() or 1
            r, dt = cpu_sample_rate(cores, L=big)
            line["cpu_baseline"] = {"value": r, "unit": UNIT, "cores": cores, "kind": "oracle",
                                    "sample": "%d chains of L=%d (one per core), 1 trajectory, "
                                              "N_md=%d, %.1f s" % (cores, big, N_MD, dt)}
        line["summary"] = summary(line)
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def summary(line):
    """The headline comparisons in a few numbers, emitted as the line's last key
    (so that a truncated copy of the line still carries them)."""
    def g(*path):
        d = line
        for p in path:
            if not isinstance(d, dict) or p not in d:
                return None
            d = d[p]
        return round(d, 4) if isinstance(d, float) else d
    out = {"speedup_vs_plain": g("speedup_vs_plain"), "stencil_frac": g("roofline", "frac")}
    for L in LS:
        c = g("plain_form", "by_L", str(L))
        if c:
            out["acc_L%d" % L] = {"chosen": g("plain_form", "by_L", str(L), "chosen", "acceptance"),
                                  "plain": g("plain_form", "by_L", str(L), "plain", "acceptance"),
                                  "diff": g("plain_form", "by_L", str(L), "acc_diff"),
                                  "err": g("plain_form", "by_L", str(L), "acc_diff_err"),
                                  "within_2pct": c.get("within_2pct"),
                                  "creutz_ok": c.get("stationary_creutz_3sigma")}
    out["onsager_L256_max_dev_sigma"] = g("onsager", "max_abs_dev_sigma_off_critical")
    out["onsager_L256_pass"] = g("onsager", "pass_3sigma_off_critical")
    out["mixed_3d_frac"] = g("mixed_3d", "roofline", "frac")
    out["dense_bf16_frac"] = g("dense", "roofline", "frac")
    for f in ("bf16", "fp8"):
        d = g("dense", "precision_error", f + "_minus_fp64")
        if d:
            out["dense_%s_minus_fp64_sigma" % f] = {k: round(d[k]["sigma"], 2)
                                                    for k in ("m", "E", "abs_m")}
    out["mh_frac"] = g("mh", "roofline", "frac")
    out["t_hmc_over_t_mh"] = g("mh", "t_hmc_over_t_mh")
    out["infinite_resident_frac"] = g("infinite", "resident", "roofline", "frac")
    out["serve_p50_p99_s"] = [g("serve", "p50_s"), g("serve", "p99_s")]
    out["serve_queue_end_by_rho"] = {k: v.get("queued_at_end_of_arrivals")
                                     for k, v in (g("serve", "by_rho") or {}).items()}
    out["serve_served_over_rho_cap"] = {k: round(v.get("served_over_rho_capacity", 0), 3)
                                        for k, v in (g("serve", "by_rho") or {}).items()}
    return out


def _pick_stationary(betas, per_group, groups=4):
    """Chains of the `groups` beta values farthest from beta_c (two on each
    side), `per_group` of each: chains that become stationary within a few
    dozen trajectories (correlation lengths of a few sites)."""
    ub = np.unique(betas)
    far = list(ub[:groups // 2]) + list(ub[-(groups // 2):])
    idx = np.concatenate([np.flatnonzero(betas == b)[:per_group] for b in far])
    return idx, [float(b) for b in far]


def _arm_stats(sums, n_traj, k):
    """Acceptance (binomial error over chain-trajectories) and Creutz's
    <exp(-dH)> (standard error of the per-chain means) from chain sums."""
    n_meas = sums[:, 0]
    acc = float(sums[:, 1].sum() / n_meas.sum())
    e_chain = sums[:, 9] / n_meas
    return {"acceptance": acc, "acceptance_err": math.sqrt(acc * (1 - acc) / (k * n_traj)),
            "mean_exp_mdH": float(e_chain.mean()),
            "exp_mdH_err": float(e_chain.std(ddof=1) / math.sqrt(k)),
            "mean_dH": float(sums[:, 8].sum() / n_meas.sum())}


def acceptance_compare(pkg, L, betas, C, tuned, stream, per_group=32, therm=100, n=32, seed=77):
    """The metric's condition: the chosen form (FP32 fused, batched) and the
    plain form (FP64 state and force, one chain per launch, unfused) at equal
    acceptance within 2%.  Chains of the four beta values farthest from beta_c
    (per_group each) are copied from the tuned handle, thermalised for `therm`
    more trajectories in the chosen form at their tuned eps, and from that
    common snapshot both forms run `n` trajectories at the same eps and N_md
    with the same seed and trajectory indices (their momenta come from the
    same Philox draws, rounded differently).  Per arm: acceptance with its
    binomial error over all chain-trajectories (>= 4096), Creutz's
    <exp(-dH)> = 1 as the stationarity check.  The plain arm's n
    trajectories are timed with CUDA events: its site-steps/s."""
    import torch
    idx, far = _pick_stationary(betas, per_group)
    k = len(idx)
    eps = np.asarray(tuned._eps, dtype=np.float64)[idx]
    n_all = pkg.binding.load().ising_hmc_n_chains(tuned.h)
    full = torch.empty(n_all, L * L, device="cuda", dtype=torch.float32)
    pkg.ising_hmc_get_state_native(tuned.h, full.data_ptr())
    start = full[torch.as_tensor(idx, device="cuda")].contiguous()
    del full
    kw = dict(dim=2, L=(L, L), beta=betas[idx], C=C[idx], eps=eps, n_md=N_MD, n_chains=k,
              stream=stream.cuda_stream)
    t0_idx = 5 * 10 ** 6
    chosen = pkg.IsingHMC(precision=pkg.ISING_PREC_FP32, **kw)
    try:
        torch.cuda.synchronize()
        pkg.ising_hmc_set_state_native(chosen.h, start.data_ptr(), t0_idx - therm)
        chosen.trajectories(therm, seed + 1)
        snap = chosen.state(pkg.ISING_STATE_PSI)
        chosen.reset_sums()
        chosen.trajectories(n, seed)
        a_chosen = _arm_stats(chosen.chain_sums(), n, k)
    finally:
        chosen.close()
    del start
    plain = pkg.IsingHMC(precision=pkg.ISING_PREC_PLAIN_FP64, **kw)
    try:
        plain.set_state(snap, next_traj=t0_idx)
        plain.reset_sums()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = plain.launches
        e0.record(stream)
        plain.trajectories(n, seed)
        e1.record(stream)
        torch.cuda.synchronize()
        dt = e0.elapsed_time(e1) / 1e3
        launches = plain.launches - l0
        a_plain = _arm_stats(plain.chain_sums(), n, k)
    finally:
        plain.close()
    d = a_chosen["acceptance"] - a_plain["acceptance"]
    d_err = math.hypot(a_chosen["acceptance_err"], a_plain["acceptance_err"])
    stationary = all(abs(a["mean_exp_mdH"] - 1.0) <= 3.0 * a["exp_mdH_err"]
                     for a in (a_chosen, a_plain))
    return {"L": L, "betas": far, "chains": k, "trajectories_per_chain": n,
            "chain_trajectories_per_arm": k * n, "therm_before": therm,
            "chosen": a_chosen, "plain": a_plain, "acc_diff": d, "acc_diff_err": d_err,
            "within_2pct": bool(abs(d) < 0.02), "stationary_creutz_3sigma": bool(stationary),
            "plain_rate": k * L * L * N_MD * n / dt, "plain_launches": int(launches),
            "plain_dtype": "f64"}


def onsager_sweep(pkg, stream, tuned, betas_tuned, L=256, per_beta=32, therm=1500, n=1000,
                  seed=83):
    """Sec. 4 / Fig. 1 on the headline lattice: E/beta, the energy per site, for
    the 16 betas of the sweep against Onsager's infinite-lattice u(beta).
    per_beta chains per beta at that beta's tuned eps (taken from the tuned
    handle), started in the phase they equilibrate to, `therm` trajectories
    discarded and `n` measured; the error is the standard error of the chain
    means.  Betas within 0.02 of beta_c are marked critical: their
    correlation length and relaxation time grow with L (finite-size shifts,
    tau ~ L^z) and they are not part of the pass test; elsewhere xi << L and
    the lattice result equals u(beta) within its error."""
    ub = np.unique(betas_tuned)
    eps_t = np.asarray(tuned._eps, dtype=np.float64)
    eps_b = {b: float(eps_t[betas_tuned == b].mean()) for b in ub}
    betas = np.repeat(ub, per_beta)
    C = workloads.lattice_C(betas, 2)
    sim = pkg.IsingHMC(dim=2, L=(L, L), beta=betas, C=C,
                       eps=np.array([eps_b[b] for b in betas]), n_md=N_MD,
                       n_chains=len(betas), n_therm=therm, stream=stream.cuda_stream)
    try:
        hot_start(pkg, {L: sim}, seed, betas, C)
        sim.trajectories(therm + n, seed)
        sums = sim.chain_sums()
    finally:
        sim.close()
    rows, worst = {}, 0.0
    for b in ub:
        sel = betas == b
        nm = np.maximum(sums[sel, 0], 1)
        e = sums[sel, 4] / nm / b
        m, err = float(e.mean()), float(e.std(ddof=1) / math.sqrt(sel.sum()))
        u = onsager_u(float(b))
        crit = abs(b - BETA_C) < 0.02
        dev = (m - u) / max(err, 1e-300)
        rows["%.4f" % b] = {"E_per_site": m, "err": err, "onsager_u": u, "dev_sigma": dev,
                            "acceptance": float(sums[sel, 1].sum() / nm.sum()),
                            "critical": bool(crit)}
        if not crit:
            worst = max(worst, abs(dev))
    return {"L": L, "chains_per_beta": per_beta, "therm": therm, "measured": n,
            "by_beta": rows, "max_abs_dev_sigma_off_critical": worst,
            "pass_3sigma_off_critical": bool(worst <= 3.0)}


def _dense_tuned_run(pkg, J, hv, beta, C, B, n_md, prec, stream, steps, seed, tune_rounds, n_force):
    """Tune eps towards ~85% acceptance, then time `steps` trajectories and,
    separately, `n_force` force evaluations with CUDA events on the stream."""
    import torch
    sim = pkg.IsingHMC(kind="dense", J=J, h=hv, beta=beta, C=C, eps=0.05, n_md=n_md, n_chains=B,
                       precision=prec, stream=stream.cuda_stream)
    try:
        C_used = float(sim.params[0, 1])   # the library's default shift when C is None
        eps = 0.05
        trace = []
        sim.trajectories(4, seed)
        for _ in range(tune_rounds):
            sim.trajectories(2, seed)
            acc = float(sim.records()[:, 2].mean())
            trace.append((round(eps, 5), round(acc, 3)))
            eps *= 1.35 if acc > 0.93 else 1.12 if acc > 0.85 else 0.75 if acc < 0.6 else \
                0.92 if acc < 0.75 else 1.0
            sim.set_eps(np.full(B, eps))
        sim.trajectories(2, seed)
        sim.reset_sums()
        torch.cuda.synchronize()
        l0 = sim.launches
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.trajectories(steps, seed)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_traj = e0.elapsed_time(e1) / steps
        launches = sim.launches - l0
        obs = sim.observables()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        sim.dense_forces(2)
        f0.record(stream)
        sim.dense_forces(n_force)
        f1.record(stream)
        torch.cuda.synchronize()
        ms_force = f0.elapsed_time(f1) / n_force
    finally:
        sim.close()
    return dict(ms_traj=ms_traj, launches=launches, acc=obs["acceptance"], eps=eps, trace=trace,
                ms_force=ms_force, C=C_used)


def dense_rate(pkg, stream, steps=4, n_md=10, seed=77, tune_rounds=6, n_force=10):
    """Dense all-to-all couplings: SK model N = 4096, J_ij ~ N(0, 1/N) symmetric
    with J_ii = 0, h_i ~ N(0, 0.1^2), beta = 0.5, C = beta |lambda_min(J)| + 0.1,
    1024 chains, BF16 tensor-core force with FP32 state, FP64-accurate action
    (exact digit-sliced tensor-core product), N_md = 10, eps tuned towards 85%
    acceptance.  Times whole trajectories and, separately, force evaluations
    (two 4096 x 4096 x 1024 GEMMs each), both with CUDA events on the
    handle's stream.  The FP8 (E4M3) force variant is measured the same way
    (key `fp8`, its own tuned eps)."""
    import torch
    N, B, beta = 4096, 1024, 0.5
    J = workloads.dense_couplings(N, seed=1)
    hv = workloads.dense_fields(N, 0.1, seed=2)
    # C = beta |lambda_min(J)| + 0.1, chosen by the library (Lanczos) and reused
    r = _dense_tuned_run(pkg, J, hv, beta, None, B, n_md, pkg.ISING_PREC_BF16, stream, steps, seed,
                         tune_rounds, n_force)
    C = r["C"]
    flops_force = 2 * 2.0 * N * N * B
    peaks = measured_peaks_all()
    peak = peaks.get("bf16_tflops") or 1900.0
    src = "measured bf16 burst (MEASURED_PEAKS.json)" if peaks.get("bf16_tflops") else "fallback"
    tf = flops_force / (r["ms_force"] * 1e-3) / 1e12
    out = {"workload": "dense SK couplings N=%d, J~N(0,1/N), h~N(0,0.01), beta=%g, "
                       "C=beta|lambda_min|+0.1=%.4f, %d chains, N_md=%d, eps tuned"
                       % (N, beta, C, B, n_md),
           "value": N * B * n_md / (r["ms_traj"] * 1e-3), "unit": UNIT,
           "ms_per_trajectory": r["ms_traj"], "acceptance": r["acc"], "eps": r["eps"],
           "tuning": r["trace"], "gpu_launches_per_trajectory": r["launches"] / steps,
           "fixed_ms_per_trajectory": r["ms_traj"] - (n_md + 1) * r["ms_force"],
           "roofline": {"bound": "tensor", "achieved": tf, "peak": peak, "unit": "TFLOP/s",
                        "frac": tf / peak, "peak_source": src,
                        "kernel": "force1_kernel + force2_kernel (one force evaluation)",
                        "algorithmic_flops_per_force": flops_force, "ms_per_force": r["ms_force"]}}
    r8 = _dense_tuned_run(pkg, J, hv, beta, C, B, n_md, pkg.ISING_PREC_FP8, stream, steps, seed,
                          tune_rounds, n_force)
    tf8 = flops_force / (r8["ms_force"] * 1e-3) / 1e12
    out["fp8"] = {"value": N * B * n_md / (r8["ms_traj"] * 1e-3), "unit": UNIT,
                  "ms_per_trajectory": r8["ms_traj"], "acceptance": r8["acc"], "eps": r8["eps"],
                  "tuning": r8["trace"],
                  "roofline": {"bound": "tensor", "achieved": tf8, "peak": 2.0 * peak,
                               "unit": "TFLOP/s", "frac": tf8 / (2.0 * peak),
                               "peak_source": "measured bf16 burst x 2 (nominal FP8:BF16 ratio)",
                               "kernel": "force1_kernel + force2_kernel, E4M3 operands",
                               "ms_per_force": r8["ms_force"]}}
    eps = r["eps"]
    out["precision_error"] = dense_precision(pkg, J, hv, beta, C, eps, n_md, stream)
    # plain one-chain-per-launch FP64 form on a few chains of the same model
    try:
        k = 2
        pl = pkg.IsingHMC(kind="dense", J=J, h=hv, beta=beta, C=C, eps=eps, n_md=n_md, n_chains=k,
                          precision=pkg.ISING_PREC_PLAIN_FP64, stream=stream.cuda_stream)
        pl.trajectories(1, seed)
        torch.cuda.synchronize()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        pl.trajectories(1, seed)
        p1.record(stream)
        torch.cuda.synchronize()
        rate = N * k * n_md / (p0.elapsed_time(p1) * 1e-3)
        pl.close()
        out["plain_form"] = {"value": rate, "unit": UNIT, "chains": k}
        out["speedup_vs_plain"] = out["value"] / rate
    except Exception as e:   # report, do not hide
        out["plain_form"] = {"error": str(e)}
    return out


def _chain_means(sums):
    """Per-observable mean over chains of the per-chain averages, with the
    standard error of those chain means."""
    n = np.maximum(sums[:, 0], 1)
    out = {}
    for name, col in (("m", 2), ("E", 4), ("abs_m", 6)):
        v = sums[:, col] / n
        out[name] = (float(v.mean()), float(v.std(ddof=1) / math.sqrt(len(v))))
    out["acceptance"] = (float(sums[:, 1].sum() / n.sum()), 0.0)
    return out


def dense_precision(pkg, J, hv, beta, C, eps, n_md, stream, therm=10, n=30, seed=91):
    """Chosen-precision error against FP64, per observable, on the dense SK
    workload: the BF16 and FP8 tensor-core forms (256 chains each) and the plain
    FP64 form (128 chains), all at the same eps and N_md, started at psi = 0,
    `therm` trajectories discarded, `n` measured.  A deterministic reversible
    force keeps HMC exact, so each difference should be zero within its
    combined standard error; the acceptance shows what the precision costs."""
    forms = (("bf16", pkg.ISING_PREC_BF16, 256), ("fp8", pkg.ISING_PREC_FP8, 256),
             ("fp64", pkg.ISING_PREC_PLAIN_FP64, 128))
    res = {}
    for name, prec, B in forms:
        sim = pkg.IsingHMC(kind="dense", J=J, h=hv, beta=beta, C=C, eps=eps, n_md=n_md,
                           n_chains=B, n_therm=therm, precision=prec, stream=stream.cuda_stream)
        try:
            sim.trajectories(therm + n, seed)
            res[name] = _chain_means(sim.chain_sums())
        finally:
            sim.close()
    out = {"eps": eps, "n_md": n_md, "therm": therm, "measured": n,
           "chains": {name: B for name, _, B in forms}}
    for name in ("bf16", "fp8", "fp64"):
        out[name] = {k: {"value": v[0], "err": v[1]} for k, v in res[name].items()}
    for name in ("bf16", "fp8"):
        d = {}
        for k in ("m", "E", "abs_m"):
            diff = res[name][k][0] - res["fp64"][k][0]
            err = math.hypot(res[name][k][1], res["fp64"][k][1])
            d[k] = {"diff": diff, "err": err, "sigma": diff / max(err, 1e-300)}
        d["acceptance_diff"] = res[name]["acceptance"][0] - res["fp64"]["acceptance"][0]
        out[name + "_minus_fp64"] = d
    return out


def integrator_compare(pkg, tuned, betas, stream, L=1024, per_beta=19, therm=4, steps=6, seed=55):
    """Omelyan's second-order minimum-norm integrator against KDK leapfrog at
    equal cost and equal trajectory length: 21 force evaluations each
    (leapfrog N_md = 20 at each chain's tuned eps, Omelyan N_md = 10 at twice
    it), both started from the same equilibrated configurations (the first
    per_beta chains of every beta of the tuned handle, copied on the device);
    acceptance, <dH> and time per trajectory (CUDA events)."""
    import torch
    n_all = pkg.binding.load().ising_hmc_n_chains(tuned.h)
    per_block = n_all // len(np.unique(betas))
    idx = np.concatenate([np.arange(b * per_block, b * per_block + per_beta)
                          for b in range(n_all // per_block)])
    full = torch.empty(n_all, L * L, device="cuda", dtype=torch.float32)
    pkg.ising_hmc_get_state_native(tuned.h, full.data_ptr())
    start = full[torch.as_tensor(idx, device="cuda")].contiguous()
    del full
    bsub = betas[idx]
    C = workloads.lattice_C(bsub, 2)
    eps = np.asarray(tuned._eps, dtype=np.float64)[idx]
    out = {}
    for name, integ, n_md, e in (("leapfrog", pkg.ISING_INTEGRATOR_LEAPFROG, N_MD, eps),
                                 ("omelyan", pkg.ISING_INTEGRATOR_OMELYAN, N_MD // 2, 2 * eps)):
        sim = pkg.IsingHMC(dim=2, L=(L, L), beta=bsub, C=C, eps=e, n_md=n_md, n_chains=len(bsub),
                           precision=pkg.ISING_PREC_FP32, integrator=integ,
                           stream=stream.cuda_stream)
        try:
            torch.cuda.synchronize()
            pkg.ising_hmc_set_state_native(sim.h, start.data_ptr(), 0)
            sim.trajectories(therm, seed)
            sim.reset_sums()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sim.trajectories(steps, seed)
            e1.record(stream)
            torch.cuda.synchronize()
            obs = sim.observables()
            out[name] = {"n_md": n_md, "force_evaluations": n_md + 1 if integ == 0 else 2 * n_md + 1,
                         "ms_per_trajectory": e0.elapsed_time(e1) / steps,
                         "acceptance": obs["acceptance"], "mean_dH": obs["mean_dH"],
                         "mean_exp_mdH": obs["mean_exp_mdH"]}
        finally:
            sim.close()
    del start
    out["chains"] = int(len(bsub))
    out["L"] = L
    out["start"] = "equilibrated configurations of the tuned handle; %d trajectories before " \
                   "measuring, %d measured" % (therm, steps)
    return out


# FP32-pipe operations per site and force evaluation of the resident
# infinite-range kernel, counted from its source: tanh argument and tanh 12,
# u 1, F 3, kick 1, drift 1, quad sums and double-float accumulation 4.5
INF_OPS_PER_SITE_PASS = 22.5


def infinite_rate(pkg, stream, steps=4, therm=20, seed=41):
    """Infinite-range (all-to-all) model of the appendix at the critical
    coupling beta*J = 1, h = 0, C = 1 (A's spectrum in [1, 2]), N_md =
    floor(ln N), in both kernel variants: N = 4096 (chain resident in
    registers; bound by the FP32 pipe) and N = 65536 (streaming; bound by HBM
    at 16 algorithmic bytes per site-step: psi and p read, p and psi'
    written).  eps starts at 1/N_md (unit trajectory length) and is moved,
    during thermalisation only and never above 1/N_md, into the 75-90%
    acceptance band where that start falls short (erfc(sqrt(<dH>)/2)
    acceptance model, eps^4 scaling of <dH>; the larger N, the larger <dH> at
    a given eps).  Site-steps/s and time
    per trajectory from CUDA events, one launch per trajectory."""
    import torch
    from scipy.special import erfcinv
    target = 4.0 * erfcinv(TARGET_ACC) ** 2
    out = {}
    for name, N, n_chains in (("resident", 4096, 152 * 32), ("streaming", 65536, 152 * 4)):
        n_md = workloads.n_md_default(N)
        eps = 1.0 / n_md
        sim = pkg.IsingHMC(kind="infinite", n_sites=N, beta=1.0, C=1.0, eps=eps,
                           n_md=n_md, n_chains=n_chains, precision=pkg.ISING_PREC_FP32,
                           stream=stream.cuda_stream)
        try:
            sim.trajectories(therm // 2, seed)
            for r in range(4):
                acc = 0.0
                for m in range(2):
                    sim.trajectories(1, seed + 100 + 10 * r + m)
                    dH = sim.records()[:, 0]
                    acc += float(np.minimum(1.0, np.exp(-np.clip(dH, -50, 50))).mean()) / 2
                if 0.75 <= acc <= 0.90 or (acc > 0.90 and eps >= 1.0 / n_md):
                    break
                eff = 4.0 * erfcinv(float(np.clip(acc, 1e-3, 1 - 1e-6))) ** 2
                eps = min(1.0 / n_md, eps * float(np.clip((target / eff) ** 0.25, 0.5, 1.5)))
                sim.set_eps(np.full(n_chains, eps))
            sim.trajectories(therm // 2, seed + 1)
            sim.reset_sums()
            torch.cuda.synchronize()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(steps)]
            l0 = sim.launches
            for k in range(steps):
                ev[k][0].record(stream)
                sim.trajectories(1, seed)
                ev[k][1].record(stream)
            torch.cuda.synchronize()
            ms = [a.elapsed_time(b) for a, b in ev]
            obs = sim.observables()
            launches = int(sim.launches - l0)
        finally:
            sim.close()
        dur = float(np.mean(ms)) / 1e3
        site_steps = float(N) * n_chains * n_md
        r = {"workload": "all-to-all N=%d, %d chains, beta*J=1, h=0, C=1, N_md=%d, eps=%.4f "
                         "(1/N_md = %.4f; tuned toward 80%% acceptance during thermalisation)"
                         % (N, n_chains, n_md, eps, 1.0 / n_md),
             "value": site_steps / dur, "unit": UNIT, "ms_per_trajectory": dur * 1e3,
             "launches": launches, "acceptance": obs["acceptance"],
             "E": obs["E"], "E_err": obs["E_err"]}
        if name == "resident":
            # FP32 lanes x SM clock: 152 SMs x 128 lanes x 2.07 GHz
            ops = INF_OPS_PER_SITE_PASS * float(N) * n_chains * (n_md + 1) / dur / 1e9
            peak = 152 * 128 * 2.07
            r["roofline"] = {"bound": "alu", "achieved": ops, "peak": peak, "unit": "Gop/s",
                             "frac": ops / peak, "peak_source": "derived (FP32 lanes x max clock)",
                             "kernel": "infinite_kernel<resident>",
                             "ops_per_site_pass": INF_OPS_PER_SITE_PASS}
        else:
            peak, peak_kind = measured_peaks()
            achieved = 16.0 * site_steps / dur / 1e9
            r["roofline"] = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak, "peak_source": peak_kind,
                             "kernel": "infinite_kernel<streaming>",
                             "algorithmic_bytes_per_launch": 16.0 * site_steps}
        out[name] = r
    return out


def mh_rate(pkg, stream, L, betas, hmc_ms, steps=4, warm=2, seed=61):
    """The Sec. 4 comparator on the same batch as the headline step (2D L x L,
    the same chains and betas, h = 0): checkerboard Metropolis-Hastings sweeps
    timed with CUDA events, and the cost ratio T_HMC / T_MH (the paper reports
    ~4 N_step for its implementation).  L = 1024 rows take the multi-spin-
    coded kernel, which is bound by the ALU pipe, not by HBM (0.25 B of spins
    per site and sweep): its roofline is the ALU-pipe saturation rate; the
    HBM fraction at 2 B per site-sweep (int8 spins) is kept for comparison
    with the byte kernels."""
    import torch
    n = len(betas)
    sim = pkg.IsingMH(dim=2, L=(L, L), beta=betas, n_chains=n, stream=stream.cuda_stream)
    try:
        sim.sweeps(warm, seed)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = sim.launches
        e0.record(stream)
        sim.sweeps(steps, seed)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        launches = int(sim.launches - l0)
        acc = sim.observables()["acceptance"]
    finally:
        sim.close()
    sites = float(L) * L * n
    peak, peak_kind = measured_peaks()
    achieved = 2.0 * sites / (ms / 1e3) / 1e9
    # the packed kernel is bound by the ALU pipe (Philox and bit logic): peak =
    # the decision rate at which that pipe would be saturated, from the ncu
    # capture of one colour launch of 2048 chains at L = 1024 (1.0737e9
    # decisions in 1.564 ms with the ALU pipe 68.86% busy)
    alu_peak = 1.0737e9 / 1.564e-3 / 0.6886
    return {"workload": "2D L=%d, %d chains (16 betas in [0.38, 0.50]), J=1, h=0, checkerboard, "
                        "spins start +1, %d warm-up sweeps" % (L, n, warm),
            "value": sites / (ms / 1e3), "unit": "site-updates/s", "ms_per_sweep": ms,
            "launches_per_sweep": launches / steps, "flip_fraction": acc,
            "t_hmc_over_t_mh": hmc_ms / ms, "n_step": N_MD, "paper_4_n_step": 4 * N_MD,
            "roofline": {"bound": "alu", "achieved": sites / (ms / 1e3), "peak": alu_peak,
                         "unit": "site-updates/s", "frac": sites / (ms / 1e3) / alu_peak,
                         "peak_source": "derived: ALU-pipe saturation rate from the ncu counters "
                                        "(profiles/mh_packed_kernel_2d_L1024.md)",
                         "kernel": "mh_packed_kernel (both colours + measurement)",
                         "hbm_fraction_at_2_bytes_per_site_sweep": achieved / peak}}


def _tau_abs_m(pkg, stream, L, C_over_beta, n_chains, therm, n, seed):
    """tau_int of |m| (Gamma method over the chains' device-recorded series) of
    the 2D lattice at the critical coupling, N_md = floor(ln N), unit
    trajectory length in the paper's units (eps = 1 / (N_md sqrt(beta)))."""
    beta = math.log(1 + math.sqrt(2)) / 2
    n_md = workloads.n_md_default(L * L)
    sim = pkg.IsingHMC(dim=2, L=(L, L), beta=beta, C=C_over_beta * beta,
                       eps=1.0 / (n_md * math.sqrt(beta)), n_md=n_md, n_chains=n_chains,
                       stream=stream.cuda_stream)
    try:
        sim.trajectories(therm, seed)
        sim.series_enable(n)
        sim.trajectories(n, seed)
        ser = sim.series()
        acc = sim.observables()["acceptance"]
    finally:
        sim.close()
    r = pkg.binding.ising_gamma_method(ser[:, :, 2])
    return {"tau_int": r["tau_int"], "tau_err": r["tau_err"], "abs_m": r["mean"],
            "abs_m_err": r["err"], "acceptance": acc, "n_md": n_md}


def autocorr_run(pkg, stream, n_chains=128, therm=200, n=1500, seed=71):
    """Sec. 4, Fig. 2 and Fig. 3 on synthetic chains: tau_int of |m| at beta_c
    for L = 8, 16, 32 (C = 5 beta, i.e. the paper's C_p = n + 1 with n = 4
    neighbours) and the dynamic exponent from a log-log fit; and a scan of the
    shift at L = 15, C_p - n in {0.1, 0.5, 1, 2, 4}."""
    import time as _t
    t0 = _t.perf_counter()
    sizes = {}
    for L in (8, 16, 32):
        sizes[str(L)] = _tau_abs_m(pkg, stream, L, 5.0, n_chains, therm, n, seed)
    Ls = np.array([8.0, 16.0, 32.0])
    taus = np.array([sizes[str(int(L))]["tau_int"] for L in Ls])
    z = float(np.polyfit(np.log(Ls), np.log(taus), 1)[0])
    scan = {}
    for dc in (0.1, 0.5, 1.0, 2.0, 4.0):
        scan[str(dc)] = _tau_abs_m(pkg, stream, 15, 4.0 + dc, n_chains, therm, n, seed)
    best = min(scan, key=lambda k: scan[k]["tau_int"])
    return {"workload": "2D periodic lattice at beta_c, h = 0, %d chains, %d trajectories "
                        "recorded after %d" % (n_chains, n, therm),
            "tau_abs_m_by_L": sizes, "z_fit": z, "c_scan_L15": scan, "c_p_minus_n_best": float(best),
            "seconds": _t.perf_counter() - t0}


def mixed_3d_rate(pkg, steps=4, seed=31):
    """3D simple-cubic lattices L in {16,24,32,48,64}, 64 chains each, J=1,
    h=0.05, beta=0.2217, C=6 beta+0.1, N_md=floor(ln N), eps=1/(N_md sqrt(beta))
    (unit trajectory length in the paper's units): one CUDA-graph launch per
    step for all five sizes; each size's launch shape from the autotuner, the
    CTAs per chain from the group autotuner (the whole launch timed)."""
    import torch
    beta = 0.2217
    sims = []
    for L in (16, 24, 32, 48, 64):
        n_md = workloads.n_md_default(L ** 3)
        sims.append(pkg.IsingHMC(dim=3, L=(L, L, L), beta=beta, h=0.05, C=6 * beta + 0.1,
                                 eps=1.0 / (n_md * math.sqrt(beta)), n_md=n_md, n_chains=64))
    tuned = {}
    for s in sims:
        ms = s.autotune(reps=1)
        tuned[s.kw["L"][0]] = dict(zip(("threads", "depth"), s.launch), ms_alone=ms)
    grp = pkg.IsingGroup(sims)
    try:
        # the members' chain splits (CTAs per chain) for the whole group's launch
        group_ms = grp.autotune(reps=4)
        for s in sims:
            tuned[s.kw["L"][0]]["ctas_per_chain"] = s.chain_split
            tuned[s.kw["L"][0]]["staging"] = STAGING_NAMES[s.staging]
        grp.trajectories(2, seed)
        grp.sync()
        gs = torch.cuda.ExternalStream(grp.stream)
        l0 = grp.launches
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(gs)
        grp.trajectories(steps, seed)
        e1.record(gs)
        grp.sync()
        torch.cuda.synchronize()
        dt = e0.elapsed_time(e1) / 1e3
        work = sum(s.kw["L"][0] ** 3 * 64 * s.kw["n_md"] for s in sims) * steps
        acc = [s.observables()["acceptance"] for s in sims]
        peak, peak_kind = measured_peaks()
        achieved = 16.0 * work / dt / 1e9
        return {"value": work / dt, "unit": UNIT, "graph_launches": grp.launches - l0,
                "steps": steps, "ms_per_step": dt * 1e3 / steps,
                "sites": sum(s.kw["L"][0] ** 3 * 64 for s in sims),
                "tuned_launch": tuned, "group_autotune_ms": group_ms, "acceptance": acc,
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak, "peak_source": peak_kind,
                             "kernel": "group graph (fused_lattice_kernel, five sizes)",
                             "algorithmic_bytes_per_step": 16.0 * work / steps}}
    finally:
        grp.close()
        for s in sims:
            s.close()


_DENSE_POOL = {}


def dense_model(n):
    """SK couplings of size n for serving requests (a small pool of models, as
    a service would host; generated once)."""
    if n not in _DENSE_POOL:
        _DENSE_POOL[n] = workloads.dense_couplings(n, seed=100 + n)
    return _DENSE_POOL[n]


DENSE_SIZES = (512, 1024, 1536, 2048, 3072, 4096)


def serve_requests(rng, n, scale, dense_share=0.1):
    """Requests drawn as in the serving workload: 2D L in [32,1024], 3D L in
    [16,64] or (with probability `dense_share`) dense SK couplings N in
    [512,4096] (BF16 tensor-core form, N from a pool of six sizes), beta in
    [0.15,0.6], h in [0,0.2], 100-5000 trajectories (times `scale`, at least
    1), 1-256 chains; N_md = floor(ln N), eps = 1/(N_md sqrt(beta)), C = 2d beta
    + 0.1 (lattices) or beta |lambda_min(J)| + 0.1 (dense)."""
    out = []
    for _ in range(n):
        beta = float(rng.uniform(0.15, 0.6))
        chains = int(rng.integers(1, 257))
        traj = max(1, int(round(int(rng.integers(100, 5001)) * scale)))
        h0 = float(rng.uniform(0, 0.2))
        seed = int(rng.integers(1, 2 ** 31))
        if rng.random() < dense_share:
            N = int(DENSE_SIZES[int(rng.integers(0, len(DENSE_SIZES)))])
            J = dense_model(N)
            n_md = workloads.n_md_default(N)
            # C left to the library: beta |lambda_min(J)| + 0.1 (Lanczos at create)
            out.append(dict(n_traj=traj, seed=seed, kind="dense", J=J, beta=beta, h=h0,
                            eps=1.0 / (n_md * math.sqrt(beta)), n_md=n_md,
                            n_chains=chains, precision=2))   # ISING_PREC_BF16
            continue
        dim = 2 if rng.random() < 0.5 else 3
        L = int(rng.integers(32, 1025)) if dim == 2 else int(rng.integers(16, 65))
        if dim == 3 and L % 4:
            L += 4 - L % 4   # keep the vector path; the scalar path serves any L
        N = L ** dim
        n_md = workloads.n_md_default(N)
        out.append(dict(n_traj=traj, seed=seed, dim=dim, L=(L,) * dim, beta=beta, h=h0,
                        C=2 * dim * beta + 0.1, eps=1.0 / (n_md * math.sqrt(beta)), n_md=n_md,
                        n_chains=chains))
    return out


def request_sites(r):
    return r["J"].shape[0] if r.get("kind") == "dense" else int(np.prod(r["L"]))


def _serve_window(pkg, reqs, arrivals, budget_gb, drain=True):
    """Submit `reqs` at `arrivals` (s) to a fresh server; with drain, wait for
    all of them and return latencies; without, stop at the last arrival and
    report the queue."""
    srv = pkg.IsingServer(int(budget_gb * 1e9), 4)
    try:
        ids = []
        t0 = time.perf_counter()
        for ta, r in zip(arrivals, reqs):
            dt = ta - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            ids.append(srv.submit(**r))
        t_sub = time.perf_counter() - t0
        st_sub = srv.stats()
        if not drain:
            return {"submitted": len(ids), "seconds": t_sub, "admitted": int(st_sub["admitted"]),
                    "completed": int(st_sub["completed"]), "queued": int(st_sub["queued"]),
                    "active": int(st_sub["active"]), "rejected": int(st_sub["rejected"])}
        srv.drain(600.0)
        t_all = time.perf_counter() - t0
        res = [srv.poll(i) for i in ids]
        st = srv.stats()
    finally:
        srv.close()
    return {"res": res, "t_sub": t_sub, "t_all": t_all, "st": st,
            "peak_queue": int(st_sub["queued"])}


def _scaled(reqs, scale):
    """The same requests with their trajectory counts times `scale` (at least 1)."""
    out = []
    for r in reqs:
        q = dict(r)
        q["n_traj"] = max(1, int(round(r["n_traj"] * scale)))
        out.append(q)
    return out


def _serve_burst(pkg, reqs, budget_gb):
    """Submit every request at once to a fresh server and drain it: the work
    served per second with the queue never empty (the server's capacity for
    requests of this mix and size)."""
    work = lambda r: (request_sites(r) * r["n_chains"] * r["n_traj"] * r["n_md"])
    srv = pkg.IsingServer(int(budget_gb * 1e9), 4)
    try:
        t0 = time.perf_counter()
        for r in reqs:
            srv.submit(**r)
        srv.drain(600.0)
        dt = time.perf_counter() - t0
    finally:
        srv.close()
    return sum(work(r) for r in reqs) / dt


def serve_run(pkg, seconds, rate=200.0, rhos=(0.5, 0.8, 0.95), seed=2, budget_gb=120.0):
    """Serving: Poisson arrivals of the serving mix at `rate` requests/s with
    trajectory counts scaled so the offered load is rho of the server's
    capacity (where one trajectory per request already offers more, one
    trajectory each at a lower arrival rate), for each rho; p50/p99 latency,
    the queue when arrivals end, and the served rate.  The capacity is measured on the same mix at the same
    trajectory scale (a burst of one second's requests submitted at once and
    drained), twice: per-request costs make it depend on the scale.  Last, the
    literal workload (unscaled trajectory counts, far beyond any GPU) for a
    short window: queue growth and admissions."""
    rng = np.random.default_rng(seed)
    work = lambda r: (request_sites(r) * r["n_chains"] * r["n_traj"] * r["n_md"])
    sample = serve_requests(np.random.default_rng(7), 4000, 1.0)

    def mean_work(scale):
        return float(np.mean([work(r) for r in _scaled(sample, scale)]))

    def scale_for(load):
        """Trajectory scale at which `rate` requests/s offer `load` site-steps/s."""
        lo, hi = 1e-7, 1.0
        for _ in range(60):
            mid = math.sqrt(lo * hi)
            if rate * mean_work(mid) < load:
                lo = mid
            else:
                hi = mid
        return math.sqrt(lo * hi)

    floor_w = mean_work(1e-9)   # one trajectory per request

    def plan(load):
        """(trajectory scale, arrival rate) offering `load` site-steps/s: the
        workload's rate with scaled trajectory counts, or, where even one
        trajectory per request offers more, one trajectory each at a lower rate."""
        if rate * floor_w >= load:
            return 1e-9, load / floor_w
        return scale_for(load), rate

    cap = 1.0e11
    calib = []
    for _ in range(2):
        sc, _r = plan(cap)
        burst = _scaled(serve_requests(rng, int(rate), 1.0), sc)
        cap = _serve_burst(pkg, burst, budget_gb)
        calib.append({"trajectory_scale": sc, "capacity_site_steps_per_s": cap})
    by_rho = {}
    main = None
    # common random numbers: one request list and one unit-rate Poisson
    # process for every load, so the loads differ only in rate and scale
    secs = seconds
    base_reqs = serve_requests(rng, int(rate * secs * 1.5) + 64, 1.0)
    base_t = np.cumsum(rng.exponential(1.0, len(base_reqs)))
    for rho in rhos:
        scale, rate_rho = plan(rho * cap)
        arrivals = base_t / rate_rho
        n = int(np.searchsorted(arrivals, secs))
        arrivals = arrivals[:n]
        reqs = _scaled(base_reqs[:n], scale)
        w = _serve_window(pkg, reqs, arrivals, budget_gb)
        res, st = w["res"], w["st"]
        lat = np.array([r["latency"] for r in res if r["state"] == 2])
        done_work = sum(work(r) for r, x in zip(reqs, res) if x["state"] == 2)
        row = {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
               "mean_s": float(lat.mean()), "requests": n, "completed": int(st["completed"]),
               "rejected": int(st["rejected"]), "arrival_seconds": secs,
               "total_seconds": w["t_all"], "site_steps_per_s": done_work / w["t_all"],
               "offered_site_steps_per_s": sum(work(r) for r in reqs) / secs,
               "served_over_rho_capacity": done_work / w["t_all"] / (rho * cap),
               "trajectory_scale": scale, "arrival_rate": rate_rho,
               "queued_at_end_of_arrivals": w["peak_queue"],
               "server_seconds": {k: round(st[k], 3) for k in ("create_s", "graph_s", "quanta_s",
                                                                "retire_s")},
               "drain_seconds": w["t_all"] - w["t_sub"],
               "dense_requests": int(sum(1 for r in reqs if r.get("kind") == "dense"))}
        by_rho[str(rho)] = row
        if rho == 0.8:
            main = dict(row, rho=rho, submit_seconds=w["t_sub"],
                        capacity_site_steps_per_s=cap,
                        shared_graph_launches=int(st["group_launches"]), quanta=int(st["quanta"]))
    out = main if main is not None else {}
    out["by_rho"] = by_rho
    out["calibration"] = calib
    ks = sorted(by_rho, key=float)
    out["p50_p99_rise_with_rho"] = bool(all(
        by_rho[a]["p50_s"] <= by_rho[b]["p50_s"] and by_rho[a]["p99_s"] <= by_rho[b]["p99_s"]
        for a, b in zip(ks, ks[1:])))
    lit_secs = 2.0
    n = int(rng.poisson(rate * lit_secs))
    arrivals = np.sort(rng.uniform(0, lit_secs, n))
    reqs = serve_requests(rng, n, 1.0)
    out["literal"] = dict(_serve_window(pkg, reqs, arrivals, budget_gb, drain=False),
                          offered_site_steps=float(sum(work(r) for r in reqs)),
                          note="unscaled trajectory counts; the window ends at the last arrival, "
                               "queued work is dropped with the server")
    return out


def e2e_rate(pkg, sims, Ls, n_chains, seed, stream, steps=3):
    """Through the public C ABI with host buffers: each step uploads every chain's
    configuration from pinned host memory, runs one trajectory and reads the
    observables back."""
    import torch
    host = {}
    for L in Ls:
        host[L] = torch.empty(n_chains * L * L, dtype=torch.float32, pin_memory=True)
        pkg.ising_hmc_get_state_native(sims[L].h, host[L].data_ptr())
    h2d = sum(host[L].numel() * 4 for L in Ls)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(steps):
        # every size's upload and trajectory are queued before any result is
        # read, so a size's trajectory runs while the next size uploads
        for L in Ls:
            traj = sims[L].traj_index
            pkg.ising_hmc_set_state_native(sims[L].h, host[L].data_ptr(), traj)
            sims[L].trajectories(1, seed)
        for L in Ls:
            sims[L].observables()
    dt = time.perf_counter() - t0
    site_steps = sum(L * L for L in Ls) * n_chains * N_MD * steps
    # observables() copies the per-chain state records (sums, record, scalars) back
    d2h = len(Ls) * n_chains * 8 * (5 + 10 + 8 + 1)
    return {"value": site_steps / dt, "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "steps": steps}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
