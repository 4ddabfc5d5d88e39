// runtime.cu -- host runtime of the C ABI declared in include/ising_hmc.h.
// Owns the device state of a simulation handle and queues the kernels of the
// HMC algorithm (Sec. 3) on the handle's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include <atomic>
#include <nvtx3/nvToolsExt.h>

#include "internal.h"

using namespace ihmc;

struct ising_hmc {
    // configuration
    int kind = 0, dim = 0, L[3] = {1, 1, 1};
    int64_t N = 0;
    int n_chains = 0, n_md = 0, n_therm = 0, prec = 0, integrator = 0, flip_every = 0;
    Geometry g{};
    Schedule sched{};
    std::vector<ChainParams> params;
    bool has_h = false;
    // device
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    void *psi[3] = {nullptr, nullptr, nullptr};  // FP32 lattice: 3 buffers; plain: psi_cur, psi
    void *p = nullptr;
    double *plain_a = nullptr, *plain_u = nullptr, *plain_F = nullptr, *partials = nullptr;
    int *flags = nullptr;
    ChainParams *d_params = nullptr;
    ChainState *d_state = nullptr;
    float *d_h32 = nullptr;
    double *d_h64 = nullptr;
    double *d_J = nullptr;
    float *d_lpe = nullptr;
    int *d_err = nullptr;
    // launch shape of the fused kernel: threads per CTA, prefetch depth, CTAs per chain
    int threads = 0, depth = 0, cs = 1, staging = ISING_STAGING_AUTO;
    // FP32 lattice form: the configurations were set from outside and their
    // action is evaluated by the next trajectory's first force pass
    bool eval_pending = false;
    // dense couplings on the tensor cores
    bool dense_tc = false;
    int b_pad = 0;
    DenseArgs dense{};
    void *dJ16 = nullptr, *dJhi = nullptr, *dJlo = nullptr, *dpsi16 = nullptr, *du32 = nullptr,
         *du16 = nullptr, *dGhi = nullptr, *dGlo = nullptr;
    void *dsJ8 = nullptr;   // FP8 form: per-row scales of J
    void *dJdig = nullptr, *dpsidig = nullptr, *drow_exp = nullptr, *dchain_exp = nullptr,
         *dGint = nullptr;
    // per-trajectory series (m, E, |m| per chain and trajectory)
    double *series = nullptr;
    int64_t series_cap = 0, series_n = 0;
    // counters
    int64_t traj = 0;
    int64_t launches = 0;
    int64_t bytes = 0;
    char err[512] = {0};
};

static thread_local char g_create_err[512];

static ising_status fail(ising_hmc *h, ising_status st, const char *fmt, ...) {
    char *buf = h ? h->err : g_create_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, 512, fmt, ap);
    va_end(ap);
    return st;
}

#define CUDA_OR_FAIL(h, call)                                                           \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return fail((h), ISING_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                        __FILE__, __LINE__);                                            \
    } while (0)

static bool is_dense_tc(const ising_hmc *h) {
    return h->kind == ISING_KIND_DENSE &&
           (h->prec == ISING_PREC_BF16 || h->prec == ISING_PREC_FP8);
}

static bool is_fp32_lattice(const ising_hmc *h) {
    return h->kind == ISING_KIND_LATTICE && h->prec == ISING_PREC_FP32;
}

// Forms run by one fused whole-trajectory kernel over three state buffers:
// the FP32 lattice and the infinite-range model.
static bool is_fused(const ising_hmc *h) {
    return is_fp32_lattice(h) || h->kind == ISING_KIND_INFINITE;
}

static size_t state_elem(const ising_hmc *h) {
    return h->prec == ISING_PREC_PLAIN_FP64 ? sizeof(double) : sizeof(float);
}

// Default shift: the positive-definiteness bound of Sec. 2 plus this margin
// (the shift C = bound + 0.1 the paper's workloads use).
static constexpr double DEFAULT_SHIFT_MARGIN = 0.1;
// automatic plane staging: bulk copies from this plane size up
static constexpr int64_t BULK_AUTO_MIN_BYTES = 4096;

// Integrator schedules (Sec. 3: symmetric symplectic integrators).
static void make_schedule(int integrator, int n_md, Schedule &s) {
    if (integrator == ISING_INTEGRATOR_OMELYAN) {
        // Omelyan-Mryglod-Folk second-order minimum-norm scheme, kicks merged
        // between consecutive steps: lam, (1-2lam), 2lam, ..., (1-2lam), lam.
        const double lam = 0.1931833275037836;
        s.n_pass = 2 * n_md + 1;
        for (int j = 0; j < s.n_pass; ++j) {
            if (j == 0 || j == s.n_pass - 1) s.kick[j] = lam;
            else s.kick[j] = (j & 1) ? (1.0 - 2.0 * lam) : 2.0 * lam;
            s.drift[j] = (j == s.n_pass - 1) ? 0.0 : 0.5;
        }
    } else {
        // kick-drift-kick leapfrog with n_md drifts
        s.n_pass = n_md + 1;
        for (int j = 0; j < s.n_pass; ++j) {
            s.kick[j] = (j == 0 || j == s.n_pass - 1) ? 0.5 : 1.0;
            s.drift[j] = (j == s.n_pass - 1) ? 0.0 : 1.0;
        }
    }
}

// Device memory of a handle comes from the device's stream-ordered pool
// (cudaMallocAsync / cudaFreeAsync on the handle's stream): destroying a
// handle queues its frees behind its own work instead of synchronising the
// whole device, so a server retiring requests does not stall the others, and
// the pool keeps up to POOL_KEEP_BYTES of freed memory for the next handles.
static constexpr uint64_t POOL_KEEP_BYTES = (uint64_t)16 << 30;

// NVTX range for the duration of a scope (a profiler's timeline shows the
// library's calls; no cost without a tool attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

// Test hook (ising_hmc_inject_alloc_failure): the k-th next device
// allocation fails as if the device were out of memory.
static std::atomic<int64_t> g_fail_alloc_in{0};

static cudaError_t pool_alloc(void **ptr, size_t bytes, cudaStream_t s) {
    if (g_fail_alloc_in.load() > 0 && g_fail_alloc_in.fetch_sub(1) == 1) {
        *ptr = nullptr;
        return cudaErrorMemoryAllocation;
    }
    static thread_local int configured_dev = -1;
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && dev != configured_dev) {
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t keep = POOL_KEEP_BYTES;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
        cudaGetLastError();
        configured_dev = dev;
    }
    return cudaMallocAsync(ptr, bytes, s);
}

// Smallest eigenvalue of a dense symmetric matrix by Lanczos with full
// reorthogonalisation (Lanczos 1950), then Sturm-sequence bisection on the
// tridiagonal matrix.  Used only to validate the shift C (Sec. 2).  The
// products J q run on the device from dJ (the FP64 couplings already there)
// when given, else on the host from J.
static double lanczos_lambda_min(const double *J, const double *dJ, int64_t N, int steps) {
    steps = (int)std::min<int64_t>(steps, N);
    std::vector<double> Q((size_t)steps * N), w(N), alpha(steps), beta(steps);
    double *dq = nullptr, *dw = nullptr;
    if (dJ && (pool_alloc((void **)&dq, N * sizeof(double), nullptr) != cudaSuccess ||
               pool_alloc((void **)&dw, N * sizeof(double), nullptr) != cudaSuccess)) {
        cudaGetLastError();
        dJ = nullptr;
    }
    auto matvec = [&](const double *q) {
        if (dJ) {
            if (cudaMemcpy(dq, q, N * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess &&
                dense_matvec_f64(dJ, dq, dw, N, 0) == cudaSuccess &&
                cudaMemcpy(w.data(), dw, N * sizeof(double), cudaMemcpyDeviceToHost) == cudaSuccess)
                return;
            cudaGetLastError();
            dJ = nullptr;   // the host loop below takes over
        }
        for (int64_t i = 0; i < N; ++i) {
            double s = 0;
            const double *row = J + i * N;
            for (int64_t j = 0; j < N; ++j) s += row[j] * q[j];
            w[i] = s;
        }
    };
    // deterministic start vector
    double nrm = 0;
    for (int64_t i = 0; i < N; ++i) {
        Q[i] = 1.0 + 0.37 * std::sin(0.71 * (double)i + 0.3);
        nrm += Q[i] * Q[i];
    }
    nrm = std::sqrt(nrm);
    for (int64_t i = 0; i < N; ++i) Q[i] /= nrm;
    int k = 0;
    for (; k < steps; ++k) {
        const double *q = &Q[(size_t)k * N];
        matvec(q);
        double a = 0;
        for (int64_t i = 0; i < N; ++i) a += w[i] * q[i];
        alpha[k] = a;
        for (int pass = 0; pass < 2; ++pass) {
            for (int j = 0; j <= k; ++j) {
                const double *qj = &Q[(size_t)j * N];
                double d = 0;
                for (int64_t i = 0; i < N; ++i) d += w[i] * qj[i];
                for (int64_t i = 0; i < N; ++i) w[i] -= d * qj[i];
            }
        }
        double b = 0;
        for (int64_t i = 0; i < N; ++i) b += w[i] * w[i];
        b = std::sqrt(b);
        beta[k] = b;
        if (k + 1 >= steps || b < 1e-12) {
            ++k;
            break;
        }
        double *qn = &Q[(size_t)(k + 1) * N];
        for (int64_t i = 0; i < N; ++i) qn[i] = w[i] / b;
    }
    const int m = k;
    // bisection for the smallest eigenvalue of T (alpha, beta[0..m-2])
    double lo = 1e300, hi = -1e300;
    for (int i = 0; i < m; ++i) {
        const double r = (i > 0 ? std::fabs(beta[i - 1]) : 0) + (i + 1 < m ? std::fabs(beta[i]) : 0);
        lo = std::min(lo, alpha[i] - r);
        hi = std::max(hi, alpha[i] + r);
    }
    auto count_below = [&](double x) {
        int c = 0;
        double d = 1.0;
        for (int i = 0; i < m; ++i) {
            const double b2 = i > 0 ? beta[i - 1] * beta[i - 1] : 0.0;
            d = alpha[i] - x - (i > 0 ? b2 / d : 0.0);
            if (d == 0.0) d = 1e-300;
            if (d < 0) ++c;
        }
        return c;
    };
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (count_below(mid) >= 1) hi = mid;
        else lo = mid;
    }
    if (dq) cudaFreeAsync(dq, nullptr);
    if (dw) cudaFreeAsync(dw, nullptr);
    return 0.5 * (lo + hi);
}

// Table of g(y) = log(1 + exp(-y)) at y_k = k/32 with s = 1/(1 + e^{y_k})
// (layout in df32.cuh), each value split into a double-float pair.
void ihmc::build_log1pexp_table(float *out) {
    for (int k = 0; k < LOG1PEXP_NODES; ++k) {
        const double y = (double)k / 32.0;
        const double g0 = std::log1p(std::exp(-y));
        const double sg = 1.0 / (1.0 + std::exp(y));
        float *q = out + 4 * k;
        q[0] = (float)g0;
        q[1] = (float)(g0 - (double)q[0]);
        q[2] = (float)sg;
        q[3] = (float)(sg - (double)q[2]);
    }
}

static void free_all(ising_hmc *h) {
    for (auto &b : h->psi) {
        if (b) cudaFreeAsync(b, h->stream);
        b = nullptr;
    }
    void *bufs[] = {h->p, h->plain_a, h->plain_u, h->plain_F, h->partials, h->flags, h->d_params,
                    h->d_state, h->d_h32, h->d_h64, h->d_J, h->d_lpe, h->d_err, h->dJ16,
                    h->dJhi, h->dJlo, h->dpsi16, h->du32, h->du16, h->dGhi, h->dGlo,
                    h->dJdig, h->dpsidig, h->drow_exp, h->dchain_exp, h->dGint, h->dsJ8,
                    h->series};
    for (void *b : bufs)
        if (b) cudaFreeAsync(b, h->stream);
    h->p = nullptr;
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    h->stream = nullptr;
}

static int64_t plan_bytes(int kind, int prec, int64_t N, int n_chains, bool has_h) {
    const int64_t C = n_chains;
    int64_t b = 0;
    if (kind == ISING_KIND_DENSE && (prec == ISING_PREC_BF16 || prec == ISING_PREC_FP8)) {
        const int64_t Bp = (C + 127) / 128 * 128;
        const int64_t lb = prec == ISING_PREC_FP8 ? 1 : 2;   // bytes of the low-precision copies
        b += Bp * N * (3 * 4 + lb + 4 + lb);            // psi x2, p, psi low, u32, u low
        b += N * N * lb + (prec == ISING_PREC_FP8 ? N * 4 : 0);   // J low (+ FP8 row scales)
        if (N <= ACT_MAX_N) {                            // digit planes, exponents, G as int64
            b += (int64_t)ACT_DIGITS * (N * N + Bp * N) * 2 + Bp * N * 8 + (N + Bp) * 4;
        } else {                                         // J as two FP32, G hi/lo
            b += N * N * 8 + Bp * N * 8;
        }
        b += C * (int64_t)(sizeof(ChainParams) + sizeof(ChainState) + 2 * sizeof(int));
        if (has_h) b += N * (int64_t)(2 * sizeof(float) + sizeof(double));
        return b + 4 * LOG1PEXP_NODES * 4;
    }
    if (prec == ISING_PREC_PLAIN_FP64) {
        b += 6 * C * N * (int64_t)sizeof(double);
        b += C * 7 * (int64_t)plain_partial_blocks(N) * (int64_t)sizeof(double);
    } else {
        b += 4 * C * N * (int64_t)sizeof(float);
    }
    b += C * (int64_t)(sizeof(ChainParams) + sizeof(ChainState) + 2 * sizeof(int));
    if (has_h) b += N * (int64_t)(2 * sizeof(float) + sizeof(double));
    if (kind == ISING_KIND_DENSE) b += N * N * (int64_t)sizeof(double);
    return b;
}

template <typename T>
static ising_status dalloc(ising_hmc *h, T **ptr, size_t bytes) {
    cudaError_t e = pool_alloc((void **)ptr, bytes ? bytes : 16, h->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *ptr = nullptr;
        return fail(h, ISING_ENOMEM, "device allocation (%zu bytes) failed: %s", bytes,
                    cudaGetErrorString(e));
    }
    h->bytes += (int64_t)bytes;
    return ISING_OK;
}

static PlainArgs plain_args(ising_hmc *h, int c) {
    PlainArgs a{};
    const int64_t N = h->N;
    a.psi_cur = (double *)h->psi[0] + (int64_t)c * N;
    a.psi = (double *)h->psi[1] + (int64_t)c * N;
    a.p = (double *)h->p + (int64_t)c * N;
    a.a = h->plain_a + (int64_t)c * N;
    a.u = h->plain_u + (int64_t)c * N;
    a.F = h->plain_F + (int64_t)c * N;
    a.partials = h->partials + (int64_t)c * 7 * plain_partial_blocks(N);
    a.h64 = h->has_h ? h->d_h64 : nullptr;
    a.J = h->d_J;
    a.params = h->d_params + c;
    a.state = h->d_state + c;
    a.flag = h->flags + 2 * c;
    a.g = h->g;
    a.kind = h->kind;
    a.chain = (uint32_t)c;
    return a;
}

static cudaError_t launch_fused(ising_hmc *h, const FusedArgs &a) {
    if (h->kind == ISING_KIND_INFINITE) return launch_infinite(a, h->sched, h->stream);
    return launch_fused_lattice(a, h->sched, h->threads, h->depth, h->stream);
}


// Plane staging of the lattice kernel: bulk copies need planes of whole
// 16-byte vectors; automatic choice: bulk for planes of at least 4 KB (small
// planes stage faster with every thread's cp.async).
static int staging_bulk(const ising_hmc *h) {
    const Geometry &g = h->g;
    if (!(g.X % 4 == 0 && g.P % 4 == 0)) return 0;
    if (h->staging == ISING_STAGING_BULK) return 1;
    if (h->staging == ISING_STAGING_THREADS) return 0;
    return (int64_t)g.P * 4 >= BULK_AUTO_MIN_BYTES;
}
static FusedArgs fused_args(ising_hmc *h) {
    FusedArgs a{};
    for (int i = 0; i < 3; ++i) a.psi[i] = (float *)h->psi[i];
    a.p = (float *)h->p;
    a.hdf = h->has_h ? reinterpret_cast<const float2 *>(h->d_h32) : nullptr;
    a.lpe_tab = reinterpret_cast<const float4 *>(h->d_lpe);
    a.params = h->d_params;
    a.state = h->d_state;
    a.g = h->g;
    a.n_therm = h->n_therm;
    a.flip_every = h->flip_every;
    a.chain0 = 0;
    a.n_chains = h->n_chains;
    a.cs = is_fp32_lattice(h) ? h->cs : 1;
    a.bulk = staging_bulk(h);
    a.err = h->d_err;
    return a;
}

// Recompute S and the observables of the current configurations.
static ising_status eval_current(ising_hmc *h) {
    if (is_dense_tc(h)) {
        CUDA_OR_FAIL(h, dense_eval(h->dense, h->stream, &h->launches));
        return ISING_OK;
    }
    if (is_fused(h)) {
        FusedArgs a = fused_args(h);
        a.mode = MODE_EVAL;
        a.seed = 0;
        a.traj0 = TRAJ_INIT_INDEX;
        a.n_traj = 0;
        CUDA_OR_FAIL(h, launch_fused(h, a));
        h->launches += 1;
    } else {
        for (int c = 0; c < h->n_chains; ++c) {
            PlainArgs a = plain_args(h, c);
            CUDA_OR_FAIL(h, plain_eval(a, h->stream, &h->launches));
        }
    }
    return ISING_OK;
}

static ising_status upload_params(ising_hmc *h) {
    CUDA_OR_FAIL(h, cudaMemcpyAsync(h->d_params, h->params.data(),
                                    sizeof(ChainParams) * h->n_chains, cudaMemcpyHostToDevice,
                                    h->stream));
    return cudaStreamSynchronize(h->stream) == cudaSuccess
               ? ISING_OK
               : fail(h, ISING_ECUDA, "parameter upload failed");
}

// Series record of trajectory k: each chain's m, E, |m| (the values the
// measurement step adds to its sums) into series[(c * cap + k) * 3 + j].
__global__ void k_series_record(const ChainState *st, double *series, int n_chains, int64_t cap,
                                int64_t k) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_chains) return;
    double *r = series + ((size_t)c * cap + k) * 3;
    r[0] = st[c].obs[0];
    r[1] = st[c].obs[1];
    r[2] = st[c].obs[2];
}

static cudaError_t launch_series_record(const ChainState *st, double *series, int n_chains,
                                        int64_t cap, int64_t k, cudaStream_t s) {
    k_series_record<<<(n_chains + 127) / 128, 128, 0, s>>>(st, series, n_chains, cap, k);
    return cudaGetLastError();
}

// Chain-averaged observables from per-chain sums (ISING_NSUMS per chain):
// standard errors of the per-chain means for several chains, the naive
// sigma/sqrt(n) of the single chain otherwise.
void ihmc::obs_from_sums(const double *sums, int C, int64_t n_traj, ising_obs *out) {
    std::memset(out, 0, sizeof(*out));
    double nmeas = 0, nacc = 0, sdh = 0, sexp = 0;
    std::vector<double> cm(C), ca(C), ce(C), cx(C);
    double vm = 0, va = 0, ve = 0;
    for (int c = 0; c < C; ++c) {
        const double *s = sums + (size_t)c * ISING_NSUMS;
        const double n = s[ISING_SUM_NMEAS];
        nmeas += n;
        nacc += s[ISING_SUM_NACC];
        sdh += s[ISING_SUM_DH];
        sexp += s[ISING_SUM_EXPMDH];
        const double inv = n > 0 ? 1.0 / n : 0.0;
        cm[c] = s[ISING_SUM_M] * inv;
        ca[c] = s[ISING_SUM_ABSM] * inv;
        ce[c] = s[ISING_SUM_E] * inv;
        cx[c] = s[ISING_SUM_EXPMDH] * inv;
        if (C == 1 && n > 1) {
            vm = (s[ISING_SUM_M2] * inv - cm[c] * cm[c]) / (n - 1);
            va = (s[ISING_SUM_ABSM2] * inv - ca[c] * ca[c]) / (n - 1);
            ve = (s[ISING_SUM_E2] * inv - ce[c] * ce[c]) / (n - 1);
        }
    }
    auto mean = [&](const std::vector<double> &v) {
        double s = 0;
        for (double x : v) s += x;
        return s / (double)v.size();
    };
    auto sem = [&](const std::vector<double> &v, double mu) {
        if (v.size() < 2) return 0.0;
        double s = 0;
        for (double x : v) s += (x - mu) * (x - mu);
        return std::sqrt(s / ((double)v.size() - 1) / (double)v.size());
    };
    out->m = mean(cm);
    out->abs_m = mean(ca);
    out->E = mean(ce);
    out->mean_exp_mdH = nmeas > 0 ? sexp / nmeas : 0;
    if (C > 1) {
        out->m_err = sem(cm, out->m);
        out->abs_m_err = sem(ca, out->abs_m);
        out->E_err = sem(ce, out->E);
        out->exp_mdH_err = sem(cx, mean(cx));
    } else {
        out->m_err = std::sqrt(std::max(vm, 0.0));
        out->abs_m_err = std::sqrt(std::max(va, 0.0));
        out->E_err = std::sqrt(std::max(ve, 0.0));
    }
    out->acceptance = nmeas > 0 ? nacc / nmeas : 0;
    out->mean_dH = nmeas > 0 ? sdh / nmeas : 0;
    out->n_traj = n_traj;
    out->n_meas = (int64_t)nmeas;
}

extern "C" {

const char *ising_hmc_last_create_error(void) { return g_create_err; }

int64_t ising_hmc_estimate_bytes(const ising_hmc_config *cfg) {
    if (!cfg) return -1;
    int64_t N = 0;
    if (cfg->kind == ISING_KIND_DENSE || cfg->kind == ISING_KIND_INFINITE) N = cfg->n_sites;
    else {
        N = 1;
        for (int d = 0; d < cfg->dim && d < 3; ++d) N *= cfg->L[d];
    }
    return plan_bytes(cfg->kind, cfg->precision, N, cfg->n_chains, cfg->h != nullptr);
}

ising_status ising_hmc_create(const ising_hmc_config *cfg, ising_hmc_t **out) {
    NvtxRange nvtx_range("ising_hmc_create");
    g_create_err[0] = 0;
    if (!cfg || !out) return fail(nullptr, ISING_EINVAL, "null config or output pointer");
    *out = nullptr;
    ising_hmc *h = new (std::nothrow) ising_hmc();
    if (!h) return fail(nullptr, ISING_ENOMEM, "host allocation failed");
    auto bail = [&](ising_status st) {
        std::snprintf(g_create_err, sizeof g_create_err, "%s", h->err);
        free_all(h);
        delete h;
        return st;
    };
    h->kind = cfg->kind;
    h->prec = cfg->precision;
    h->n_chains = cfg->n_chains;
    h->n_md = cfg->n_md;
    h->n_therm = cfg->n_therm;
    h->integrator = cfg->integrator;
    h->flip_every = cfg->flip_every;
    if (h->n_chains < 1) return bail(fail(h, ISING_EINVAL, "n_chains must be >= 1"));
    if (h->n_md < 1) return bail(fail(h, ISING_EINVAL, "n_md must be >= 1"));
    if (h->integrator != ISING_INTEGRATOR_LEAPFROG && h->integrator != ISING_INTEGRATOR_OMELYAN)
        return bail(fail(h, ISING_EINVAL, "unknown integrator %d", h->integrator));
    const int passes = h->integrator == ISING_INTEGRATOR_OMELYAN ? 2 * h->n_md + 1 : h->n_md + 1;
    if (passes > MAX_PASSES) return bail(fail(h, ISING_EINVAL, "n_md too large (%d)", h->n_md));
    if (h->flip_every < 0) return bail(fail(h, ISING_EINVAL, "flip_every must be >= 0"));
    if (cfg->kind == ISING_KIND_LATTICE) {
        if (cfg->dim < 1 || cfg->dim > 3) return bail(fail(h, ISING_EINVAL, "dim must be 1..3"));
        h->dim = cfg->dim;
        int64_t N = 1;
        for (int d = 0; d < 3; ++d) {
            h->L[d] = d < cfg->dim ? cfg->L[d] : 1;
            if (d < cfg->dim && cfg->L[d] < 3)
                return bail(fail(h, ISING_EINVAL, "lattice extent L[%d]=%d < 3", d, cfg->L[d]));
            N *= h->L[d];
        }
        if (N > (int64_t)1 << 31) return bail(fail(h, ISING_EINVAL, "too many sites per chain"));
        h->N = N;
        Geometry &g = h->g;
        g.dim = h->dim;
        g.X = h->L[0];
        g.Y = h->L[1];
        g.Z = h->L[2];
        g.N = N;
        if (h->dim == 1) { g.P = g.X; g.nplanes = 1; }
        else if (h->dim == 2) { g.P = g.X; g.nplanes = g.Y; }
        else { g.P = g.X * g.Y; g.nplanes = g.Z; }
        if (h->prec != ISING_PREC_PLAIN_FP64 && h->prec != ISING_PREC_FP32)
            return bail(fail(h, ISING_EINVAL, "precision %d not available for lattices", h->prec));
    } else if (cfg->kind == ISING_KIND_DENSE) {
        if (cfg->n_sites < 1 || cfg->n_sites > 65536 || !cfg->J)
            return bail(fail(h, ISING_EINVAL, "dense model needs 1 <= n_sites <= 65536 and J"));
        h->dim = 0;
        h->N = cfg->n_sites;
        h->g.dim = 0;
        h->g.X = (int)h->N; h->g.Y = 1; h->g.Z = 1; h->g.P = (int)h->N; h->g.nplanes = 1;
        h->g.N = h->N;
        if (h->prec == ISING_PREC_BF16 || h->prec == ISING_PREC_FP8) {
            if (h->N % 128)
                return bail(fail(h, ISING_EINVAL,
                                 "tensor-core dense form needs n_sites a multiple of 128"));
            h->dense_tc = true;
            h->b_pad = (h->n_chains + 127) / 128 * 128;
        } else if (h->prec != ISING_PREC_PLAIN_FP64) {
            return bail(fail(h, ISING_EINVAL, "precision %d not available for dense couplings in this build",
                             h->prec));
        }
    } else if (cfg->kind == ISING_KIND_INFINITE) {
        if (cfg->n_sites < 2 || cfg->n_sites > ((int64_t)1 << 31))
            return bail(fail(h, ISING_EINVAL, "infinite-range model needs 2 <= n_sites <= 2^31"));
        if (h->prec != ISING_PREC_FP32)
            return bail(fail(h, ISING_EINVAL,
                             "precision %d not available for the infinite-range model", h->prec));
        h->dim = 0;
        h->N = cfg->n_sites;
        h->g.dim = 0;
        h->g.X = 1; h->g.Y = 1; h->g.Z = 1; h->g.P = 1; h->g.nplanes = 1;
        h->g.N = h->N;
    } else {
        return bail(fail(h, ISING_EINVAL, "unknown kind %d", cfg->kind));
    }
    const int64_t N = h->N;
    // per-chain parameters and the positive-definiteness check (Sec. 2)
    double lam_min = 0.0;
    if (h->kind == ISING_KIND_DENSE) {
        for (int64_t i = 0; i < N; ++i) {
            if (cfg->J[i * N + i] != 0.0) return bail(fail(h, ISING_EINVAL, "J_ii must be 0"));
            for (int64_t j = 0; j < i; ++j)
                if (cfg->J[i * N + j] != cfg->J[j * N + i])
                    return bail(fail(h, ISING_EINVAL, "J must be symmetric"));
        }
        // FP64 couplings on the device (the plain form keeps them, the BF16
        // form derives its operands from them), also used by the Lanczos check
        const size_t jb = (size_t)N * N * sizeof(double);
        int dev0 = 0;
        if (cudaGetDevice(&dev0) == cudaSuccess &&
            pool_alloc((void **)&h->d_J, jb, nullptr) == cudaSuccess &&
            cudaMemcpy(h->d_J, cfg->J, jb, cudaMemcpyHostToDevice) == cudaSuccess) {
            h->bytes += (int64_t)jb;
        } else {
            cudaGetLastError();
            if (h->d_J) cudaFreeAsync(h->d_J, nullptr);
            h->d_J = nullptr;
        }
        lam_min = lanczos_lambda_min(cfg->J, h->d_J, N, (int)std::min<int64_t>(N, 96));
    }
    h->params.resize(h->n_chains);
    for (int c = 0; c < h->n_chains; ++c) {
        ChainParams &p = h->params[c];
        const double beta = cfg->beta_chain ? cfg->beta_chain[c] : cfg->beta;
        double C = cfg->C_chain ? cfg->C_chain[c] : cfg->C;
        const double eps = cfg->eps_chain ? cfg->eps_chain[c] : cfg->eps;
        const double h0 = cfg->h0_chain ? cfg->h0_chain[c] : cfg->h0;
        if (!(beta > 0) || !(eps > 0) || !std::isfinite(C) || !std::isfinite(h0))
            return bail(fail(h, ISING_EINVAL, "chain %d: need beta > 0, eps > 0, finite C and h0", c));
        // Sec. 2: A = beta*J*K + C*1 is positive definite iff C exceeds minus
        // the smallest eigenvalue of beta*J*K; C <= 0 selects that bound + 0.1
        double bound;
        const char *what;
        if (h->kind == ISING_KIND_LATTICE) {
            bound = beta * std::fabs(cfg->Jnn) * 2 * h->dim;
            what = "beta*|J|*2*dim";
        } else if (h->kind == ISING_KIND_INFINITE) {
            // eigenvalues of beta*J*K: -beta*J/N (N-1 times), beta*J*(N-1)/N
            const double Nd = (double)N;
            bound = cfg->Jnn >= 0 ? beta * cfg->Jnn / Nd : beta * -cfg->Jnn * (Nd - 1.0) / Nd;
            what = "the largest -eigenvalue of beta*J*K";
        } else {
            bound = beta * std::fabs(lam_min);
            what = "beta*|lambda_min(J)|";
        }
        if (C <= 0.0) C = bound + DEFAULT_SHIFT_MARGIN;
        const bool ok = h->kind == ISING_KIND_DENSE ? C > bound * (1.0 + 1e-9) + 1e-12 : C > bound;
        if (!ok)
            return bail(fail(h, ISING_ENOTPD, "chain %d: C=%g must exceed %s=%g (Sec. 2)", c, C,
                             what, bound));
        p.beta = beta;
        // lattice: beta*J; dense: beta (J carries the couplings); infinite:
        // kappa = beta*J/N, the coupling of every pair
        p.bJ = h->kind == ISING_KIND_LATTICE    ? beta * cfg->Jnn
               : h->kind == ISING_KIND_INFINITE ? beta * cfg->Jnn / (double)N
                                                : beta;
        p.C = C;
        p.eps = eps;
        p.hp = beta * h0;
        p.betaf = (float)p.beta;
        p.bJf = (float)p.bJ;
        p.Cf = (float)p.C;
        p.epsf = (float)p.eps;
        p.hpf = (float)p.hp;
    }
    make_schedule(h->integrator, h->n_md, h->sched);
    h->has_h = cfg->h != nullptr;
    if (is_fp32_lattice(h)) {
        if (fused_lattice_pick(h->g, &h->threads, &h->depth) < 0)
            return bail(fail(h, ISING_EINVAL, "lattice plane of %d sites does not fit on chip", h->g.P));
    }
    // device state
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return bail(fail(h, ISING_ECUDA, "no CUDA device"));
    if (cfg->stream) {
        h->stream = (cudaStream_t)cfg->stream;
    } else {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess)
            return bail(fail(h, ISING_ECUDA, "stream creation failed"));
        h->own_stream = true;
    }
    // every dense form computes from the FP64 couplings on the device
    if (h->kind == ISING_KIND_DENSE && !h->d_J)
        return bail(fail(h, ISING_ENOMEM, "device allocation of the %lld x %lld couplings failed",
                         (long long)N, (long long)N));
    const size_t elem = state_elem(h);
    const size_t sbytes = (size_t)(h->dense_tc ? h->b_pad : h->n_chains) * N * elem;
    ising_status st;
    const int nbuf = is_fused(h) ? 3 : 2;
    for (int i = 0; i < nbuf; ++i)
        if ((st = dalloc(h, &h->psi[i], sbytes)) != ISING_OK) return bail(st);
    if ((st = dalloc(h, &h->p, sbytes)) != ISING_OK) return bail(st);
    if (h->prec == ISING_PREC_PLAIN_FP64) {
        const size_t nb = (size_t)h->n_chains * N * sizeof(double);
        if ((st = dalloc(h, &h->plain_a, nb)) != ISING_OK) return bail(st);
        if ((st = dalloc(h, &h->plain_u, nb)) != ISING_OK) return bail(st);
        if ((st = dalloc(h, &h->plain_F, nb)) != ISING_OK) return bail(st);
        if ((st = dalloc(h, &h->partials,
                         (size_t)h->n_chains * 7 * plain_partial_blocks(N) * sizeof(double))) != ISING_OK)
            return bail(st);
    }
    if ((st = dalloc(h, &h->flags, (size_t)h->n_chains * 2 * sizeof(int))) != ISING_OK) return bail(st);
    if ((st = dalloc(h, &h->d_params, sizeof(ChainParams) * h->n_chains)) != ISING_OK) return bail(st);
    if ((st = dalloc(h, &h->d_state, sizeof(ChainState) * h->n_chains)) != ISING_OK) return bail(st);
    if ((st = dalloc(h, &h->d_err, sizeof(int))) != ISING_OK) return bail(st);
    if (is_fused(h) || is_dense_tc(h)) {
        std::vector<float> tab(4 * LOG1PEXP_NODES);
        build_log1pexp_table(tab.data());
        if ((st = dalloc(h, &h->d_lpe, tab.size() * sizeof(float))) != ISING_OK) return bail(st);
        if (cudaMemcpyAsync(h->d_lpe, tab.data(), tab.size() * sizeof(float), cudaMemcpyHostToDevice,
                            h->stream) != cudaSuccess)
            return bail(fail(h, ISING_ECUDA, "table upload failed"));
    }
    if (h->has_h) {
        // FP32 form: h_i as a double-float pair (hi, lo)
        std::vector<float> h32(2 * N);
        for (int64_t i = 0; i < N; ++i) {
            h32[2 * i] = (float)cfg->h[i];
            h32[2 * i + 1] = (float)(cfg->h[i] - (double)h32[2 * i]);
        }
        if ((st = dalloc(h, &h->d_h32, 2 * N * sizeof(float))) != ISING_OK) return bail(st);
        if ((st = dalloc(h, &h->d_h64, N * sizeof(double))) != ISING_OK) return bail(st);
        if (cudaMemcpyAsync(h->d_h32, h32.data(), 2 * N * sizeof(float), cudaMemcpyHostToDevice,
                            h->stream) != cudaSuccess ||
            cudaMemcpyAsync(h->d_h64, cfg->h, N * sizeof(double), cudaMemcpyHostToDevice,
                            h->stream) != cudaSuccess)
            return bail(fail(h, ISING_ECUDA, "field upload failed"));
    }
    if (is_dense_tc(h)) {
        const size_t bn = (size_t)h->b_pad * N;
        const bool fp8 = h->prec == ISING_PREC_FP8;
        const size_t lb = fp8 ? 1 : 2;   // low-precision copies of psi, u, J: E4M3 or BF16
        if ((st = dalloc(h, &h->dpsi16, bn * lb)) != ISING_OK) return bail(st);
        if ((st = dalloc(h, &h->du32, bn * 4)) != ISING_OK) return bail(st);
        if ((st = dalloc(h, &h->du16, bn * lb)) != ISING_OK) return bail(st);
        const bool act_tc = N <= ACT_MAX_N;
        if (!h->d_J) return bail(fail(h, ISING_ECUDA, "coupling upload failed"));
        if ((st = dalloc(h, &h->dJ16, (size_t)N * N * lb)) != ISING_OK) return bail(st);
        if (fp8 && (st = dalloc(h, &h->dsJ8, (size_t)N * sizeof(float))) != ISING_OK) return bail(st);
        if (cudaMemsetAsync(h->dpsi16, 0, bn * lb, h->stream) != cudaSuccess ||
            cudaMemsetAsync(h->du32, 0, bn * 4, h->stream) != cudaSuccess ||
            cudaMemsetAsync(h->du16, 0, bn * lb, h->stream) != cudaSuccess ||
            cudaMemsetAsync(h->psi[1], 0, bn * 4, h->stream) != cudaSuccess)
            return bail(fail(h, ISING_ECUDA, "dense upload failed"));
        if (act_tc) {
            // J in ACT_DIGITS base-2^ACT_BITS digit planes of row-scaled J (exact)
            const size_t nn = (size_t)N * N;
            if ((st = dalloc(h, &h->dJdig, (size_t)ACT_DIGITS * nn * 2)) != ISING_OK) return bail(st);
            if ((st = dalloc(h, &h->dpsidig, (size_t)ACT_DIGITS * bn * 2)) != ISING_OK) return bail(st);
            if ((st = dalloc(h, &h->drow_exp, (size_t)N * sizeof(int))) != ISING_OK) return bail(st);
            if ((st = dalloc(h, &h->dchain_exp, (size_t)h->b_pad * sizeof(int))) != ISING_OK)
                return bail(st);
            if ((st = dalloc(h, &h->dGint, bn * 8)) != ISING_OK) return bail(st);
            if (cudaMemsetAsync(h->dpsidig, 0, (size_t)ACT_DIGITS * bn * 2, h->stream) != cudaSuccess)
                return bail(fail(h, ISING_ECUDA, "dense upload failed"));
        } else {
            if ((st = dalloc(h, &h->dGhi, bn * 4)) != ISING_OK) return bail(st);
            if ((st = dalloc(h, &h->dGlo, bn * 4)) != ISING_OK) return bail(st);
            if ((st = dalloc(h, &h->dJhi, (size_t)N * N * 4)) != ISING_OK) return bail(st);
            if ((st = dalloc(h, &h->dJlo, (size_t)N * N * 4)) != ISING_OK) return bail(st);
        }
        // BF16 copy and the action's operands, derived on the device; the FP64
        // couplings are not needed afterwards
        if (dense_prepare(h->d_J, N, fp8 ? nullptr : (uint16_t *)h->dJ16, (uint16_t *)h->dJdig,
                          (int *)h->drow_exp, (float *)h->dJhi, (float *)h->dJlo,
                          fp8 ? (uint8_t *)h->dJ16 : nullptr, (float *)h->dsJ8,
                          h->stream) != cudaSuccess ||
            cudaStreamSynchronize(h->stream) != cudaSuccess)
            return bail(fail(h, ISING_ECUDA, "dense set-up failed: %s",
                             cudaGetErrorString(cudaGetLastError())));
        cudaFreeAsync(h->d_J, h->stream);
        h->d_J = nullptr;
        h->bytes -= (int64_t)N * N * (int64_t)sizeof(double);
        DenseArgs &d = h->dense;
        d.fp8 = fp8 ? 1 : 0;
        d.J16 = fp8 ? nullptr : (const __nv_bfloat16 *)h->dJ16;
        d.J8 = fp8 ? (const uint8_t *)h->dJ16 : nullptr;
        d.sJ8 = (const float *)h->dsJ8;
        d.psi8 = fp8 ? (uint8_t *)h->dpsi16 : nullptr;
        d.u8 = fp8 ? (uint8_t *)h->du16 : nullptr;
        d.Jhi = (const float *)h->dJhi;
        d.Jlo = (const float *)h->dJlo;
        d.psi_cur = (float *)h->psi[0];
        d.psi = (float *)h->psi[1];
        d.psi16 = fp8 ? nullptr : (__nv_bfloat16 *)h->dpsi16;
        d.p = (float *)h->p;
        d.u32 = (float *)h->du32;
        d.u16 = fp8 ? nullptr : (__nv_bfloat16 *)h->du16;
        d.Ghi = (float *)h->dGhi;
        d.Glo = (float *)h->dGlo;
        d.action_tc = act_tc ? 1 : 0;
        d.Jdig = (const __nv_bfloat16 *)h->dJdig;
        d.psidig = (__nv_bfloat16 *)h->dpsidig;
        d.row_exp = (const int *)h->drow_exp;
        d.chain_exp = (int *)h->dchain_exp;
        d.Gint = (long long *)h->dGint;
        d.hdf = h->has_h ? (const float2 *)h->d_h32 : nullptr;
        d.lpe_tab = (const float4 *)h->d_lpe;
        d.params = h->d_params;
        d.state = h->d_state;
        d.N = (int)N;
        d.n_chains = h->n_chains;
        d.b_pad = h->b_pad;
        d.err = h->d_err;
        if (dense_setup(d) != cudaSuccess)
            return bail(fail(h, ISING_ECUDA, "tensor map setup failed"));
    } else if (h->kind == ISING_KIND_DENSE) {
        if (!h->d_J) return bail(fail(h, ISING_ECUDA, "coupling upload failed"));
    }
    // zero state, psi = 0
    std::vector<ChainState> hs(h->n_chains);
    std::memset(hs.data(), 0, sizeof(ChainState) * h->n_chains);
    for (auto &s : hs) { s.start = 0; s.prop = 0; }
    // every upload of the set-up runs on the handle's stream, which the
    // stream-ordered allocations above are ordered on
    if (cudaMemcpyAsync(h->d_state, hs.data(), sizeof(ChainState) * h->n_chains,
                        cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
        cudaMemsetAsync(h->psi[0], 0, sbytes, h->stream) != cudaSuccess ||
        cudaMemsetAsync(h->p, 0, sbytes, h->stream) != cudaSuccess ||
        cudaMemsetAsync(h->d_err, 0, sizeof(int), h->stream) != cudaSuccess ||
        cudaMemsetAsync(h->flags, 0, (size_t)h->n_chains * 2 * sizeof(int), h->stream) != cudaSuccess)
        return bail(fail(h, ISING_ECUDA, "state initialisation failed"));
    if ((st = upload_params(h)) != ISING_OK) return bail(st);
    if ((st = eval_current(h)) != ISING_OK) return bail(st);
    if (cudaStreamSynchronize(h->stream) != cudaSuccess)
        return bail(fail(h, ISING_ECUDA, "initial evaluation failed: %s",
                         cudaGetErrorString(cudaGetLastError())));
    *out = h;
    return ISING_OK;
}

static ising_status run_trajectories(ising_hmc *h, int64_t n, uint64_t seed);

ising_status ising_hmc_trajectories(ising_hmc_t *h, int64_t n, uint64_t seed) {
    NvtxRange nvtx_range("ising_hmc_trajectories");
    if (!h) return ISING_EINVAL;
    if (n < 0) return fail(h, ISING_EINVAL, "n must be >= 0");
    if (n == 0) return ISING_OK;
    // while a series is recorded: one trajectory per launch, then its record
    while (n > 0 && h->series && h->series_n < h->series_cap) {
        ising_status st = run_trajectories(h, 1, seed);
        if (st != ISING_OK) return st;
        CUDA_OR_FAIL(h, launch_series_record(h->d_state, h->series, h->n_chains, h->series_cap,
                                             h->series_n, h->stream));
        h->launches += 1;
        h->series_n += 1;
        --n;
    }
    return n > 0 ? run_trajectories(h, n, seed) : ISING_OK;
}

ising_status ising_hmc_solve_A(ising_hmc_t *h, int chain, const double *b, double *x, double tol,
                               int max_iter, int *iters, double *resid) {
    if (!h || !b || !x) return ISING_EINVAL;
    if (chain < 0 || chain >= h->n_chains) return fail(h, ISING_EINVAL, "chain %d out of range", chain);
    if (h->kind == ISING_KIND_DENSE && !(h->prec == ISING_PREC_PLAIN_FP64 && h->d_J))
        return fail(h, ISING_EINVAL,
                    "solve_A with dense couplings needs the plain FP64 form (it keeps J in FP64)");
    if (!(tol > 0) || max_iter < 1) return fail(h, ISING_EINVAL, "need tol > 0 and max_iter >= 1");
    ising_status st = ising_hmc_sync(h);
    if (st != ISING_OK) return st;
    const int64_t N = h->N;
    double *buf = nullptr;   // b, x, r, d, Ad, then resid and iters
    const size_t bytes = (size_t)5 * N * sizeof(double) + 2 * sizeof(double);
    if (cudaMalloc((void **)&buf, bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(h, ISING_ENOMEM, "solve_A: device allocation of %zu bytes failed", bytes);
    }
    double *dres = buf + 5 * N;
    int *dit = reinterpret_cast<int *>(buf + 5 * N + 1);
    const ChainParams &p = h->params[chain];
    cudaError_t e = cudaMemcpyAsync(buf, b, N * sizeof(double), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
        e = solve_A(buf, buf + N, buf + 2 * N, N, h->kind, h->dim, h->L, p.bJ, p.C, tol, max_iter,
                    dit, dres, h->stream, h->kind == ISING_KIND_DENSE ? h->d_J : nullptr);
    double res = 0;
    int it = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(x, buf + N, N * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&res, dres, sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&it, dit, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(buf);
    if (e != cudaSuccess) return fail(h, ISING_ECUDA, "solve_A: %s", cudaGetErrorString(e));
    h->launches += 1;
    if (iters) *iters = it;
    if (resid) *resid = res;
    return ISING_OK;
}

ising_status ising_hmc_series_enable(ising_hmc_t *h, int64_t capacity) {
    if (!h) return ISING_EINVAL;
    if (capacity < 0) return fail(h, ISING_EINVAL, "capacity must be >= 0");
    ising_status st = ising_hmc_sync(h);
    if (st != ISING_OK) return st;
    if (h->series) {
        cudaFreeAsync(h->series, h->stream);
        h->bytes -= h->series_cap * h->n_chains * 3 * (int64_t)sizeof(double);
        h->series = nullptr;
    }
    h->series_cap = 0;
    h->series_n = 0;
    if (capacity == 0) return ISING_OK;
    st = dalloc(h, &h->series, (size_t)capacity * h->n_chains * 3 * sizeof(double));
    if (st != ISING_OK) return st;
    h->series_cap = capacity;
    return ISING_OK;
}

ising_status ising_hmc_series_get(ising_hmc_t *h, double *out, int64_t *n_out) {
    if (!h || !n_out) return ISING_EINVAL;
    ising_status st = ising_hmc_sync(h);
    if (st != ISING_OK) return st;
    *n_out = h->series_n;
    if (!h->series || h->series_n == 0 || !out) return ISING_OK;   // NULL out: query n only
    // device layout [chain][capacity][3] -> host [chain][n][3]
    for (int c = 0; c < h->n_chains; ++c)
        CUDA_OR_FAIL(h, cudaMemcpy(out + (size_t)c * h->series_n * 3,
                                   h->series + (size_t)c * h->series_cap * 3,
                                   (size_t)h->series_n * 3 * sizeof(double), cudaMemcpyDeviceToHost));
    return ISING_OK;
}

// Gamma method with automatic windowing (Wolff, Comput. Phys. Commun. 156
// (2004) 143): R replicas of length n; Gamma(t) from all replicas about the
// global mean, tau_int(W) = 1/2 + sum_{t<=W} Gamma(t)/Gamma(0), W the first
// window with exp(-W/tau_W) - tau_W/sqrt(W N) < 0 where tau_W =
// S / ln((2 tau_int + 1)/(2 tau_int - 1)); the bias of Gamma from the
// estimated mean is corrected by C_W / N (his Eq. 31).
ising_status ising_gamma_method(const double *x, int64_t n, int n_rep, double S, double *out) {
    if (!x || !out || n < 2 || n_rep < 1 || !(S > 0))
        return fail(nullptr, ISING_EINVAL, "gamma method: need n >= 2, n_rep >= 1, S > 0");
    const double Ntot = (double)n * n_rep;
    double mean = 0;
    for (int64_t i = 0; i < n * n_rep; ++i) mean += x[i];
    mean /= Ntot;
    auto gamma = [&](int64_t t) {
        double g = 0;
        for (int r = 0; r < n_rep; ++r) {
            const double *xr = x + (size_t)r * n;
            for (int64_t i = 0; i + t < n; ++i) g += (xr[i] - mean) * (xr[i + t] - mean);
        }
        return g / ((double)(n - t) * n_rep);
    };
    std::vector<double> G;
    G.push_back(gamma(0));
    for (int k = 0; k < 5; ++k) out[k] = 0;
    out[0] = mean;
    if (G[0] <= 0) {
        out[2] = 0.5;
        return ISING_OK;
    }
    int64_t W = 0;
    double csum = G[0];   // G(0) + 2 sum_{t<=W} G(t)
    const int64_t Wmax = n / 2;
    for (int64_t t = 1; t <= Wmax; ++t) {
        G.push_back(gamma(t));
        csum += 2 * G[t];
        const double tau = csum / (2 * G[0]);
        if (tau <= 0.5) { W = t; break; }
        const double tw = S / std::log((2 * tau + 1) / (2 * tau - 1));
        if (std::exp(-(double)t / tw) - tw / std::sqrt((double)t * Ntot) < 0) { W = t; break; }
        W = t;
    }
    // bias correction, then tau_int and the errors at the chosen window
    const double CW = csum;
    double g0 = G[0] + CW / Ntot, cs = g0;
    for (int64_t t = 1; t <= W; ++t) cs += 2 * (G[t] + CW / Ntot);
    double tau = std::max(cs / (2 * g0), 0.5);
    out[1] = std::sqrt(std::max(cs, 0.0) / Ntot);
    out[2] = tau;
    out[3] = tau * std::sqrt(std::max(4.0 / Ntot * ((double)W + 0.5 - tau), 0.0));
    out[4] = (double)W;
    return ISING_OK;
}

static ising_status run_trajectories(ising_hmc *h, int64_t n, uint64_t seed) {
    if (h->traj + n > (int64_t)0xfffffffe) return fail(h, ISING_EINVAL, "trajectory counter overflow");
    if (is_dense_tc(h)) {
        for (int64_t t = 0; t < n; ++t) {
            const uint32_t tr = (uint32_t)(h->traj + t);
            const int flip = h->flip_every > 0 && ((tr + 1) % (uint32_t)h->flip_every) == 0;
            CUDA_OR_FAIL(h, dense_trajectory(h->dense, h->sched, seed, tr,
                                             (int64_t)tr >= (int64_t)h->n_therm, flip, h->stream,
                                             &h->launches));
        }
        h->traj += n;
        return ISING_OK;
    }
    if (is_fused(h)) {
        // trajectories per launch: keep each launch to a bounded amount of work
        const double work = (double)h->N * h->n_chains * h->sched.n_pass;
        int64_t per = (int64_t)std::max(1.0, std::floor(4.0e9 / std::max(work, 1.0)));
        per = std::min<int64_t>(per, 4096);
        int64_t done = 0;
        while (done < n) {
            const int64_t k = std::min(per, n - done);
            FusedArgs a = fused_args(h);
            a.mode = MODE_TRAJ;
            a.seed = seed;
            a.traj0 = (uint32_t)(h->traj + done);
            a.n_traj = (int)k;
            a.eval_start = done == 0 && h->eval_pending;
            CUDA_OR_FAIL(h, launch_fused(h, a));
            h->eval_pending = false;
            h->launches += 1;
            done += k;
        }
    } else {
        for (int64_t t = 0; t < n; ++t) {
            const uint32_t tr = (uint32_t)(h->traj + t);
            const int measure = (int64_t)tr >= (int64_t)h->n_therm;
            const int flip = h->flip_every > 0 && ((tr + 1) % (uint32_t)h->flip_every) == 0;
            for (int c = 0; c < h->n_chains; ++c) {
                PlainArgs a = plain_args(h, c);
                CUDA_OR_FAIL(h, plain_trajectory(a, h->sched, seed, tr, measure, flip, h->stream,
                                                 &h->launches));
            }
        }
    }
    h->traj += n;
    return ISING_OK;
}

ising_status ising_hmc_sync(ising_hmc_t *h) {
    if (!h) return ISING_EINVAL;
    CUDA_OR_FAIL(h, cudaStreamSynchronize(h->stream));
    int err = 0;
    CUDA_OR_FAIL(h, cudaMemcpy(&err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err & KERR_TIMEOUT) return fail(h, ISING_ETIMEOUT, "a device-side wait gave up");
    if (err) return fail(h, ISING_ECUDA, "device error word %d", err);
    return ISING_OK;
}

static ising_status fetch_states(ising_hmc *h, std::vector<ChainState> &hs) {
    ising_status st = ising_hmc_sync(h);
    if (st != ISING_OK) return st;
    hs.resize(h->n_chains);
    CUDA_OR_FAIL(h, cudaMemcpy(hs.data(), h->d_state, sizeof(ChainState) * h->n_chains,
                               cudaMemcpyDeviceToHost));
    return ISING_OK;
}

ising_status ising_hmc_chain_sums(ising_hmc_t *h, double *out) {
    if (!h || !out) return ISING_EINVAL;
    std::vector<ChainState> hs;
    ising_status st = fetch_states(h, hs);
    if (st != ISING_OK) return st;
    for (int c = 0; c < h->n_chains; ++c)
        std::memcpy(out + (size_t)c * ISING_NSUMS, hs[c].sums, sizeof(double) * ISING_NSUMS);
    return ISING_OK;
}

ising_status ising_hmc_last_records(ising_hmc_t *h, double *out) {
    if (!h || !out) return ISING_EINVAL;
    std::vector<ChainState> hs;
    ising_status st = fetch_states(h, hs);
    if (st != ISING_OK) return st;
    for (int c = 0; c < h->n_chains; ++c)
        std::memcpy(out + (size_t)c * ISING_NREC, hs[c].rec, sizeof(double) * ISING_NREC);
    return ISING_OK;
}

ising_status ising_hmc_reset_sums(ising_hmc_t *h) {
    if (!h) return ISING_EINVAL;
    std::vector<ChainState> hs;
    ising_status st = fetch_states(h, hs);
    if (st != ISING_OK) return st;
    for (auto &s : hs) std::memset(s.sums, 0, sizeof(s.sums));
    CUDA_OR_FAIL(h, cudaMemcpy(h->d_state, hs.data(), sizeof(ChainState) * h->n_chains,
                               cudaMemcpyHostToDevice));
    return ISING_OK;
}

ising_status ising_hmc_set_sums(ising_hmc_t *h, const double *in) {
    if (!h || !in) return ISING_EINVAL;
    std::vector<ChainState> hs;
    ising_status st = fetch_states(h, hs);
    if (st != ISING_OK) return st;
    for (int c = 0; c < h->n_chains; ++c)
        std::memcpy(hs[c].sums, in + (size_t)c * ISING_NSUMS, sizeof(double) * ISING_NSUMS);
    CUDA_OR_FAIL(h, cudaMemcpy(h->d_state, hs.data(), sizeof(ChainState) * h->n_chains,
                               cudaMemcpyHostToDevice));
    return ISING_OK;
}

ising_status ising_hmc_observables(ising_hmc_t *h, ising_obs *out) {
    NvtxRange nvtx_range("ising_hmc_observables");
    if (!h || !out) return ISING_EINVAL;
    std::vector<ChainState> hs;
    ising_status st = fetch_states(h, hs);
    if (st != ISING_OK) return st;
    std::vector<double> sums((size_t)h->n_chains * ISING_NSUMS);
    for (int c = 0; c < h->n_chains; ++c)
        std::memcpy(&sums[(size_t)c * ISING_NSUMS], hs[c].sums, sizeof(double) * ISING_NSUMS);
    obs_from_sums(sums.data(), h->n_chains, h->traj, out);
    return ISING_OK;
}

ising_status ising_hmc_get_chains(ising_hmc_t *h, int which, int chain0, int count, double *out) {
    if (!h || !out) return ISING_EINVAL;
    if (which < 0 || which > 2) return fail(h, ISING_EINVAL, "unknown state %d", which);
    if (chain0 < 0 || count < 0 || chain0 + count > h->n_chains)
        return fail(h, ISING_EINVAL, "chain range [%d, %d) out of [0, %d)", chain0, chain0 + count,
                    h->n_chains);
    std::vector<ChainState> hs;
    ising_status st = fetch_states(h, hs);
    if (st != ISING_OK) return st;
    const int64_t N = h->N;
    std::vector<float> tmp;
    for (int k = 0; k < count; ++k) {
        const int c = chain0 + k;
        const void *src;
        if (which == ISING_STATE_P_END) src = (const char *)h->p + (size_t)c * N * state_elem(h);
        else if (is_fused(h)) {
            const int b = which == ISING_STATE_PSI ? hs[c].start : hs[c].prop;
            src = (const char *)h->psi[b] + (size_t)c * N * sizeof(float);
        } else {
            src = (const char *)h->psi[which == ISING_STATE_PSI ? 0 : 1] + (size_t)c * N * state_elem(h);
        }
        if (state_elem(h) == sizeof(double)) {
            CUDA_OR_FAIL(h, cudaMemcpy(out + (size_t)k * N, src, N * sizeof(double), cudaMemcpyDeviceToHost));
        } else {
            tmp.resize(N);
            CUDA_OR_FAIL(h, cudaMemcpy(tmp.data(), src, N * sizeof(float), cudaMemcpyDeviceToHost));
            for (int64_t i = 0; i < N; ++i) out[(size_t)k * N + i] = tmp[i];
        }
    }
    return ISING_OK;
}

ising_status ising_hmc_get_state(ising_hmc_t *h, int which, double *out) {
    if (!h) return ISING_EINVAL;
    return ising_hmc_get_chains(h, which, 0, h->n_chains, out);
}

static ising_status after_set_state(ising_hmc_t *h, int64_t next_traj) {
    if (is_fp32_lattice(h)) {
        // current configuration in buffer 0; S and the observables come from
        // the first force pass of the next trajectory (no extra sweep)
        CUDA_OR_FAIL(h, launch_reset_chain_start(h->d_state, h->n_chains, h->stream));
        h->eval_pending = true;
        h->traj = next_traj;
        return ising_hmc_sync(h);
    }
    std::vector<ChainState> hs;
    ising_status st = fetch_states(h, hs);
    if (st != ISING_OK) return st;
    for (auto &s : hs) { s.start = 0; s.prop = 0; }
    CUDA_OR_FAIL(h, cudaMemcpy(h->d_state, hs.data(), sizeof(ChainState) * h->n_chains,
                               cudaMemcpyHostToDevice));
    h->traj = next_traj;
    st = eval_current(h);
    if (st != ISING_OK) return st;
    return ising_hmc_sync(h);
}

ising_status ising_hmc_set_state(ising_hmc_t *h, const double *psi, int64_t next_traj) {
    NvtxRange nvtx_range("ising_hmc_set_state");
    if (!h || !psi) return ISING_EINVAL;
    if (next_traj < 0 || next_traj > (int64_t)0xfffffffe) return fail(h, ISING_EINVAL, "bad trajectory index");
    ising_status st = ising_hmc_sync(h);
    if (st != ISING_OK) return st;
    const size_t total = (size_t)h->n_chains * h->N;
    if (state_elem(h) == sizeof(double)) {
        CUDA_OR_FAIL(h, cudaMemcpy(h->psi[0], psi, total * sizeof(double), cudaMemcpyHostToDevice));
    } else {
        std::vector<float> tmp(total);
        for (size_t i = 0; i < total; ++i) tmp[i] = (float)psi[i];
        CUDA_OR_FAIL(h, cudaMemcpy(h->psi[0], tmp.data(), total * sizeof(float), cudaMemcpyHostToDevice));
    }
    return after_set_state(h, next_traj);
}

ising_status ising_hmc_set_state_native(ising_hmc_t *h, const void *psi_dev, int64_t next_traj) {
    NvtxRange nvtx_range("ising_hmc_set_state_native");
    if (!h || !psi_dev) return ISING_EINVAL;
    if (next_traj < 0 || next_traj > (int64_t)0xfffffffe) return fail(h, ISING_EINVAL, "bad trajectory index");
    ising_status st = ising_hmc_sync(h);
    if (st != ISING_OK) return st;
    const size_t bytes = (size_t)h->n_chains * h->N * state_elem(h);
    // pinned (or mapped) host memory the device can read, 16-byte aligned:
    // the SMs copy it over the CPU-GPU link; anything else by cudaMemcpyAsync
    cudaPointerAttributes pa{};
    const bool host_mapped = cudaPointerGetAttributes(&pa, psi_dev) == cudaSuccess &&
                             pa.type == cudaMemoryTypeHost && pa.devicePointer != nullptr;
    cudaGetLastError();
    if (host_mapped && bytes % 16 == 0 && ((uintptr_t)pa.devicePointer % 16) == 0 &&
        ((uintptr_t)h->psi[0] % 16) == 0) {
        CUDA_OR_FAIL(h, launch_copy16(pa.devicePointer, h->psi[0], bytes, h->stream));
        h->launches += 1;
    } else {
        CUDA_OR_FAIL(h, cudaMemcpyAsync(h->psi[0], psi_dev, bytes, cudaMemcpyDefault, h->stream));
    }
    return after_set_state(h, next_traj);
}

ising_status ising_hmc_momenta(ising_hmc_t *h, uint64_t seed, int64_t traj, int chain0, int count,
                               double *out) {
    if (!h || !out) return ISING_EINVAL;
    if (traj < 0 || traj > (int64_t)0xfffffffe) return fail(h, ISING_EINVAL, "bad trajectory index");
    if (chain0 < 0 || count < 0 || chain0 + count > h->n_chains)
        return fail(h, ISING_EINVAL, "chain range out of bounds");
    if (is_dense_tc(h)) {
        CUDA_OR_FAIL(h, dense_momenta(h->dense, seed, (uint32_t)traj, h->stream, &h->launches));
    } else if (is_fused(h)) {
        FusedArgs a = fused_args(h);
        a.mode = MODE_MOMENTA;
        a.seed = seed;
        a.traj0 = (uint32_t)traj;
        a.chain0 = chain0;
        a.n_chains = chain0 + count;
        CUDA_OR_FAIL(h, launch_fused(h, a));
        h->launches += 1;
    } else {
        for (int c = chain0; c < chain0 + count; ++c) {
            PlainArgs a = plain_args(h, c);
            CUDA_OR_FAIL(h, plain_momenta(a, seed, (uint32_t)traj, h->stream, &h->launches));
        }
    }
    return ising_hmc_get_chains(h, ISING_STATE_P_END, chain0, count, out);
}

ising_status ising_hmc_set_eps(ising_hmc_t *h, const double *eps) {
    if (!h || !eps) return ISING_EINVAL;
    for (int c = 0; c < h->n_chains; ++c) {
        if (!(eps[c] > 0)) return fail(h, ISING_EINVAL, "eps[%d] must be > 0", c);
        h->params[c].eps = eps[c];
        h->params[c].epsf = (float)eps[c];
    }
    ising_status st = ising_hmc_sync(h);
    if (st != ISING_OK) return st;
    return upload_params(h);
}

ising_status ising_hmc_chain_params(const ising_hmc_t *h, double *out) {
    if (!h || !out) return ISING_EINVAL;
    for (int c = 0; c < h->n_chains; ++c) {
        out[3 * c + 0] = h->params[c].beta;
        out[3 * c + 1] = h->params[c].C;
        out[3 * c + 2] = h->params[c].eps;
    }
    return ISING_OK;
}

ising_status ising_hmc_get_state_native(ising_hmc_t *h, void *out) {
    if (!h || !out) return ISING_EINVAL;
    std::vector<ChainState> hs;
    ising_status st = fetch_states(h, hs);
    if (st != ISING_OK) return st;
    const size_t cb = (size_t)h->N * state_elem(h);
    for (int c = 0; c < h->n_chains; ++c) {
        const int b = is_fused(h) ? hs[c].start : 0;
        CUDA_OR_FAIL(h, cudaMemcpyAsync((char *)out + c * cb, (const char *)h->psi[b] + c * cb, cb,
                                        cudaMemcpyDefault, h->stream));
    }
    CUDA_OR_FAIL(h, cudaStreamSynchronize(h->stream));
    return ISING_OK;
}

int ising_hmc_state_elem_bytes(const ising_hmc_t *h) { return h ? (int)state_elem(h) : -1; }

int64_t ising_hmc_traj_index(const ising_hmc_t *h) { return h ? h->traj : -1; }
int64_t ising_hmc_n_sites(const ising_hmc_t *h) { return h ? h->N : -1; }
int ising_hmc_n_chains(const ising_hmc_t *h) { return h ? h->n_chains : -1; }
int64_t ising_hmc_device_bytes(const ising_hmc_t *h) { return h ? h->bytes : -1; }
int64_t ising_hmc_launch_count(const ising_hmc_t *h) { return h ? h->launches : -1; }

ising_status ising_hmc_selftest(int which, const void *in, void *out, int64_t n) {
    g_create_err[0] = 0;
    if (!in || !out || n < 0) return fail(nullptr, ISING_EINVAL, "selftest: bad arguments");
    if (n == 0) return ISING_OK;
    const size_t el = which == ISING_SELFTEST_TANH ? sizeof(float) : sizeof(double);
    if (which != ISING_SELFTEST_TANH && which != ISING_SELFTEST_LOG1PEXP)
        return fail(nullptr, ISING_EINVAL, "selftest: unknown function %d", which);
    void *din = nullptr, *dout = nullptr;
    float *dtab = nullptr;
    ising_status st = ISING_OK;
    if (cudaMalloc(&din, n * el) != cudaSuccess || cudaMalloc(&dout, n * el) != cudaSuccess) {
        st = fail(nullptr, ISING_ENOMEM, "selftest: device allocation failed");
    } else if (cudaMemcpy(din, in, n * el, cudaMemcpyHostToDevice) != cudaSuccess) {
        st = fail(nullptr, ISING_ECUDA, "selftest: upload failed");
    } else {
        cudaError_t e;
        if (which == ISING_SELFTEST_TANH) {
            e = launch_tanh_selftest((const float *)din, (float *)dout, n, 0);
        } else {
            std::vector<float> tab(4 * LOG1PEXP_NODES);
            build_log1pexp_table(tab.data());
            e = cudaMalloc(&dtab, tab.size() * sizeof(float));
            if (e == cudaSuccess)
                e = cudaMemcpy(dtab, tab.data(), tab.size() * sizeof(float), cudaMemcpyHostToDevice);
            if (e == cudaSuccess)
                e = launch_log1pexp_selftest((const double *)din, (double *)dout, n,
                                             reinterpret_cast<const float4 *>(dtab), 0);
        }
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e == cudaSuccess) e = cudaMemcpy(out, dout, n * el, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) st = fail(nullptr, ISING_ECUDA, "selftest: %s", cudaGetErrorString(e));
    }
    if (din) cudaFree(din);
    if (dout) cudaFree(dout);
    if (dtab) cudaFree(dtab);
    return st;
}

ising_status ising_hmc_set_launch(ising_hmc_t *h, int threads, int depth) {
    if (!h) return ISING_EINVAL;
    if (!is_fp32_lattice(h)) return fail(h, ISING_EINVAL, "launch shape applies to the FP32 lattice form");
    if (!fused_lattice_valid_split(h->g, threads, depth, h->cs))
        return fail(h, ISING_EINVAL, "invalid launch shape threads=%d depth=%d (%d CTAs per chain)",
                    threads, depth, h->cs);
    h->threads = threads;
    h->depth = depth;
    return ISING_OK;
}

ising_status ising_hmc_get_launch(const ising_hmc_t *h, int *threads, int *depth) {
    if (!h || !threads || !depth) return ISING_EINVAL;
    *threads = h->threads;
    *depth = h->depth;
    return ISING_OK;
}

ising_status ising_hmc_set_chain_split(ising_hmc_t *h, int ctas) {
    if (!h) return ISING_EINVAL;
    if (!is_fp32_lattice(h)) return fail(h, ISING_EINVAL, "chain split applies to the FP32 lattice form");
    if (!fused_lattice_valid_split(h->g, h->threads, h->depth, ctas))
        return fail(h, ISING_EINVAL, "invalid chain split %d (threads=%d depth=%d, %d planes)", ctas,
                    h->threads, h->depth, h->g.nplanes);
    h->cs = ctas;
    return ISING_OK;
}

int ising_hmc_get_chain_split(const ising_hmc_t *h) { return h ? h->cs : -1; }

ising_status ising_hmc_set_staging(ising_hmc_t *h, int mode) {
    if (!h) return ISING_EINVAL;
    if (!is_fp32_lattice(h)) return fail(h, ISING_EINVAL, "plane staging applies to the FP32 lattice form");
    if (mode < ISING_STAGING_AUTO || mode > ISING_STAGING_BULK)
        return fail(h, ISING_EINVAL, "unknown staging mode %d", mode);
    if (mode == ISING_STAGING_BULK && !(h->g.X % 4 == 0 && h->g.P % 4 == 0))
        return fail(h, ISING_EINVAL, "bulk staging needs rows of a multiple of 4 sites");
    h->staging = mode;
    return ISING_OK;
}

int ising_hmc_get_staging(const ising_hmc_t *h) { return h ? h->staging : -1; }

ising_status ising_hmc_dense_forces(ising_hmc_t *h, int n) {
    if (!h) return ISING_EINVAL;
    if (!is_dense_tc(h)) return fail(h, ISING_EINVAL, "dense_forces applies to the BF16 dense form");
    if (n < 0) return fail(h, ISING_EINVAL, "n must be >= 0");
    for (int i = 0; i < n; ++i) {
        const cudaError_t e = dense_force_once(h->dense, h->stream);
        h->launches += 2;
        if (e != cudaSuccess) return fail(h, ISING_ECUDA, "dense force: %s", cudaGetErrorString(e));
    }
    return ISING_OK;
}

// A temporary FP32 lattice handle with h's lattice, integrator and the
// parameters of h's first nt chains, on h's stream (for the autotuners: the
// handle's own chains never move).
static ising_status clone_for_tuning(ising_hmc *h, int nt, ising_hmc **out) {
    ising_hmc_config cfg{};
    cfg.kind = ISING_KIND_LATTICE;
    cfg.dim = h->dim;
    for (int d = 0; d < 3; ++d) cfg.L[d] = h->L[d];
    std::vector<double> beta(nt), C(nt), eps(nt), h0(nt);
    for (int c = 0; c < nt; ++c) {
        beta[c] = h->params[c].beta;
        C[c] = h->params[c].C;
        eps[c] = h->params[c].eps;
        h0[c] = h->params[c].hp / h->params[c].beta;
    }
    cfg.Jnn = h->params[0].bJ / h->params[0].beta;
    cfg.beta = beta[0];
    cfg.C = C[0];
    cfg.eps = eps[0];
    cfg.beta_chain = beta.data();
    cfg.C_chain = C.data();
    cfg.eps_chain = eps.data();
    cfg.h0_chain = h0.data();
    cfg.n_md = h->n_md;
    cfg.n_chains = nt;
    cfg.precision = ISING_PREC_FP32;
    cfg.integrator = h->integrator;
    cfg.stream = h->stream;
    ising_status st = ising_hmc_create(&cfg, out);
    if (st == ISING_OK) {
        (*out)->threads = h->threads;
        (*out)->depth = h->depth;
        (*out)->cs = h->cs;
        (*out)->staging = h->staging;
    }
    return st;
}

// Time of `reps` trajectories (after one untimed) of handle t, in ms per
// trajectory; negative if the launch failed.
static double time_trajectories(ising_hmc *t, int reps, cudaEvent_t e0, cudaEvent_t e1) {
    if (ising_hmc_trajectories(t, 1, 99) != ISING_OK) return -1.0;   // warm-up
    cudaEventRecord(e0, t->stream);
    if (ising_hmc_trajectories(t, reps, 99) != ISING_OK) return -1.0;
    cudaEventRecord(e1, t->stream);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
        cudaGetLastError();
        return -1.0;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    return ms / reps;
}

// Autotuner: time one trajectory of every valid (threads, depth) on a
// temporary copy of the handle's geometry and parameters (so the handle's own
// chains do not move) and keep the fastest; then try splitting every chain
// over 2, 4 and 8 CTAs at the best thread count and at 256..512 threads, every
// depth; then, if the staging is automatic, both staging modes at the result.
ising_status ising_hmc_autotune(ising_hmc_t *h, int reps, double *best_ms) {
    NvtxRange nvtx_range("ising_hmc_autotune");
    if (!h) return ISING_EINVAL;
    if (!is_fp32_lattice(h)) return fail(h, ISING_EINVAL, "autotune applies to the FP32 lattice form");
    if (reps < 1) reps = 1;
    ising_status st = ising_hmc_sync(h);
    if (st != ISING_OK) return st;
    // temporary handle: same lattice and first chains' parameters, at most 2 waves of CTAs
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int nt = std::min(h->n_chains, std::max(1, 2 * nsm));
    ising_hmc *t = nullptr;
    st = clone_for_tuning(h, nt, &t);
    if (st != ISING_OK) return fail(h, st, "autotune: %s", ising_hmc_last_create_error());
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = 1e300;
    int bt = h->threads, bd = h->depth, bc = 1;
    const int cand_t[] = {32, 64, 96, 128, 160, 192, 224, 256};
    const int cand_d[] = {1, 2, 4};
    const int cand_c[] = {2, 4, 8};
    t->cs = 1;
    for (int th : cand_t) {
        for (int dp : cand_d) {
            if (!fused_lattice_valid_launch(h->g, th, dp)) continue;
            t->threads = th;
            t->depth = dp;
            const double ms = time_trajectories(t, reps, e0, e1);
            if (ms > 0 && ms < best) {
                best = ms;
                bt = th;
                bd = dp;
            }
        }
    }
    const int th1 = bt;
    const int cand_ts[] = {th1, 256, 320, 384, 448, 512};
    for (int c : cand_c) {
        for (int i = 0; i < 6; ++i) {
            const int th = cand_ts[i];
            if (i > 0 && th == th1) continue;
            for (int dp : cand_d) {
                if (!fused_lattice_valid_split(h->g, th, dp, c)) continue;
                t->threads = th;
                t->depth = dp;
                t->cs = c;
                const double ms = time_trajectories(t, reps, e0, e1);
                if (ms > 0 && ms < best) {
                    best = ms;
                    bt = th;
                    bd = dp;
                    bc = c;
                }
            }
        }
    }
    // plane staging (when left to the automatic choice): both modes timed at
    // the chosen shape, back to back
    int stg = h->staging;
    if (h->staging == ISING_STAGING_AUTO && h->g.X % 4 == 0 && h->g.P % 4 == 0) {
        t->threads = bt;
        t->depth = bd;
        t->cs = bc;
        double ms_mode[2] = {0.0, 0.0};
        const int modes[2] = {ISING_STAGING_THREADS, ISING_STAGING_BULK};
        for (int i = 0; i < 2; ++i) {
            t->staging = modes[i];
            ms_mode[i] = time_trajectories(t, reps, e0, e1);
        }
        if (ms_mode[0] > 0 && ms_mode[1] > 0) {
            const int i = ms_mode[1] < ms_mode[0] ? 1 : 0;
            stg = modes[i];
            best = ms_mode[i];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ising_hmc_destroy(t);
    h->threads = bt;
    h->depth = bd;
    h->cs = bc;
    h->staging = stg;
    if (best_ms) *best_ms = best;
    return ISING_OK;
}

// ---------------------------------------------------------------------------
// Groups: several FP32 lattice handles (any mix of lattice sizes) advanced by
// one CUDA-graph launch with one kernel node per member, nodes independent so
// they run concurrently.
// ---------------------------------------------------------------------------
struct ising_group {
    std::vector<ising_hmc *> m;
    std::vector<FusedArgs> args;
    std::vector<std::array<void *, 2>> argv;
    std::vector<cudaGraphNode_t> nodes;
    std::vector<int> shape;  // threads, depth, CTAs per chain, bulk staging of every member
                             // at instantiation
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    int64_t launches = 0;
    char err[512] = {0};
};

static ising_status gfail(ising_group *g, ising_status st, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g ? g->err : g_create_err, 512, fmt, ap);
    va_end(ap);
    return st;
}

static void group_free_graph(ising_group *g) {
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    g->exec = nullptr;
    g->graph = nullptr;
    g->nodes.clear();
}

static ising_status group_build_graph(ising_group *g) {
    group_free_graph(g);
    const size_t n = g->m.size();
    g->args.resize(n);
    g->argv.resize(n);
    g->nodes.resize(n);
    g->shape.assign(4 * n, 0);
    if (cudaGraphCreate(&g->graph, 0) != cudaSuccess) return gfail(g, ISING_ECUDA, "graph create failed");
    // nodes are added largest work first: independent nodes start roughly in
    // the order they were added, and the longest members are the critical path
    std::vector<size_t> order(n);
    for (size_t i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) {
        const double wa = (double)g->m[a]->N * g->m[a]->n_chains * g->m[a]->sched.n_pass;
        const double wb = (double)g->m[b]->N * g->m[b]->n_chains * g->m[b]->sched.n_pass;
        return wa > wb;
    });
    for (size_t i : order) {
        ising_hmc *h = g->m[i];
        g->args[i] = fused_args(h);
        g->args[i].mode = MODE_TRAJ;
        g->args[i].n_traj = 1;
        g->argv[i] = {&g->args[i], &h->sched};
        cudaKernelNodeParams np;
        cudaError_t e = fused_lattice_node(g->args[i], h->threads, h->depth, &np, g->argv[i].data());
        if (e == cudaSuccess) e = cudaGraphAddKernelNode(&g->nodes[i], g->graph, nullptr, 0, &np);
        if (e == cudaSuccess && h->cs > 1) e = fused_lattice_node_cluster(g->nodes[i], h->cs);
        if (e != cudaSuccess) return gfail(g, ISING_ECUDA, "graph node: %s", cudaGetErrorString(e));
        g->shape[4 * i] = h->threads;
        g->shape[4 * i + 1] = h->depth;
        g->shape[4 * i + 2] = h->cs;
        g->shape[4 * i + 3] = staging_bulk(h);
    }
    cudaError_t e = cudaGraphInstantiate(&g->exec, g->graph, 0);
    if (e != cudaSuccess) return gfail(g, ISING_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    return ISING_OK;
}

ising_status ising_group_create(ising_hmc_t *const *members, int n, ising_group_t **out) {
    g_create_err[0] = 0;
    if (!members || n < 1 || !out) return gfail(nullptr, ISING_EINVAL, "group: need members");
    *out = nullptr;
    ising_group *g = new (std::nothrow) ising_group();
    if (!g) return gfail(nullptr, ISING_ENOMEM, "group: host allocation failed");
    for (int i = 0; i < n; ++i) {
        if (!members[i] || !is_fp32_lattice(members[i])) {
            delete g;
            return gfail(nullptr, ISING_EINVAL, "group member %d is not an FP32 lattice handle", i);
        }
        for (int j = 0; j < i; ++j)
            if (members[j] == members[i]) {
                delete g;
                return gfail(nullptr, ISING_EINVAL, "group member %d repeated", i);
            }
        g->m.push_back(members[i]);
    }
    if (cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&g->ev, cudaEventDisableTiming) != cudaSuccess) {
        delete g;
        return gfail(nullptr, ISING_ECUDA, "group: stream/event creation failed");
    }
    ising_status st = group_build_graph(g);
    if (st != ISING_OK) {
        std::snprintf(g_create_err, sizeof g_create_err, "%s", g->err);
        group_free_graph(g);
        cudaEventDestroy(g->ev);
        cudaStreamDestroy(g->stream);
        delete g;
        return st;
    }
    *out = g;
    return ISING_OK;
}

ising_status ising_group_trajectories(ising_group_t *g, int64_t n, uint64_t seed) {
    if (!g) return ISING_EINVAL;
    std::vector<uint64_t> seeds(g->m.size(), seed);
    return ising_group_trajectories_seeds(g, n, seeds.data());
}

ising_status ising_group_trajectories_seeds(ising_group_t *g, int64_t n, const uint64_t *seeds) {
    NvtxRange nvtx_range("ising_group_trajectories");
    if (!g || !seeds) return ISING_EINVAL;
    if (n < 0) return gfail(g, ISING_EINVAL, "n must be >= 0");
    if (n == 0) return ISING_OK;
    // rebuild if a member's launch shape changed (autotune, set_launch)
    for (size_t i = 0; i < g->m.size(); ++i)
        if (g->shape[4 * i] != g->m[i]->threads || g->shape[4 * i + 1] != g->m[i]->depth ||
            g->shape[4 * i + 2] != g->m[i]->cs || g->shape[4 * i + 3] != staging_bulk(g->m[i])) {
            ising_status st = group_build_graph(g);
            if (st != ISING_OK) return st;
            break;
        }
    // trajectories per graph launch: bounded work per kernel, like the single-handle path
    int64_t per = 4096;
    for (ising_hmc *h : g->m) {
        const double work = (double)h->N * h->n_chains * h->sched.n_pass;
        per = std::min<int64_t>(per, (int64_t)std::max(1.0, std::floor(4.0e9 / std::max(work, 1.0))));
        if (h->traj + n > (int64_t)0xfffffffe) return gfail(g, ISING_EINVAL, "trajectory counter overflow");
    }
    // order after work already queued on the members' streams
    for (ising_hmc *h : g->m) {
        if (cudaEventRecord(g->ev, h->stream) != cudaSuccess ||
            cudaStreamWaitEvent(g->stream, g->ev, 0) != cudaSuccess)
            return gfail(g, ISING_ECUDA, "group: stream ordering failed");
    }
    int64_t done = 0;
    while (done < n) {
        const int64_t k = std::min(per, n - done);
        for (size_t i = 0; i < g->m.size(); ++i) {
            ising_hmc *h = g->m[i];
            g->args[i] = fused_args(h);
            g->args[i].mode = MODE_TRAJ;
            g->args[i].seed = seeds[i];
            g->args[i].traj0 = (uint32_t)(h->traj + done);
            g->args[i].n_traj = (int)k;
            g->args[i].eval_start = done == 0 && h->eval_pending;
            cudaKernelNodeParams np;
            cudaError_t e = fused_lattice_node(g->args[i], h->threads, h->depth, &np, g->argv[i].data());
            if (e == cudaSuccess) e = cudaGraphExecKernelNodeSetParams(g->exec, g->nodes[i], &np);
            if (e != cudaSuccess) return gfail(g, ISING_ECUDA, "graph update: %s", cudaGetErrorString(e));
        }
        cudaError_t e = cudaGraphLaunch(g->exec, g->stream);
        if (e != cudaSuccess) return gfail(g, ISING_ECUDA, "graph launch: %s", cudaGetErrorString(e));
        g->launches += 1;
        done += k;
    }
    for (ising_hmc *h : g->m) {
        h->traj += n;
        h->launches += (n + per - 1) / per;
        h->eval_pending = false;
    }
    // members' later work waits for the group's
    if (cudaEventRecord(g->ev, g->stream) != cudaSuccess) return gfail(g, ISING_ECUDA, "group: event");
    for (ising_hmc *h : g->m)
        if (cudaStreamWaitEvent(h->stream, g->ev, 0) != cudaSuccess)
            return gfail(g, ISING_ECUDA, "group: stream ordering failed");
    return ISING_OK;
}

// Group autotuner: the members' chains are split over CTAs by what the
// whole mixed launch gains, not what a size gains alone (a size that fills
// the GPU alone competes with the others in the group).  On temporary copies
// of every member (all their chains, same launch shapes), one member at a
// time, largest work first, each split in {1, 2, 4, 8} that fits is timed on
// the whole group's launch and the fastest kept; two rounds.
ising_status ising_group_autotune(ising_group_t *g, int reps, double *best_ms) {
    NvtxRange nvtx_range("ising_group_autotune");
    if (!g) return ISING_EINVAL;
    if (reps < 1) reps = 1;
    ising_status st = ising_group_sync(g);
    if (st != ISING_OK) return st;
    const size_t n = g->m.size();
    int64_t need = 0;
    for (ising_hmc *h : g->m) need += h->bytes;
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess || (double)need > 0.8 * (double)fr)
        return gfail(g, ISING_ENOMEM, "group autotune: temporary copies need %lld bytes",
                     (long long)need);
    std::vector<ising_hmc *> tmp(n, nullptr);
    ising_group *tg = nullptr;
    auto cleanup = [&]() {
        if (tg) ising_group_destroy(tg);
        for (ising_hmc *t : tmp)
            if (t) ising_hmc_destroy(t);
    };
    for (size_t i = 0; i < n; ++i) {
        st = clone_for_tuning(g->m[i], g->m[i]->n_chains, &tmp[i]);
        if (st != ISING_OK) {
            cleanup();
            return gfail(g, st, "group autotune: %s", ising_hmc_last_create_error());
        }
    }
    st = ising_group_create(tmp.data(), (int)n, &tg);
    if (st != ISING_OK) {
        cleanup();
        return gfail(g, st, "group autotune: %s", g_create_err);
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // the better of two timings of `reps` group trajectories (after one untimed)
    auto time_group = [&]() -> double {
        if (ising_group_trajectories(tg, 1, 99) != ISING_OK) return -1.0;
        double best_t = -1.0;
        for (int rep = 0; rep < 2; ++rep) {
            cudaEventRecord(e0, tg->stream);
            if (ising_group_trajectories(tg, reps, 99) != ISING_OK) return -1.0;
            cudaEventRecord(e1, tg->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                cudaGetLastError();
                return -1.0;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (best_t < 0 || ms / reps < best_t) best_t = ms / reps;
        }
        return best_t;
    };
    std::vector<size_t> order(n);
    for (size_t i = 0; i < n; ++i) order[i] = i;
    std::sort(order.begin(), order.end(), [&](size_t a, size_t b) {
        const double wa = (double)g->m[a]->N * g->m[a]->n_chains * g->m[a]->sched.n_pass;
        const double wb = (double)g->m[b]->N * g->m[b]->n_chains * g->m[b]->sched.n_pass;
        return wa > wb;
    });
    // start from the better of the members' current splits and no splits at all
    double best = time_group();
    {
        std::vector<int> cur(n);
        bool any = false, unsplit_ok = true;
        for (size_t i = 0; i < n; ++i) {
            cur[i] = tmp[i]->cs;
            any |= cur[i] != 1;
            unsplit_ok &= fused_lattice_valid_split(tmp[i]->g, tmp[i]->threads, tmp[i]->depth, 1) != 0;
        }
        if (any && unsplit_ok) {
            for (size_t i = 0; i < n; ++i) tmp[i]->cs = 1;
            const double t1 = time_group();
            if (t1 > 0 && (best < 0 || t1 < best)) best = t1;
            else
                for (size_t i = 0; i < n; ++i) tmp[i]->cs = cur[i];
        }
    }
    for (int round = 0; round < 2; ++round) {
        for (size_t i : order) {
            ising_hmc *t = tmp[i];
            const int keep = t->cs;
            int bc = keep;
            for (int c : {1, 2, 4, 8}) {
                if (c == keep || !fused_lattice_valid_split(t->g, t->threads, t->depth, c)) continue;
                t->cs = c;
                const double ms = time_group();
                if (ms > 0 && (best < 0 || ms < best)) {
                    best = ms;
                    bc = c;
                }
            }
            t->cs = bc;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (size_t i = 0; i < n; ++i) g->m[i]->cs = tmp[i]->cs;
    cleanup();
    if (best_ms) *best_ms = best;
    return best > 0 ? ISING_OK : gfail(g, ISING_ECUDA, "group autotune: no launch succeeded");
}

ising_status ising_group_sync(ising_group_t *g) {
    if (!g) return ISING_EINVAL;
    if (cudaStreamSynchronize(g->stream) != cudaSuccess)
        return gfail(g, ISING_ECUDA, "group sync: %s", cudaGetErrorString(cudaGetLastError()));
    for (ising_hmc *h : g->m) {
        ising_status st = ising_hmc_sync(h);
        if (st != ISING_OK) return gfail(g, st, "member: %s", h->err);
    }
    return ISING_OK;
}

int64_t ising_group_launch_count(const ising_group_t *g) { return g ? g->launches : -1; }

void *ising_group_stream(const ising_group_t *g) { return g ? (void *)g->stream : nullptr; }

const char *ising_group_last_error(const ising_group_t *g) { return g ? g->err : g_create_err; }

void ising_group_destroy(ising_group_t *g) {
    if (!g) return;
    if (g->stream) cudaStreamSynchronize(g->stream);
    group_free_graph(g);
    if (g->ev) cudaEventDestroy(g->ev);
    if (g->stream) cudaStreamDestroy(g->stream);
    delete g;
}

ising_status ising_hmc_selftest_gemm(int M, int N, int K, const uint16_t *A, const uint16_t *B,
                                     float *D) {
    g_create_err[0] = 0;
    if (!A || !B || !D || M <= 0 || N <= 0 || K <= 0 || M % 128 || N % 128 || K % 64)
        return fail(nullptr, ISING_EINVAL, "selftest_gemm: M, N multiples of 128, K of 64");
    void *dA = nullptr, *dB = nullptr, *dD = nullptr;
    int *derr = nullptr;
    ising_status st = ISING_OK;
    cudaError_t e = cudaMalloc(&dA, (size_t)M * K * 2);
    if (e == cudaSuccess) e = cudaMalloc(&dB, (size_t)N * K * 2);
    if (e == cudaSuccess) e = cudaMalloc(&dD, (size_t)M * N * 4);
    if (e == cudaSuccess) e = cudaMalloc(&derr, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(derr, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(dA, A, (size_t)M * K * 2, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dB, B, (size_t)N * K * 2, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_gemm_store(dA, dB, (float *)dD, M, N, K, derr, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(D, dD, (size_t)M * N * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) st = fail(nullptr, ISING_ECUDA, "selftest_gemm: %s", cudaGetErrorString(e));
    else if (herr) st = fail(nullptr, ISING_ETIMEOUT, "selftest_gemm: a pipeline wait ran out");
    cudaFree(dA);
    cudaFree(dB);
    cudaFree(dD);
    cudaFree(derr);
    return st;
}

void ising_hmc_inject_alloc_failure(int64_t k) { g_fail_alloc_in.store(k > 0 ? k : 0); }

ising_status ising_hmc_inject_device_error(ising_hmc_t *h, int bits) {
    if (!h) return ISING_EINVAL;
    if (bits & ~(KERR_TIMEOUT | KERR_BOUNDS)) return fail(h, ISING_EINVAL, "unknown error bits %d", bits);
    // OR into the word on the device, ordered after the handle's queued work
    int cur = 0;
    ising_status st = ISING_OK;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess ||
        cudaMemcpy(&cur, h->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(h, ISING_ECUDA, "inject: %s", cudaGetErrorString(cudaGetLastError()));
    cur |= bits;
    if (cudaMemcpy(h->d_err, &cur, sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
        st = fail(h, ISING_ECUDA, "inject: %s", cudaGetErrorString(cudaGetLastError()));
    return st;
}

void ising_hmc_destroy(ising_hmc_t *h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    free_all(h);
    delete h;
}

const char *ising_hmc_last_error(const ising_hmc_t *h) { return h ? h->err : g_create_err; }

}  // extern "C"
