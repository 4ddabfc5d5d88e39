/*
 * ising_hmc.h -- C ABI of the GB300 (sm_103a) Hybrid Monte Carlo library for
 * the Ising model in its Hubbard-Stratonovich (HS) auxiliary-field form
 * (Ostmeyer, Berkowitz, Luu, Petschlies, Pittler, "The Ising Model with Hybrid
 * Monte Carlo", arXiv:1912.03278).
 *
 * The method (Sec. 2, Eqs. absorb_beta .. phi_psi_substitution; Sec. 3):
 * with A = beta*J*K + C*1 positive definite (K the connectivity, C the shift of
 * Sec. 2) and h' = beta*h, the spins are summed out and the field psi carries
 *     S(psi) = 1/2 psi.A.psi - sum_i log 2cosh((A psi)_i + h'_i).
 * A trajectory draws momenta p ~ N(0,1) (Sec. 3, Eq. momentum distribution),
 * integrates dpsi/dt = p, dp/dt = F(psi) = A (tanh(A psi + h') - psi) with a
 * symmetric symplectic integrator for one unit of MD time, and accepts the end
 * point with probability min(1, exp(-dH)), H = 1/2 p.p + S(psi) (Sec. 3).
 *
 * Parametrisation.  The paper writes Kt = K + C_p*1 and phi = sqrt(J') Kt psi_p
 * - h' with J' = beta*J.  This library uses phi = A psi, i.e. C = J'*C_p,
 * psi = psi_p/sqrt(J') - A^-1 h', eps = eps_p/sqrt(J'); the two generate the
 * same Markov chain (equal dH, equal accept decisions).
 *
 * Conventions for every entry point:
 *  - No call aborts, prints or throws.  Each returns an ising_status; on error
 *    ising_hmc_last_error(handle) describes it (handle-less errors of
 *    ising_hmc_create are reported by ising_hmc_last_create_error()).
 *  - Host pointers are only read during the call (inputs are copied); the
 *    caller keeps ownership of everything it passes.  The handle owns all the
 *    device memory it allocates and frees it in ising_hmc_destroy.
 *  - Work is queued on the handle's CUDA stream (the caller's stream if one was
 *    given).  Calls that return host data synchronise that stream.
 *  - Arrays of chain state are chain-major: element [c*N + i] is site i of
 *    chain c; lattice site i = x + L0*(y + L1*z).
 *  - Philox4x32-10 (Salmon et al., SC'11) supplies every random number from a
 *    counter (index, trajectory, chain, purpose) and the key (seed lo, seed hi),
 *    so results depend only on (seed, chain, trajectory index), never on the
 *    launch shape or on how trajectories are split across calls.
 */
#ifndef ISING_HMC_H
#define ISING_HMC_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ISING_OK = 0,
    ISING_EINVAL = 1,   /* invalid argument or configuration                 */
    ISING_ENOTPD = 2,   /* C too small: A not positive definite (Sec. 2)     */
    ISING_ENOMEM = 3,   /* device or host allocation failed                  */
    ISING_ECUDA = 4,    /* a CUDA runtime call failed                        */
    ISING_ETIMEOUT = 5, /* a bounded device-side wait gave up                */
    ISING_EBUSY = 6     /* resource in use (e.g. a group already running)    */
} ising_status;

/* Kinds of coupling (Sec. 2: the Hamiltonian with connectivity K):
 *  LATTICE   periodic hypercubic lattice, nearest neighbours, coupling Jnn;
 *  DENSE     arbitrary symmetric N x N couplings J (K absorbed into J);
 *  INFINITE  the all-to-all ("infinite-range") model of the appendix:
 *            K_ij = 1/N for i != j, coupling Jnn, N = n_sites; no matrix is
 *            stored, every product with A costs O(N).  FP32 form only. */
enum { ISING_KIND_LATTICE = 0, ISING_KIND_DENSE = 1, ISING_KIND_INFINITE = 2 };

enum {
    ISING_PREC_PLAIN_FP64 = 0, /* FP64 state and force, one chain per launch, unfused */
    ISING_PREC_FP32 = 1,       /* FP32 state and force, fused, FP64-accurate action  */
    ISING_PREC_BF16 = 2,       /* dense only: BF16 tensor-core force, FP32 state      */
    ISING_PREC_FP8 = 3         /* dense only: FP8 e4m3 force with per-row scales      */
};

enum { ISING_INTEGRATOR_LEAPFROG = 0, ISING_INTEGRATOR_OMELYAN = 1 };

typedef struct {
    int kind;             /* ISING_KIND_LATTICE, ISING_KIND_DENSE or ISING_KIND_INFINITE */
    int dim;              /* lattice: 1..3                                              */
    int L[3];             /* lattice extents, each >= 3 (L = 2 would double the bonds)  */
    int64_t n_sites;      /* dense, infinite: N (ignored for lattices)                  */
    const double *J;      /* dense: host N*N row-major, symmetric, J_ii = 0; copied     */
    double Jnn;           /* lattice nearest-neighbour coupling J (Sec. 2); infinite:
                             the all-to-all coupling J (each pair couples with J/N)    */
    const double *h;      /* host per-site field h_i (N values) or NULL; copied         */
    double h0;            /* uniform field when h == NULL                               */
    double beta, C, eps;  /* defaults for every chain; C in the units of A above;
                             C <= 0 selects the default shift (see ising_hmc_create)   */
    const double *beta_chain; /* optional host arrays of n_chains values overriding    */
    const double *C_chain;    /*   beta, C, eps and h0 per chain (NULL = use the scalar) */
    const double *eps_chain;
    const double *h0_chain;
    int n_md;             /* MD steps per trajectory (leapfrog: n_md drifts)            */
    int n_chains;         /* independent Markov chains                                  */
    int n_therm;          /* trajectories with index < n_therm are not measured (Sec. 3) */
    int precision;        /* ISING_PREC_*                                               */
    int integrator;       /* ISING_INTEGRATOR_*                                         */
    int flip_every;       /* >0: global sign-flip proposal after every k-th trajectory
                             (every form; the tensor-core dense forms evaluate the
                             current configuration's A psi once more for it)       */
    void *stream;         /* cudaStream_t to queue work on, or NULL for an own stream   */
} ising_hmc_config;

/* Per-chain sums, chain-major, ISING_NSUMS doubles per chain, in this order. */
enum {
    ISING_SUM_NMEAS = 0, ISING_SUM_NACC, ISING_SUM_M, ISING_SUM_M2, ISING_SUM_E, ISING_SUM_E2,
    ISING_SUM_ABSM, ISING_SUM_ABSM2, ISING_SUM_DH, ISING_SUM_EXPMDH, ISING_NSUMS
};

/* Record of a chain's most recent trajectory, ISING_NREC doubles per chain. */
enum {
    ISING_REC_DH = 0, ISING_REC_LOGU, ISING_REC_ACCEPTED, ISING_REC_K0, ISING_REC_S0,
    ISING_REC_K1, ISING_REC_S1, ISING_REC_FLIPPED, ISING_NREC
};

typedef struct {
    double m, m_err;          /* <m>, Sec. 4 (E[s|psi] estimator, mean tanh(A psi + h'))  */
    double abs_m, abs_m_err;  /* <|m|> from one conditional spin draw per configuration   */
    double E, E_err;          /* <beta*eps> = C/2 - <a.t>/(2N) - <h'.t>/N (Sec. 4)        */
    double acceptance;
    double mean_dH;
    double mean_exp_mdH, exp_mdH_err; /* Creutz: <exp(-dH)> = 1                            */
    int64_t n_traj;           /* trajectories run so far (per chain)                      */
    int64_t n_meas;           /* measured trajectories, summed over chains                */
} ising_obs;

typedef struct ising_hmc ising_hmc_t;

/* Create a simulation: validates the model, allocates device state for
 * n_chains chains, uploads couplings and fields, and sets psi = 0 with its
 * action S(0) computed on the device.
 * Validation (Sec. 2, spectrum bound and shift): A is positive definite iff C
 * exceeds b = -lambda_min(beta*J*K).  Lattice: b = beta*|J|*2*dim (the bound
 * the paper uses); dense: b = beta*|lambda_min(J)|, lambda_min estimated by
 * Lanczos with full reorthogonalisation (min(N, 96) steps, FP64, products on
 * the device); infinite: b = beta*J/N for J >= 0 and beta*|J|*(N-1)/N for
 * J < 0 (the exact extreme eigenvalues), and 2 <= N <= 2^31.  A chain whose C
 * is <= 0 gets the default shift C = b + 0.1 (the shift of the paper's
 * workloads); ising_hmc_chain_params reports the C every chain uses.  A
 * positive C <= b is rejected with ENOTPD.
 * Errors: EINVAL (bad sizes/kinds/precision for the kind), ENOTPD, ENOMEM, ECUDA. */
ising_status ising_hmc_create(const ising_hmc_config *cfg, ising_hmc_t **out);

/* Run n trajectories on every chain (Sec. 3 algorithm: momentum refresh, MD,
 * Metropolis test, optional sign flip, measurement after n_therm).  The
 * trajectory counter persists: trajectories(a, s) then trajectories(b, s)
 * equals trajectories(a + b, s) bit for bit.  Asynchronous: returns once the
 * work is queued.  Errors: EINVAL (n < 0), ECUDA. */
ising_status ising_hmc_trajectories(ising_hmc_t *h, int64_t n, uint64_t seed);

/* Observables averaged over all chains of the handle (Sec. 4 estimators);
 * errors are the standard error of the per-chain means when n_chains > 1, and
 * the naive sigma/sqrt(n) of the single chain otherwise (no autocorrelation
 * correction).  Synchronises.  Errors: ECUDA, ETIMEOUT. */
ising_status ising_hmc_observables(ising_hmc_t *h, ising_obs *out);

/* Per-chain sums (ISING_NSUMS doubles per chain) into out[n_chains*ISING_NSUMS]. */
ising_status ising_hmc_chain_sums(ising_hmc_t *h, double *out);

/* Per-chain record of the most recent trajectory (ISING_NREC doubles per chain). */
ising_status ising_hmc_last_records(ising_hmc_t *h, double *out);

/* Zero the per-chain sums (e.g. after an equilibration phase). */
ising_status ising_hmc_reset_sums(ising_hmc_t *h);

enum { ISING_STATE_PSI = 0, ISING_STATE_PSI_PROPOSAL = 1, ISING_STATE_P_END = 2 };

/* Copy chain state to host out[n_chains*N] as FP64: the current configuration,
 * the most recent proposal (end of the last trajectory, accepted or not), or
 * the momenta at the end of the last trajectory.  Synchronises. */
ising_status ising_hmc_get_state(ising_hmc_t *h, int which, double *out);

/* Same for chains [chain0, chain0+count) only, into host out[count*N]. */
ising_status ising_hmc_get_chains(ising_hmc_t *h, int which, int chain0, int count, double *out);

/* Set every chain's configuration from host psi[n_chains*N] (rounded to the
 * state precision), set the index of the next trajectory, and have S and the
 * observables of the new configurations computed on the device: by the next
 * trajectory's first force pass in the FP32 lattice form (which reads every
 * site and its neighbours anyway: no extra sweep, same values), during the
 * call in the other forms.  Returns once the copy is complete (the caller may
 * reuse its buffer).  Checkpoint / resume: get_state + the trajectory index +
 * the sums restore a run exactly. */
ising_status ising_hmc_set_state(ising_hmc_t *h, const double *psi, int64_t next_traj);

/* Same from a buffer in the state precision (FP64 for the plain form, FP32
 * otherwise), chain-major, in device memory or in (preferably pinned) host
 * memory: the copy uses unified addressing.  Bytes read:
 * n_chains*N*ising_hmc_state_elem_bytes(h). */
ising_status ising_hmc_set_state_native(ising_hmc_t *h, const void *psi, int64_t next_traj);

/* Copy the current configurations, in the state precision, to a device or
 * host buffer of n_chains*N elements.  Synchronises. */
ising_status ising_hmc_get_state_native(ising_hmc_t *h, void *out);

/* Bytes per state element: 8 (plain FP64 form) or 4. */
int ising_hmc_state_elem_bytes(const ising_hmc_t *h);

/* Restore per-chain sums (checkpoint/resume), host in[n_chains*ISING_NSUMS]. */
ising_status ising_hmc_set_sums(ising_hmc_t *h, const double *in);

/* The momenta the library draws for trajectory traj (Sec. 3, momentum
 * refresh), computed by the same device code as the trajectories, for chains
 * [chain0, chain0+count) into host out[count*N] as FP64.  Overwrites the
 * stored end-of-trajectory momenta.  For checks on the GPU's own MD end points. */
ising_status ising_hmc_momenta(ising_hmc_t *h, uint64_t seed, int64_t traj, int chain0, int count,
                               double *out);

/* Replace the per-chain step sizes (host eps[n_chains]); used by the step-size
 * tuner during equilibration only. */
ising_status ising_hmc_set_eps(ising_hmc_t *h, const double *eps);

/* Per-chain parameters as the handle uses them, host out[n_chains*3]:
 * (beta, C, eps) for every chain -- C after the default of ising_hmc_create
 * was applied (Sec. 2, shift), eps after any ising_hmc_set_eps.
 * Errors: EINVAL (null handle or pointer). */
ising_status ising_hmc_chain_params(const ising_hmc_t *h, double *out);

/* Index of the next trajectory. */
int64_t ising_hmc_traj_index(const ising_hmc_t *h);

/* Number of sites per chain and number of chains. */
int64_t ising_hmc_n_sites(const ising_hmc_t *h);
int ising_hmc_n_chains(const ising_hmc_t *h);

/* Bytes of device memory the handle holds. */
int64_t ising_hmc_device_bytes(const ising_hmc_t *h);

/* Device memory a configuration would need, without creating it (admission). */
int64_t ising_hmc_estimate_bytes(const ising_hmc_config *cfg);

/* Kernel launches queued by this handle so far (for launch accounting). */
int64_t ising_hmc_launch_count(const ising_hmc_t *h);

/* Synchronise the handle's stream; ETIMEOUT if a device wait gave up. */
ising_status ising_hmc_sync(ising_hmc_t *h);

/* Launch shape of the fused FP32 lattice kernel: threads per CTA (a multiple
 * of 32, at most 4 float4 vectors of a plane per thread; 32..256 with one CTA
 * per chain, up to 512 when chains are split over CTAs, see
 * ising_hmc_set_chain_split) and the prefetch depth in planes (1, 2 or 4; the
 * shared-memory rings must fit).  EINVAL for other forms or invalid shapes. */
ising_status ising_hmc_set_launch(ising_hmc_t *h, int threads, int depth);
ising_status ising_hmc_get_launch(const ising_hmc_t *h, int *threads, int *depth);

/* CTAs per chain of the fused FP32 lattice kernel (1, 2, 4 or 8; default 1):
 * with ctas > 1 every chain runs on a thread-block cluster of that many CTAs,
 * each streaming a slab of the chain's planes (2D rows, 3D xy-slabs; at
 * least two planes per slab), so a few large chains fill the GPU.  The CTAs
 * meet at one cluster barrier per force evaluation and add their per-chain
 * sums in rank order: psi and p are bit for bit those of ctas = 1, the FP64
 * sums (action, energies, estimators) equal them to rounding; for a given
 * split, results are reproducible and independent of how trajectories are
 * split across calls.  EINVAL for other forms, 1D lattices, too few planes,
 * or a cluster the device cannot hold at the current launch shape. */
ising_status ising_hmc_set_chain_split(ising_hmc_t *h, int ctas);
int ising_hmc_get_chain_split(const ising_hmc_t *h);

/* How the fused FP32 lattice kernel stages psi and p planes into its
 * shared-memory rings (Sec. 3's force evaluation streams the lattice plane by
 * plane): ISING_STAGING_THREADS, every thread copies its share of a plane
 * with cp.async; ISING_STAGING_BULK, one lane issues each plane as a bulk
 * copy completing on an mbarrier (planes of whole 16-byte vectors: rows of a
 * multiple of 4 sites); ISING_STAGING_AUTO (default), bulk for planes of at
 * least 4 KB.  Results are bit for bit the same in every mode.  EINVAL for
 * other forms, unknown modes, or bulk on rows that are not a multiple of 4. */
enum { ISING_STAGING_AUTO = 0, ISING_STAGING_THREADS = 1, ISING_STAGING_BULK = 2 };
ising_status ising_hmc_set_staging(ising_hmc_t *h, int mode);
int ising_hmc_get_staging(const ising_hmc_t *h);

/* Autotuner: times `reps` trajectories for every valid launch shape on a
 * temporary handle with the same lattice and the first chains' parameters
 * (the handle's own chains are not advanced), keeps the fastest shape, and
 * returns its time per trajectory in *best_ms (may be NULL).  The search
 * covers threads and depth at one CTA per chain, then chain splits of 2, 4
 * and 8 CTAs at the best thread count, then (if the plane staging is
 * ISING_STAGING_AUTO and the rows allow bulk copies) both staging modes at
 * the chosen shape, setting the faster one explicitly.  Allocates the
 * temporary handle; synchronises. */
ising_status ising_hmc_autotune(ising_hmc_t *h, int reps, double *best_ms);

/* Groups: FP32 lattice handles of any mix of lattice sizes advanced together
 * by one CUDA-graph launch per call (one kernel node per member, the nodes
 * independent so they run concurrently on the device).  The graph is built
 * once and its nodes' parameters (trajectory index, count, seed) are updated
 * per call; it is rebuilt if a member's launch shape changes.  A group does
 * not own its members; destroy the group before them.  Work already queued on
 * a member's stream runs before the group's, and later member work after it. */
typedef struct ising_group ising_group_t;
ising_status ising_group_create(ising_hmc_t *const *members, int n, ising_group_t **out);
/* n trajectories of every chain of every member (same semantics as
 * ising_hmc_trajectories per member).  Asynchronous. */
ising_status ising_group_trajectories(ising_group_t *g, int64_t n, uint64_t seed);
/* Same with one seed per member (seeds[i] for the i-th member). */
ising_status ising_group_trajectories_seeds(ising_group_t *g, int64_t n, const uint64_t *seeds);

/* Group autotuner: picks every member's chain split (CTAs per chain, see
 * ising_hmc_set_chain_split) for the fastest launch of the whole group, by
 * timing `reps` group trajectories per candidate (twice, the better time
 * kept) on temporary copies of the members (all their chains, their current
 * launch shapes; the members' chains are not advanced).  Greedy from the
 * better of the current splits and none: members in order of work, each
 * split in {1, 2, 4, 8} that fits, two rounds.  Sets the members' splits; *best_ms
 * (may be NULL) gets the time per group trajectory.  Allocates the copies
 * (ENOMEM if they would take more than 80% of the free device memory);
 * synchronises. */
ising_status ising_group_autotune(ising_group_t *g, int reps, double *best_ms);
ising_status ising_group_sync(ising_group_t *g);
int64_t ising_group_launch_count(const ising_group_t *g);   /* graph launches so far */
void *ising_group_stream(const ising_group_t *g);           /* cudaStream_t of the launches */
const char *ising_group_last_error(const ising_group_t *g);
void ising_group_destroy(ising_group_t *g);

/* Serving: a continuous-batching request loop.  A server owns an admission
 * thread and a worker thread on the current device.  Requests (a
 * configuration as for ising_hmc_create, a number of trajectories and a seed)
 * are queued from any host thread and admitted in arrival order while their
 * device memory (ising_hmc_estimate_bytes) fits the budget; their handles are
 * created on the admission thread while the worker keeps the device busy, and
 * their state stays resident until they finish.  Each quantum advances every active request by the same
 * number of trajectories (at most quantum_traj): all FP32 lattice requests in
 * one CUDA-graph launch, others on their own streams.  Finished requests keep
 * their observables and latency and free their memory for waiting ones.  A
 * request's result does not depend on the other requests in the batch.
 * Requests larger than the whole budget are rejected (state 3, ENOMEM). */
typedef struct ising_server ising_server_t;
ising_status ising_server_create(int64_t budget_bytes, int quantum_traj, ising_server_t **out);
ising_status ising_server_submit(ising_server_t *s, const ising_hmc_config *cfg, int64_t n_traj,
                                 uint64_t seed, int64_t *request_id);
/* state: 0 queued, 1 running, 2 done (obs, latency and queue time valid),
 * 3 rejected (the return value is the reason).  latency = done - submit,
 * queue = admit - submit, in seconds. */
ising_status ising_server_poll(ising_server_t *s, int64_t request_id, int *state, ising_obs *obs,
                               double *latency_s, double *queue_s);
ising_status ising_server_wait(ising_server_t *s, int64_t request_id, double timeout_s);
ising_status ising_server_drain(ising_server_t *s, double timeout_s);
/* out[ISING_SERVER_NSTATS]: admitted, completed, rejected, queued, active,
 * device bytes in use, site-steps done, shared graph launches, quanta,
 * seconds since creation, then seconds spent creating handles (admission
 * thread), building group graphs, running quanta (launch to completion) and
 * retiring requests (observables, release; worker thread). */
#define ISING_SERVER_NSTATS 14
ising_status ising_server_stats(ising_server_t *s, double *out);
const char *ising_server_last_error(const ising_server_t *s);
void ising_server_destroy(ising_server_t *s);

/* Self-test of device functions the trajectories rely on (no model state;
 * host buffers; synchronous):
 *   which = ISING_SELFTEST_TANH: out[i] = tanh(in[i]) for FP32 in/out, the
 *     force's tanh (Sec. 3 equations of motion), absolute error below 3e-7;
 *   which = ISING_SELFTEST_LOG1PEXP: out[i] = log(1 + exp(-in[i])) for FP64
 *     in/out with in[i] >= 0, the double-float evaluation inside the FP32
 *     form's action log 2cosh x = |x| + log(1 + exp(-2|x|)), absolute error
 *     below 1e-13.
 * Errors: EINVAL (unknown which, n < 0, null buffers), ENOMEM, ECUDA. */
enum { ISING_SELFTEST_TANH = 0, ISING_SELFTEST_LOG1PEXP = 1 };
ising_status ising_hmc_selftest(int which, const void *in, void *out, int64_t n);

/* Energy without allocation.  Some callers cannot call cudaMalloc: code that
 * runs inside a memory pool or arena it does not own, hosts that forbid
 * allocation after start-up, or work inside a region where an allocation
 * would stall or break the caller's stream.  For them this entry point
 * computes, in FP64 with the plain form's per-site arithmetic (in kernels of
 * its own), the action
 * S(psi) = 1/2 psi.A.psi - sum_i log 2cosh((A psi)_i + beta*h0) and the
 * kinetic energy 1/2 p.p of n_chains periodic-lattice configurations
 * (A = beta*Jnn*K + C*1), without allocating any memory.  The paper has no
 * counterpart: it is a deployment variant, not a step of the method.
 *   psi, p : device arrays of n_chains*N FP64 values, chain-major (p may be
 *            NULL, then K = 0); out: device array of 2*n_chains FP64 values,
 *            out[2c] = S of chain c, out[2c+1] = K of chain c.  The caller
 *            owns all three.
 *   stream : cudaStream_t or NULL; the call is asynchronous on it.
 * The partial sums live in one fixed device array of
 * ISING_NOALLOC_MAX_CHAINS * 256 * 2 doubles (256 KB) that every GPU loading
 * this library holds until the process exits; hence n_chains is limited to
 * ISING_NOALLOC_MAX_CHAINS (EINVAL beyond it).  Every call overwrites the
 * array's slots it uses before reading them; calls that overlap on the GPU
 * (other streams, other host threads) share the array and race, so
 * serialise them.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress, with that device current); make that first
 * call before any stream capture.  A CUDA error left pending by earlier work
 * is not cleared and not taken for this call's own: the call returns ECUDA
 * without launching, and the message says so.  Errors: EINVAL (arguments;
 * message in ising_hmc_energy_noalloc_error()), ECUDA. */
#define ISING_NOALLOC_MAX_CHAINS 64
ising_status ising_hmc_energy_noalloc(int dim, const int L[3], double beta, double Jnn, double C,
                                      double h0, int n_chains, const double *psi, const double *p,
                                      double *out, void *stream);
const char *ising_hmc_energy_noalloc_error(void);

/* Self-test of the BF16 tensor-core GEMM behind the dense force:
 * D[n*M + m] = sum_k A[m*K + k] * B[n*K + k] for host BF16 bit patterns A
 * (M x K) and B (N x K), FP32 host output D; M and N multiples of 128, K a
 * multiple of 64.  Synchronous.  Errors: EINVAL, ECUDA, ETIMEOUT (a pipeline
 * wait gave up). */
ising_status ising_hmc_selftest_gemm(int M, int N, int K, const uint16_t *A, const uint16_t *B,
                                     float *D);

/* Timing aid for the BF16 dense form (no counterpart in the paper): n
 * evaluations of the force F = A(tanh(A psi + h') - psi) (Sec. 3) on the
 * handle's working configurations, each the two tensor-core GEMMs with their
 * epilogues, queued on the handle's stream.  It overwrites only the working
 * buffers a trajectory re-initialises (proposal, momenta, u); the chains'
 * configurations, records and sums are untouched.  Asynchronous.  Errors:
 * EINVAL (not the BF16 dense form, n < 0), ECUDA. */
ising_status ising_hmc_dense_forces(ising_hmc_t *h, int n);

/* Test hooks for the failure paths (no counterpart in the paper).  They make
 * a failure on the host side, so no device wait ever has to run out:
 *  - ising_hmc_inject_alloc_failure(k): the k-th next device allocation made
 *    by the library fails as if the device were out of memory (k <= 0
 *    cancels); the call that made it returns ENOMEM and releases what it
 *    had allocated.
 *  - ising_hmc_inject_device_error(h, bits): ORs bits (1 = a bounded device
 *    wait gave up, 2 = a bounds check failed) into the handle's device error
 *    word, which kernels set when they give up; the next call that
 *    synchronises reports ETIMEOUT (bit 1) or ECUDA.  The word is not
 *    cleared: the handle stays in error until destroyed.  EINVAL for other
 *    bits. */
void ising_hmc_inject_alloc_failure(int64_t k);
ising_status ising_hmc_inject_device_error(ising_hmc_t *h, int bits);

void ising_hmc_destroy(ising_hmc_t *h);
const char *ising_hmc_last_error(const ising_hmc_t *h);
const char *ising_hmc_last_create_error(void);

/* A x = b for chain `chain`'s A = beta*J*K + C*1 (Sec. 2) by conjugate
 * gradients in FP64 on the device (one CTA; a set-up computation).  Serves the
 * paper's own parametrisation: its field is psi_p = sqrt(J') (psi + A^-1 h')
 * with J' = beta*J, and its observables carry h'^T Kt^-1 h' = J' h'^T A^-1 h'
 * (Kt = K + C_p*1 = A/J').  b, x: host arrays of N doubles.  Stops when the
 * recursive residual satisfies ||r|| <= tol ||b|| or after max_iter
 * iterations; *iters (may be NULL) gets the count, *resid (may be NULL)
 * ||r||/||b||.  Lattice and infinite-range models, and dense couplings in the
 * plain FP64 form (which keeps J in FP64 on the device; one warp per row of
 * J).  Synchronises.
 * Errors: EINVAL (kind or form, chain, tol <= 0, max_iter < 1), ENOMEM, ECUDA. */
ising_status ising_hmc_solve_A(ising_hmc_t *h, int chain, const double *b, double *x, double tol,
                               int max_iter, int *iters, double *resid);

/* ---- Per-trajectory series and autocorrelation (Sec. 4) -----------------
 * From the next trajectory on, record each chain's m, beta*eps and |m| (the
 * values the measurement step adds to the sums; recorded for every
 * trajectory, thermalisation included) for up to `capacity` trajectories
 * (3 doubles per chain and trajectory in device memory).  While recording,
 * ising_hmc_trajectories runs one trajectory per launch followed by a record
 * launch (results are unchanged); groups and servers do not record.
 * capacity 0 frees the buffer.  Synchronises.  Errors: EINVAL, ENOMEM. */
ising_status ising_hmc_series_enable(ising_hmc_t *h, int64_t capacity);
/* The recorded series into out[(c * n + t) * 3 + k] (k = 0 m, 1 beta*eps,
 * 2 |m|), n = *n_out recorded trajectories; with out NULL only *n_out is
 * set.  Synchronises.  Errors: EINVAL, ECUDA. */
ising_status ising_hmc_series_get(ising_hmc_t *h, double *out, int64_t *n_out);
/* Gamma method (U. Wolff, Comput. Phys. Commun. 156 (2004) 143) on n_rep
 * replicas of length n (x[r * n + t], host memory): the autocorrelation
 * function about the global mean, tau_int with automatic windowing (factor
 * S, 1.5 is customary) and the bias correction of the mean.  out[0] mean,
 * out[1] its error, out[2] tau_int, out[3] the error of tau_int, out[4] the
 * window W.  Host-only (no device work).  Errors: EINVAL (n < 2, n_rep < 1,
 * S <= 0; message from ising_hmc_last_create_error()). */
ising_status ising_gamma_method(const double *x, int64_t n, int n_rep, double S, double *out);

/* ---- Local Metropolis-Hastings comparator (Sec. 4) ----------------------
 * The paper's reference algorithm (single-spin-flip Metropolis sweeps on the
 * spins), run on the GPU so that the cost of an HMC trajectory can be set
 * against the cost of a sweep.  A sweep updates colour 0, then colour 1
 * (c = (x + y + z) mod 2; every extent must be even so that each bond joins
 * the two colours and a colour's sites can be updated in parallel).  Site i of
 * colour c in sweep k draws u = u23(word (j mod 4) of Philox(j / 4, 2k + c,
 * chain, 5)), j = i / 2, and flips iff u < p in FP32, where
 * p = min(1, exp(-2 beta s_i (J nb_i + h))) (nb_i the neighbour spin sum) is
 * formed in FP64 on the host and rounded to FP32.  Spins start all +1 (int8,
 * chain-major).  After each sweep with index >= n_therm the per-chain sums
 * (ISING_SUM_* order) take m = M/N, |m|, beta*eps = beta (-J B - h M) / N
 * (M the spin sum, B the bond sum) and, under ISING_SUM_NACC, the fraction of
 * spins flipped in the sweep; ISING_SUM_DH and ISING_SUM_EXPMDH stay 0.  The
 * same conventions as the HMC calls apply (status codes, stream, ownership). */
typedef struct ising_mh ising_mh_t;

/* cfg: kind LATTICE, dim 1..3, L (each even and >= 4), Jnn, h0 or h0_chain (a
 * per-site h must be NULL), beta or beta_chain (>= 0), n_chains (1..65535),
 * n_therm, stream; every other field is ignored.  Errors: EINVAL, ENOMEM,
 * ECUDA (message from ising_mh_last_error(NULL)). */
ising_status ising_mh_create(const ising_hmc_config *cfg, ising_mh_t **out);
/* n sweeps of every chain (asynchronous); the sweep counter persists, so
 * sweeps(a) then sweeps(b) equals sweeps(a + b) bit for bit.  Errors: EINVAL, ECUDA. */
ising_status ising_mh_sweeps(ising_mh_t *h, int64_t n, uint64_t seed);
/* Chain-averaged m, |m|, E and the flipped fraction (as acceptance), errors
 * as in ising_hmc_observables.  Synchronises. */
ising_status ising_mh_observables(ising_mh_t *h, ising_obs *out);
/* Per-chain sums, ISING_NSUMS doubles per chain.  Synchronises. */
ising_status ising_mh_chain_sums(ising_mh_t *h, double *out);
/* Spins of every chain to host memory (n_chains * N int8 values, +-1). */
ising_status ising_mh_get_spins(ising_mh_t *h, int8_t *out);
/* Spins from host memory (+-1 each, else EINVAL); the next sweep has index next_sweep. */
ising_status ising_mh_set_spins(ising_mh_t *h, const int8_t *in, int64_t next_sweep);
ising_status ising_mh_sync(ising_mh_t *h);
int64_t ising_mh_sweep_index(const ising_mh_t *h);
int64_t ising_mh_launch_count(const ising_mh_t *h);
/* Last error message of h, or of the failed ising_mh_create of this thread when h is NULL. */
const char *ising_mh_last_error(const ising_mh_t *h);
void ising_mh_destroy(ising_mh_t *h);

#ifdef __cplusplus
}
#endif
#endif
