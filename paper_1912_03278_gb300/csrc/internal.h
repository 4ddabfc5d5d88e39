// internal.h -- structures shared by the host runtime and the kernels.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ising_hmc.h"

namespace ihmc {

// Per-chain parameters (device).  hp = beta*h0 is the uniform part of h'.
struct __align__(16) ChainParams {
    double beta, bJ, C, eps, hp;
    float bJf, pad;
    float betaf, Cf, epsf, hpf;   // one aligned float4 (read whole by the dense epilogues)
};

// Per-chain Markov-chain state (device).
struct ChainState {
    double S;                   // action of the current configuration
    double obs[4];              // m, E, |m| (spin draw), |mean t| of the current configuration
    double sums[ISING_NSUMS];   // running sums over measured trajectories
    double rec[ISING_NREC];     // record of the most recent trajectory
    int start;                  // state-buffer index holding the current configuration
    int prop;                   // state-buffer index holding the most recent proposal
};

// Integrator schedule: force evaluation j kicks p by kick[j]*eps and, unless it
// is the last one, drifts psi by drift[j]*eps.
constexpr int MAX_PASSES = 129;
struct Schedule {
    int n_pass;
    double kick[MAX_PASSES];
    double drift[MAX_PASSES];
};

// Geometry of a periodic lattice as streamed plane by plane.  The plane is the
// set of sites with equal slowest coordinate: a row (2D), an xy-slab (3D), the
// whole ring (1D).
struct Geometry {
    int dim;
    int X, Y, Z;        // extents; unused ones are 1
    int P;              // sites per plane
    int nplanes;        // planes per chain
    int64_t N;          // sites per chain
};

// Arguments of the fused FP32 lattice trajectory kernel.
struct FusedArgs {
    float *psi[3];           // three state buffers, chain-major
    float *p;                // momenta, chain-major
    const float2 *hdf;       // per-site h_i (not scaled by beta) as hi/lo floats, or null
    const float4 *lpe_tab;   // Taylor table of log(1 + exp(-y)), see df32.cuh
    const ChainParams *params;
    ChainState *state;
    Geometry g;
    uint64_t seed;
    uint32_t traj0;          // index of the first trajectory of this launch
    int n_traj;              // trajectories per chain in this launch
    int n_therm;             // trajectories with index < n_therm are not measured
    int flip_every;
    int mode;                // 0 trajectories, 1 evaluate current state, 2 write momenta
    int chain0;              // first chain of this launch
    int n_chains;
    int cs;                  // CTAs per chain (the launch's cluster size; lattice kernel)
    int eval_start;          // lattice kernel: evaluate S and the observables of the start
                             // configuration in the first trajectory's first pass
    int bulk;                // lattice kernel: stage planes by bulk copies (16-byte planes)
    int *err;
};

enum { MODE_TRAJ = 0, MODE_EVAL = 1, MODE_MOMENTA = 2 };

// Trajectory index of the spin draw that measures a configuration set from
// outside (creation, set_state); drawn under key 0.
constexpr uint32_t TRAJ_INIT_INDEX = 0xffffffffu;

// Error bits written by kernels into the handle's error word.
enum { KERR_TIMEOUT = 1, KERR_BOUNDS = 2 };

cudaError_t launch_fused_lattice(const FusedArgs &a, const Schedule &sched, int threads,
                                 int depth, cudaStream_t s);
// dst <- src, bytes a multiple of 16 and both 16-byte aligned, by a grid-stride
// kernel (src may be pinned host memory the device can address)
cudaError_t launch_copy16(const void *src, void *dst, size_t bytes, cudaStream_t s);
// start = prop = 0 in every chain's state (a configuration was set from outside)
cudaError_t launch_reset_chain_start(ChainState *st, int n, cudaStream_t s);
int fused_lattice_smem_bytes(const Geometry &g, int depth, int vec);
// Kernel-node parameters of the same launch (for CUDA graphs); args[0..1]
// must point at the FusedArgs and Schedule values to pass.
cudaError_t fused_lattice_node(const FusedArgs &a, int threads, int depth,
                               cudaKernelNodeParams *np, void **args);
// 1 if (threads, depth) is a valid launch shape for this geometry.
int fused_lattice_valid_launch(const Geometry &g, int threads, int depth);
// 1 if a chain may be split over cs CTAs (a thread-block cluster) at that shape.
int fused_lattice_valid_split(const Geometry &g, int threads, int depth, int cs);
// Cluster size of a graph kernel node made from fused_lattice_node (cs > 1).
cudaError_t fused_lattice_node_cluster(cudaGraphNode_t node, int cs);
int fused_lattice_pick(const Geometry &g, int *threads, int *depth);

// Infinite-range (all-to-all) model, FP32 form: the same arguments, modes and
// per-chain state as the lattice kernel (g.N sites, one CTA per chain);
// ChainParams::bJ holds kappa = beta*J/N.
cudaError_t launch_infinite(const FusedArgs &a, const Schedule &sched, cudaStream_t s);
cudaError_t infinite_node(const FusedArgs &a, cudaKernelNodeParams *np, void **args);
int infinite_threads(int64_t N);

// A x = b by conjugate gradients in FP64, one CTA (lattice, infinite-range or
// dense A with coupling bJ and shift C; J the dense couplings on the device or
// null); work holds 3N doubles; iters and resid are device scalars.
cudaError_t solve_A(const double *b_dev, double *x_dev, double *work, int64_t N, int kind, int dim,
                    const int L[3], double bJ, double C, double tol, int max_iter, int *iters_dev,
                    double *resid_dev, cudaStream_t s, const double *J = nullptr);

// Chain-averaged observables from per-chain sums (ISING_NSUMS per chain).
void obs_from_sums(const double *sums, int n_chains, int64_t n_traj, ising_obs *out);

cudaError_t launch_tanh_selftest(const float *x, float *y, int64_t n, cudaStream_t s);
// BF16 tensor-core GEMM D[n*M + m] = sum_k A[m][k] B[n][k]; M, N multiples of
// 128, K a multiple of 64; *err gets bit 0 if a bounded wait ran out.
cudaError_t launch_gemm_store(const void *A, const void *B, float *D, int M, int N, int K, int *err,
                              cudaStream_t s);
cudaError_t launch_log1pexp_selftest(const double *y, double *out, int64_t n, const float4 *tab,
                                     cudaStream_t s);

// Host construction of the log(1 + exp(-y)) table (one float4 per node).
void build_log1pexp_table(float *out /* 4 * LOG1PEXP_NODES floats */);
constexpr int LOG1PEXP_NODES = 36 * 32 + 1;

// Dense couplings on the tensor cores (BF16 force, FP32 state, FP64-accurate
// action).  Arrays are chain-major with b_pad >= n_chains rows (a multiple of
// 128; padded chains stay zero) and N sites (a multiple of 128).
// Exact digit-sliced action product: ACT_DIGITS signed base-2^ACT_BITS
// digits per operand, ACT_PAIRS digit-plane products (all with s + t <=
// ACT_DIGITS - 1), exact in the FP32 accumulator up to ACT_MAX_N sites.
constexpr int ACT_BITS = 7, ACT_DIGITS = 6, ACT_PAIRS = 21, ACT_MAX_N = 4096;

// FP8 force operands psi and u are stored as x / FP8_OP_SCALE in E4M3 (largest
// value 448): a fixed scale, values beyond +-FP8_OP_RANGE saturate.
constexpr float FP8_OP_RANGE = 32.0f;
constexpr float FP8_OP_SCALE = FP8_OP_RANGE / 448.0f;

struct DenseArgs {
    const __nv_bfloat16 *J16;   // N x N BF16 couplings
    const float *Jhi, *Jlo;     // N x N couplings as a double-float pair
    float *psi_cur;             // current configurations
    float *psi;                 // working (proposal) configurations
    __nv_bfloat16 *psi16;       // BF16 copy of psi (GEMM operand)
    float *p;                   // momenta
    float *u32;                 // u = tanh(A psi + h') - psi
    __nv_bfloat16 *u16;         // BF16 copy of u (GEMM operand)
    float *Ghi, *Glo;           // J psi as a double-float pair (action, N > 4096)
    // action product on the tensor cores (N <= 4096): digit planes of J and
    // psi, exponents of their row / chain scales, exact integer digit sum
    int action_tc;
    const __nv_bfloat16 *Jdig;  // ACT_DIGITS planes of N x N
    __nv_bfloat16 *psidig;      // ACT_DIGITS planes of b_pad x N
    const int *row_exp;         // N
    int *chain_exp;             // b_pad
    long long *Gint;            // b_pad x N, chain-major
    const float2 *hdf;          // per-site h_i as hi/lo floats, or null
    const float4 *lpe_tab;      // log(1 + exp(-y)) table (global)
    const ChainParams *params;
    ChainState *state;
    int N, n_chains, b_pad;
    int pair, nclu;             // CTA-pair GEMM tiles (1) or single-CTA (0); clusters resident at once
    // FP8 force variant: E4M3 J with per-row scales sJ8, E4M3 psi and u holding
    // x / FP8_OP_SCALE
    int fp8;
    const uint8_t *J8;
    const float *sJ8;
    uint8_t *psi8, *u8;
    int *err;
    CUtensorMap tm_J, tm_psi, tm_u, tm_Jdig, tm_psidig;
};

cudaError_t dense_setup(DenseArgs &d);
// y = J x in FP64 (Lanczos at creation).
cudaError_t dense_matvec_f64(const double *J, const double *x, double *y, int64_t N,
                             cudaStream_t s);
// From FP64 couplings on the device: BF16 copy, and the action's digit planes
// and row exponents (dig, row_exp) or its double-float pair (Jhi, Jlo); null
// outputs are skipped.
cudaError_t dense_prepare(const double *J, int64_t N, uint16_t *J16, uint16_t *dig, int *row_exp,
                          float *Jhi, float *Jlo, uint8_t *J8, float *sJ8, cudaStream_t s);
cudaError_t dense_trajectory(DenseArgs &d, const Schedule &sched, uint64_t seed, uint32_t traj,
                             int measure, int flip, cudaStream_t s, int64_t *launches);
cudaError_t dense_eval(DenseArgs &d, cudaStream_t s, int64_t *launches);
cudaError_t dense_momenta(DenseArgs &d, uint64_t seed, uint32_t traj, cudaStream_t s,
                          int64_t *launches);
cudaError_t dense_force_once(DenseArgs &d, cudaStream_t s);

// Plain FP64 form: one chain per launch, unfused kernels.
struct PlainArgs {
    double *psi_cur, *psi, *p, *a, *u, *F;   // per-chain views (N doubles each)
    double *partials;                         // scratch, per-chain view
    const double *h64;                        // per-site h_i or null
    const double *J;                          // dense couplings or null
    const ChainParams *params;                // this chain's parameters
    ChainState *state;                        // this chain's state
    int *flag;                                // this chain's accept/flip flag
    Geometry g;
    int kind;
    uint32_t chain;
};

cudaError_t plain_trajectory(const PlainArgs &a, const Schedule &sched, uint64_t seed,
                             uint32_t traj, int measure, int flip, cudaStream_t s,
                             int64_t *launches);
cudaError_t plain_eval(const PlainArgs &a, cudaStream_t s, int64_t *launches);
cudaError_t plain_momenta(const PlainArgs &a, uint64_t seed, uint32_t traj, cudaStream_t s,
                          int64_t *launches);
int plain_partial_blocks(int64_t N);

}  // namespace ihmc
