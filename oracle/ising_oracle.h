/*
 * ising_oracle.h -- plain, slow FP64 CPU oracle for the Hubbard-Stratonovich
 * Hybrid Monte Carlo (HMC) of the Ising model (Ostmeyer et al., "The Ising
 * Model with Hybrid Monte Carlo", arXiv:1912.03278).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  The product path
 * (the CUDA library) never calls it, and the two share no code.
 *
 * Conventions (the "NS form" of the action; Sec. 2, Eqs. did_HS_trafo and
 * phi_psi_substitution with the substitution phi = A psi):
 *   A      = beta*J*K + C*1         (lattice: K = periodic nearest-neighbour
 *                                    adjacency; dense: beta*Jmat + C*1)
 *   h'_i   = beta*h_i
 *   S(psi) = 1/2 psi.A.psi - sum_i log 2cosh((A psi)_i + h'_i)
 *   F(psi) = -grad S = A (tanh(A psi + h') - psi)
 *   H      = 1/2 p.p + S(psi)                       (Sec. 3, HMC Hamiltonian)
 *
 * Parity status per function (what pins it; see tests/test_oracle_*.py):
 *   or_philox4x32_10    pinned: published known-answer vectors
 *   or_apply_A          pinned: plane-wave eigenvalues (lattice), numpy
 *                       matrix product of an independently built matrix
 *   or_action/or_force  pinned: central finite differences; brute force
 *   or_leapfrog         pinned: reversibility, dH ~ eps^2, P-form equivalence
 *   or_hmc_run          pinned: brute-force enumeration within 3 sigma,
 *                       Creutz <exp(-dH)> = 1, free-spin closed form
 *   or_brute_force      pinned: 1D transfer matrix, free spins
 *   or_infinite_range   pinned: brute force on the all-to-all model
 *   or_mh_run           pinned: brute force within 3 sigma
 *   or_pform_*          pinned: trajectory-by-trajectory map to the NS form
 */
#ifndef ISING_ORACLE_H
#define ISING_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Philox purposes (fourth counter word). */
enum { OR_PURPOSE_MOM = 1, OR_PURPOSE_ACC = 2, OR_PURPOSE_SPIN = 3, OR_PURPOSE_FLIP = 4,
       OR_PURPOSE_MH = 5 };

/* Momentum-draw forms: 0 = 52-bit uniforms, 2 normals per Philox call (FP64
 * form); 1 = 23-bit uniforms, 4 normals per Philox call (FP32 form). */
enum { OR_FORM_FP64 = 0, OR_FORM_FP32 = 1 };

typedef struct {
    int kind;          /* 0 = periodic hypercubic lattice, 1 = dense couplings */
    int dim;           /* lattice dimension 1..3 */
    int L[3];          /* lattice extents (x fastest), each >= 3 */
    int64_t N;         /* number of sites */
    const double *J;   /* dense: N*N row-major symmetric couplings, J_ii = 0 */
    double Jnn;        /* lattice nearest-neighbour coupling J */
    const double *h;   /* per-site field h_i (N) or NULL for uniform h0 */
    double h0;
    double beta;
    double C;          /* shift, NS units: A = beta*J*K + C*1 */
} or_model;

/* ---- random numbers (Salmon et al., SC'11: Philox4x32-10) ---- */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double or_u23(uint32_t x);
double or_u52(uint32_t a, uint32_t b);
void or_momenta(int form, uint64_t seed, uint32_t chain, uint32_t traj, int64_t N, double *p);
double or_accept_uniform(uint64_t seed, uint32_t chain, uint32_t traj);
void or_spin_uniforms(int form, uint64_t seed, uint32_t chain, uint32_t traj, int64_t N, double *u);

/* ---- model (Sec. 2) ---- */
int64_t or_num_sites(const or_model *m);
void or_neighbors(const or_model *m, int64_t *nbr /* N * 2*dim */);
void or_apply_A(const or_model *m, const double *x, double *y);
double or_action(const or_model *m, const double *psi, double *a_out, double *t_out);
void or_force(const or_model *m, const double *psi, double *F);
double or_kinetic(int64_t N, const double *p);

/* ---- molecular dynamics (Sec. 3) ---- */
void or_leapfrog(const or_model *m, double *psi, double *p, double eps, int n_md);
void or_omelyan(const or_model *m, double *psi, double *p, double eps, int n_md, double lambda);

/* ---- observables (Sec. 4) ---- */
typedef struct {
    double m;        /* (1/N) sum tanh(a + h')          */
    double E;        /* beta*epsilon, NS estimator        */
    double abs_m;    /* |(1/N) sum s| of one spin draw    */
    double abs_mt;   /* |(1/N) sum tanh(a+h')| diagnostic */
    double E_cond;   /* conditional estimator, needs A t  */
} or_obs;
void or_measure(const or_model *m, const double *psi, int form, uint64_t seed, uint32_t chain,
                uint32_t traj, or_obs *out);

/* ---- HMC chain (Sec. 3, algorithm; Sec. 4 estimators) ---- */
typedef struct {
    double *psi;      /* N, current configuration                     */
    double S;         /* S(psi) cached                                 */
    or_obs obs;       /* observables of the current configuration      */
    uint32_t traj;    /* next trajectory index                         */
    /* running sums over measured trajectories */
    double n_meas, n_acc, n_traj;
    double sum_m, sum_m2, sum_E, sum_E2, sum_am, sum_am2, sum_dH, sum_expmdH;
    double sum_Econd, sum_amt;
} or_chain;

typedef struct {
    double dH, logu, K0, S0, K1, S1;
    int accepted;
} or_traj_record;

void or_chain_init(const or_model *m, or_chain *c, int form, uint64_t seed, uint32_t chain);
/* One trajectory: momenta, KDK leapfrog (integrator 0) or Omelyan (1),
 * dH, Metropolis, measurement. psi_prop/p_end (may be NULL) receive the
 * proposal endpoint. flip_every > 0 adds a global sign-flip proposal after
 * every flip_every-th trajectory (Sec. 3, ergodicity). */
void or_trajectory(const or_model *m, or_chain *c, int form, uint64_t seed, uint32_t chain,
                   double eps, int n_md, int integrator, int measure, int flip_every,
                   or_traj_record *rec, double *psi_prop, double *p_end);
/* Run n trajectories; the first n_therm are not measured. Records (may be
 * NULL) receive one or_traj_record per trajectory. */
void or_hmc_run(const or_model *m, or_chain *c, int form, uint64_t seed, uint32_t chain,
                double eps, int n_md, int integrator, int flip_every, int64_t n, int64_t n_therm,
                or_traj_record *recs, double *series_absm);
/* Chains in parallel, one POSIX thread per chain (at most n_threads at once).
 * psi0: n_chains*N start configurations (may be NULL: zero start). Per chain
 * out: 10 doubles = n_meas, n_acc, sum_m, sum_m2, sum_E, sum_E2, sum_am,
 * sum_am2, sum_dH, sum_expmdH. */
void or_hmc_run_chains(const or_model *m, int n_chains, int form, uint64_t seed,
                       const double *eps_per_chain, const double *beta_per_chain,
                       const double *C_per_chain, int n_md, int64_t n, int64_t n_therm,
                       int n_threads, double *out);

/* ---- exact results used as pins ---- */
/* Brute force over all 2^N spin states (N <= 26). out: logZ, <m>, <|m|>,
 * <beta eps>, <m^2>. */
void or_brute_force(const or_model *m, double *out);
/* Periodic 1D chain, transfer matrix: log Z(beta, J, h, N). */
double or_ring_logZ(double beta, double J, double h, int64_t N);
/* Infinite-range model (appendix): <beta eps> with normalised weights. */
double or_infinite_range_energy(double beta, double J, double h, int64_t N);

/* ---- local Metropolis-Hastings comparator (Sec. 4) ---- */
/* n sweeps of N single-spin-flip proposals in site order, spins start all +1.
 * out: n_meas, sum|m|, sum|m|^2, sum E, sum E^2, acceptance. */
void or_mh_run(const or_model *m, uint64_t seed, int64_t n, int64_t n_therm, double *out,
               double *series_absm);
/* Checkerboard form (every lattice extent even): colour 0 then colour 1 per
 * sweep, Philox draws per (site pair, half-sweep, chain), the decision
 * u < p in FP32.  s: N spins (+-1), updated in place; sweeps sweep0 ..
 * sweep0+n-1; sums (10 values, ising_hmc.h ISING_SUM_* order) accumulate the
 * sweeps >= n_therm.  Pinned by brute force, beta = 0 and field limits. */
float or_mh_accept_prob(double beta, double J, double h, int s, int nb);
void or_mh_checkerboard(const or_model *m, uint64_t seed, uint32_t chain, int64_t sweep0,
                        int64_t n, int64_t n_therm, int8_t *s, double *sums);

/* ---- the paper's own parametrisation (P form, Sec. 2-3) ---- */
/* A_p = J'*(K + C_p*1) with J' = beta*J; S_p and its force as printed in
 * Sec. 3 (HMC Hamiltonian and equations of motion). */
double or_pform_action(const or_model *m, double Cp, const double *psip);
void or_pform_force(const or_model *m, double Cp, const double *psip, double *F);
void or_pform_leapfrog(const or_model *m, double Cp, double *psip, double *p, double eps, int n_md);
/* Solve A x = b by conjugate gradients (Sec. 2, constant h'^T Kt^-1 h'). */
int or_cg_solve(const or_model *m, const double *b, double *x, double tol, int max_iter);

#ifdef __cplusplus
}
#endif
#endif
