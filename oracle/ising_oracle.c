/*
 * ising_oracle.c -- plain, slow FP64 CPU oracle of the HS-field HMC for the
 * Ising model (arXiv:1912.03278).  TEST INFRASTRUCTURE ONLY: loaded by the
 * tests, the smoke check and the benchmark's CPU-baseline leg; never by the
 * product path.  Written for a reader who checks it against the paper by
 * eye: no blocking, no fusion, no reordering beyond the paper's algorithm.
 *
 * Every floating-point quantity is FP64.  Sums that feed the Hamiltonian use
 * Neumaier's compensated summation so that the oracle's own rounding stays
 * far below the 1e-6 tolerance on dH, even for 10^6 sites.
 */
#include "ising_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Compensated summation (Neumaier 1974).                                    */
/* ------------------------------------------------------------------------ */
typedef struct { double s, c; } ksum;
static void ks_add(ksum *k, double x) {
    double t = k->s + x;
    if (fabs(k->s) >= fabs(x)) k->c += (k->s - t) + x;
    else k->c += (x - t) + k->s;
    k->s = t;
}
static double ks_val(const ksum *k) { return k->s + k->c; }

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11).  Ten rounds of the 4x32 Philox S-box with the    */
/* round key advanced by the Weyl constants between rounds.                   */
/* ------------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t prod0 = (uint64_t)M0 * (uint64_t)x0;
        uint64_t prod1 = (uint64_t)M1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += W0;
        k1 += W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Uniform in (0,1) from the top 23 bits of one word: ((x>>9)+1/2) 2^-23.
 * Exact in FP32 and FP64. */
double or_u23(uint32_t x) { return ((double)(x >> 9) + 0.5) * 0x1p-23; }

/* Uniform in (0,1) from 52 bits of two words: ((a>>6) 2^26 + (b>>6) + 1/2) 2^-52.
 * Exact in FP64. */
double or_u52(uint32_t a, uint32_t b) {
    return ((double)(a >> 6) * 67108864.0 + (double)(b >> 6) + 0.5) * 0x1p-52;
}

static void draw(uint64_t seed, uint32_t idx, uint32_t traj, uint32_t chain, uint32_t purpose,
                 uint32_t out[4]) {
    uint32_t ctr[4] = {idx, traj, chain, purpose};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    or_philox4x32_10(ctr, key, out);
}

/* Box-Muller (1958) on one uniform pair: r = sqrt(-2 ln u1), angle 2 pi u2. */
static void box_muller(double u1, double u2, double *z0, double *z1) {
    double r = sqrt(-2.0 * log(u1));
    double ang = 2.0 * M_PI * u2;
    *z0 = r * cos(ang);
    *z1 = r * sin(ang);
}

/* Momentum refresh p ~ N(0,1) per component (Sec. 3, momentum distribution).
 * FP64 form: call j -> sites 2j, 2j+1 from (u52(x0,x1), u52(x2,x3)).
 * FP32 form: call j -> sites 4j..4j+3 from (u23(x0),u23(x1)), (u23(x2),u23(x3)). */
void or_momenta(int form, uint64_t seed, uint32_t chain, uint32_t traj, int64_t N, double *p) {
    uint32_t x[4];
    if (form == OR_FORM_FP64) {
        for (int64_t j = 0; 2 * j < N; ++j) {
            draw(seed, (uint32_t)j, traj, chain, OR_PURPOSE_MOM, x);
            double z0, z1;
            box_muller(or_u52(x[0], x[1]), or_u52(x[2], x[3]), &z0, &z1);
            p[2 * j] = z0;
            if (2 * j + 1 < N) p[2 * j + 1] = z1;
        }
    } else {
        for (int64_t j = 0; 4 * j < N; ++j) {
            draw(seed, (uint32_t)j, traj, chain, OR_PURPOSE_MOM, x);
            double z[4];
            box_muller(or_u23(x[0]), or_u23(x[1]), &z[0], &z[1]);
            box_muller(or_u23(x[2]), or_u23(x[3]), &z[2], &z[3]);
            for (int q = 0; q < 4; ++q)
                if (4 * j + q < N) p[4 * j + q] = z[q];
        }
    }
}

/* Metropolis uniform (Sec. 3, accept/reject): one u52 per chain and trajectory. */
double or_accept_uniform(uint64_t seed, uint32_t chain, uint32_t traj) {
    uint32_t x[4];
    draw(seed, 0, traj, chain, OR_PURPOSE_ACC, x);
    return or_u52(x[0], x[1]);
}

static double flip_uniform(uint64_t seed, uint32_t chain, uint32_t traj) {
    uint32_t x[4];
    draw(seed, 0, traj, chain, OR_PURPOSE_FLIP, x);
    return or_u52(x[0], x[1]);
}

/* Uniforms for the conditional spin draw: FP64 form 2 u52 per call, FP32
 * form 4 u23 per call (same layout as the momenta). */
void or_spin_uniforms(int form, uint64_t seed, uint32_t chain, uint32_t traj, int64_t N,
                      double *u) {
    uint32_t x[4];
    if (form == OR_FORM_FP64) {
        for (int64_t j = 0; 2 * j < N; ++j) {
            draw(seed, (uint32_t)j, traj, chain, OR_PURPOSE_SPIN, x);
            u[2 * j] = or_u52(x[0], x[1]);
            if (2 * j + 1 < N) u[2 * j + 1] = or_u52(x[2], x[3]);
        }
    } else {
        for (int64_t j = 0; 4 * j < N; ++j) {
            draw(seed, (uint32_t)j, traj, chain, OR_PURPOSE_SPIN, x);
            for (int q = 0; q < 4; ++q)
                if (4 * j + q < N) u[4 * j + q] = or_u23(x[q]);
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Model: connectivity K and the shifted matrix A (Sec. 2).                  */
/* ------------------------------------------------------------------------ */
int64_t or_num_sites(const or_model *m) {
    if (m->kind == 1) return m->N;
    int64_t n = 1;
    for (int d = 0; d < m->dim; ++d) n *= m->L[d];
    return n;
}

/* Periodic hypercubic lattice, site i = x + L0 (y + L1 z).  Neighbours of a
 * site in the order (+x, -x, +y, -y, +z, -z); K_ij = 1 for each listed j. */
void or_neighbors(const or_model *m, int64_t *nbr) {
    int64_t N = or_num_sites(m);
    int dim = m->dim;
    int64_t stride[3] = {1, m->L[0], (int64_t)m->L[0] * (dim > 1 ? m->L[1] : 1)};
    for (int64_t i = 0; i < N; ++i) {
        int64_t rem = i;
        int64_t coord[3] = {0, 0, 0};
        for (int d = 0; d < dim; ++d) {
            coord[d] = rem % m->L[d];
            rem /= m->L[d];
        }
        for (int d = 0; d < dim; ++d) {
            int64_t up = (coord[d] + 1) % m->L[d];
#ifdef OR_PLANT_NEIGHBOR
            int64_t dn = (coord[d] + m->L[d] - 2) % m->L[d]; /* planted mistake */
#else
            int64_t dn = (coord[d] + m->L[d] - 1) % m->L[d];
#endif
            nbr[i * 2 * dim + 2 * d] = i + (up - coord[d]) * stride[d];
            nbr[i * 2 * dim + 2 * d + 1] = i + (dn - coord[d]) * stride[d];
        }
    }
}

static double hprime(const or_model *m, int64_t i) {
    return m->beta * (m->h ? m->h[i] : m->h0);
}

/* y = A x with A = beta*J*K + C*1 (lattice) or beta*Jmat + C*1 (dense). */
void or_apply_A(const or_model *m, const double *x, double *y) {
    int64_t N = or_num_sites(m);
    if (m->kind == 1) {
        for (int64_t i = 0; i < N; ++i) {
            double s = 0.0;
            for (int64_t j = 0; j < N; ++j) s += m->J[i * N + j] * x[j];
            y[i] = m->beta * s + m->C * x[i];
        }
        return;
    }
    int nn = 2 * m->dim;
    int64_t *nbr = (int64_t *)malloc(sizeof(int64_t) * N * nn);
    or_neighbors(m, nbr);
    for (int64_t i = 0; i < N; ++i) {
        double s = 0.0;
        for (int k = 0; k < nn; ++k) s += x[nbr[i * nn + k]];
        y[i] = m->beta * m->Jnn * s + m->C * x[i];
    }
    free(nbr);
}

/* log(2 cosh x) = |x| + log(1 + exp(-2|x|)), free of overflow. */
static double log2cosh(double x) {
    double ax = fabs(x);
    return ax + log1p(exp(-2.0 * ax));
}

/* S(psi) = 1/2 psi.A psi - sum_i log 2cosh((A psi)_i + h'_i)
 * (Sec. 2, Eq. phi_psi_substitution with phi = A psi).  a_out, t_out
 * (optional) receive a = A psi and t = tanh(a + h'). */
double or_action(const or_model *m, const double *psi, double *a_out, double *t_out) {
    int64_t N = or_num_sites(m);
    double *a = a_out ? a_out : (double *)malloc(sizeof(double) * N);
    or_apply_A(m, psi, a);
    ksum S = {0, 0};
    for (int64_t i = 0; i < N; ++i) {
        double x = a[i] + hprime(m, i);
#ifdef OR_PLANT_ACTION
        ks_add(&S, psi[i] * a[i]); /* planted mistake: dropped 1/2 */
#else
        ks_add(&S, 0.5 * psi[i] * a[i]);
#endif
        ks_add(&S, -log2cosh(x));
        if (t_out) t_out[i] = tanh(x);
    }
    if (!a_out) free(a);
    return ks_val(&S);
}

/* F = -dS/dpsi = A (tanh(A psi + h') - psi)  (Sec. 3, equations of motion). */
void or_force(const or_model *m, const double *psi, double *F) {
    int64_t N = or_num_sites(m);
    double *a = (double *)malloc(sizeof(double) * N);
    double *u = (double *)malloc(sizeof(double) * N);
    or_apply_A(m, psi, a);
#ifdef OR_PLANT_FORCE_SIGN
    for (int64_t i = 0; i < N; ++i) u[i] = tanh(a[i] + hprime(m, i)) + psi[i]; /* planted */
#else
    for (int64_t i = 0; i < N; ++i) u[i] = tanh(a[i] + hprime(m, i)) - psi[i];
#endif
    or_apply_A(m, u, F);
    free(a);
    free(u);
}

double or_kinetic(int64_t N, const double *p) {
    ksum K = {0, 0};
    for (int64_t i = 0; i < N; ++i) ks_add(&K, 0.5 * p[i] * p[i]);
    return ks_val(&K);
}

/* ------------------------------------------------------------------------ */
/* Molecular dynamics (Sec. 3): symmetric symplectic integrators.            */
/* ------------------------------------------------------------------------ */
/* Kick-drift-kick leapfrog with n_md full drifts:
 *   p += eps/2 F;  (psi += eps p; p += eps F) x (n_md-1);  psi += eps p;  p += eps/2 F */
void or_leapfrog(const or_model *m, double *psi, double *p, double eps, int n_md) {
    int64_t N = or_num_sites(m);
    double *F = (double *)malloc(sizeof(double) * N);
    or_force(m, psi, F);
    for (int64_t i = 0; i < N; ++i) p[i] += 0.5 * eps * F[i];
    for (int step = 1; step <= n_md; ++step) {
        for (int64_t i = 0; i < N; ++i) psi[i] += eps * p[i];
        or_force(m, psi, F);
#ifdef OR_PLANT_LEAPFROG
        double kick = eps; /* planted mistake: full final kick */
#else
        double kick = (step == n_md) ? 0.5 * eps : eps;
#endif
        for (int64_t i = 0; i < N; ++i) p[i] += kick * F[i];
    }
    free(F);
}

/* Second-order minimum-norm integrator (Omelyan, Mryglod, Folk 2003), in its
 * position-velocity form per step of length eps:
 *   p += lambda eps F; psi += eps/2 p; p += (1-2 lambda) eps F; psi += eps/2 p;
 *   p += lambda eps F.   lambda ~ 0.1931833. */
void or_omelyan(const or_model *m, double *psi, double *p, double eps, int n_md, double lambda) {
    int64_t N = or_num_sites(m);
    double *F = (double *)malloc(sizeof(double) * N);
    for (int step = 0; step < n_md; ++step) {
        or_force(m, psi, F);
        for (int64_t i = 0; i < N; ++i) p[i] += lambda * eps * F[i];
        for (int64_t i = 0; i < N; ++i) psi[i] += 0.5 * eps * p[i];
        or_force(m, psi, F);
        for (int64_t i = 0; i < N; ++i) p[i] += (1.0 - 2.0 * lambda) * eps * F[i];
        for (int64_t i = 0; i < N; ++i) psi[i] += 0.5 * eps * p[i];
        or_force(m, psi, F);
        for (int64_t i = 0; i < N; ++i) p[i] += lambda * eps * F[i];
    }
    free(F);
}

/* ------------------------------------------------------------------------ */
/* Observables (Sec. 4).  Given phi = A psi the spins are independent with   */
/* P(s_i) ~ exp(s_i (a_i + h'_i)) (Sec. 2, Eq. did_HS_trafo), so              */
/*   <m>         = < (1/N) sum_i t_i >,   t = tanh(a + h')                    */
/*   <beta eps>  = C/2 - (1/2N) <a.t> - (1/N) <h'.t>                          */
/* (the beta-derivative of log Z as in Eq. ee_form, taken at fixed C/beta,    */
/* plus the virial identity <psi.grad S> = N; at h = 0 it is the paper's      */
/* Eq. formula_for_e with a = sqrt(J') Kt psi_p and C = J' C_p).              */
/* |m| comes from one conditional draw s_i = +1 iff u_i < (1 + t_i)/2.        */
/* ------------------------------------------------------------------------ */
void or_measure(const or_model *m, const double *psi, int form, uint64_t seed, uint32_t chain,
                uint32_t traj, or_obs *out) {
    int64_t N = or_num_sites(m);
    double *a = (double *)malloc(sizeof(double) * N);
    double *t = (double *)malloc(sizeof(double) * N);
    double *u = (double *)malloc(sizeof(double) * N);
    double *At = (double *)malloc(sizeof(double) * N);
    or_action(m, psi, a, t);
    or_spin_uniforms(form, seed, chain, traj, N, u);
    ksum st = {0, 0}, sat = {0, 0}, sht = {0, 0}, ss = {0, 0}, stAt = {0, 0};
    for (int64_t i = 0; i < N; ++i) {
        ks_add(&st, t[i]);
        ks_add(&sat, a[i] * t[i]);
        ks_add(&sht, hprime(m, i) * t[i]);
        /* FP32 form takes the spin decision in FP32, like its kernel. */
        int up;
        if (form == OR_FORM_FP32) up = (float)u[i] < (1.0f + (float)t[i]) * 0.5f;
        else up = u[i] < (1.0 + t[i]) * 0.5;
        ks_add(&ss, up ? 1.0 : -1.0);
    }
    /* conditional estimator E[beta H | psi] = -(1/2) t.(A - C) t - h'.t */
    or_apply_A(m, t, At);
    for (int64_t i = 0; i < N; ++i) ks_add(&stAt, t[i] * (At[i] - m->C * t[i]));
    double invN = 1.0 / (double)N;
    out->m = ks_val(&st) * invN;
    out->E = 0.5 * m->C - 0.5 * ks_val(&sat) * invN - ks_val(&sht) * invN;
    out->abs_m = fabs(ks_val(&ss)) * invN;
    out->abs_mt = fabs(out->m);
    out->E_cond = (-0.5 * ks_val(&stAt) - ks_val(&sht)) * invN;
    free(a);
    free(t);
    free(u);
    free(At);
}

/* ------------------------------------------------------------------------ */
/* The HMC algorithm (Sec. 3).                                               */
/* ------------------------------------------------------------------------ */
/* psi starts at zero (or the caller's psi); the observables of that start
 * configuration use the spin draw of trajectory index 0xffffffff under key 0,
 * so they do not depend on the run's seed. */
void or_chain_init(const or_model *m, or_chain *c, int form, uint64_t seed, uint32_t chain) {
    int64_t N = or_num_sites(m);
    if (!c->psi) c->psi = (double *)calloc((size_t)N, sizeof(double));
    c->S = or_action(m, c->psi, NULL, NULL);
    (void)seed;
    or_measure(m, c->psi, form, 0, chain, 0xffffffffu, &c->obs);
    c->traj = 0;
    c->n_meas = c->n_acc = c->n_traj = 0;
    c->sum_m = c->sum_m2 = c->sum_E = c->sum_E2 = c->sum_am = c->sum_am2 = 0;
    c->sum_dH = c->sum_expmdH = c->sum_Econd = c->sum_amt = 0;
}

void or_trajectory(const or_model *m, or_chain *c, int form, uint64_t seed, uint32_t chain,
                   double eps, int n_md, int integrator, int measure, int flip_every,
                   or_traj_record *rec, double *psi_prop, double *p_end) {
    int64_t N = or_num_sites(m);
    uint32_t tr = c->traj;
    double *psi = (double *)malloc(sizeof(double) * N);
    double *p = (double *)malloc(sizeof(double) * N);
    /* 1. momentum refresh */
    or_momenta(form, seed, chain, tr, N, p);
    double K0 = or_kinetic(N, p);
    double S0 = or_action(m, c->psi, NULL, NULL);
    /* 2. molecular dynamics, one trajectory */
    memcpy(psi, c->psi, sizeof(double) * N);
#ifdef OR_PLANT_OMELYAN
    const double omelyan_lambda = 0.25; /* planted mistake: not the minimum-norm value */
#else
    const double omelyan_lambda = 0.1931833275037836;
#endif
    if (integrator == 1) or_omelyan(m, psi, p, eps, n_md, omelyan_lambda);
    else or_leapfrog(m, psi, p, eps, n_md);
    /* 3. energy splitting and Metropolis test */
    double K1 = or_kinetic(N, p);
    double S1 = or_action(m, psi, NULL, NULL);
    double dH = (K1 + S1) - (K0 + S0);
    double logu = log(or_accept_uniform(seed, chain, tr));
    int acc = logu < -dH;
    int changed = 0;
    if (acc) {
        memcpy(c->psi, psi, sizeof(double) * N);
        c->S = S1;
        changed = 1;
    }
    /* 4. optional global sign flip psi -> -psi with its own Metropolis test */
    if (flip_every > 0 && ((tr + 1) % (uint32_t)flip_every) == 0) {
        double *neg = (double *)malloc(sizeof(double) * N);
        for (int64_t i = 0; i < N; ++i) neg[i] = -c->psi[i];
        double Sf = or_action(m, neg, NULL, NULL);
        double lu = log(flip_uniform(seed, chain, tr));
        if (lu < -(Sf - c->S)) {
            memcpy(c->psi, neg, sizeof(double) * N);
            c->S = Sf;
            changed = 1;
        }
        free(neg);
    }
    /* 5. measurement; a repeated configuration repeats its measurement */
    if (changed) or_measure(m, c->psi, form, seed, chain, tr, &c->obs);
    c->n_traj += 1;
    if (measure) {
        c->n_meas += 1;
        c->n_acc += acc;
        c->sum_m += c->obs.m;
        c->sum_m2 += c->obs.m * c->obs.m;
        c->sum_E += c->obs.E;
        c->sum_E2 += c->obs.E * c->obs.E;
        c->sum_am += c->obs.abs_m;
        c->sum_am2 += c->obs.abs_m * c->obs.abs_m;
        c->sum_dH += dH;
        c->sum_expmdH += exp(-dH);
        c->sum_Econd += c->obs.E_cond;
        c->sum_amt += c->obs.abs_mt;
    }
    if (rec) {
        rec->dH = dH;
        rec->logu = logu;
        rec->K0 = K0;
        rec->S0 = S0;
        rec->K1 = K1;
        rec->S1 = S1;
        rec->accepted = acc;
    }
    if (psi_prop) memcpy(psi_prop, psi, sizeof(double) * N);
    if (p_end) memcpy(p_end, p, sizeof(double) * N);
    c->traj = tr + 1;
    free(psi);
    free(p);
}

void or_hmc_run(const or_model *m, or_chain *c, int form, uint64_t seed, uint32_t chain,
                double eps, int n_md, int integrator, int flip_every, int64_t n, int64_t n_therm,
                or_traj_record *recs, double *series_absm) {
    for (int64_t k = 0; k < n; ++k) {
        int meas = k >= n_therm;
        or_trajectory(m, c, form, seed, chain, eps, n_md, integrator, meas, flip_every,
                      recs ? &recs[k] : NULL, NULL, NULL);
        if (series_absm) series_absm[k] = c->obs.abs_m;
    }
}

typedef struct {
    const or_model *m;
    int form, n_md, chain;
    uint64_t seed;
    double eps, beta, C;
    int64_t n, n_therm;
    double *out;
} chain_job;

static void *chain_worker(void *arg) {
    chain_job *job = (chain_job *)arg;
    or_model mm = *job->m;
    mm.beta = job->beta;
    mm.C = job->C;
    or_chain c;
    memset(&c, 0, sizeof(c));
    or_chain_init(&mm, &c, job->form, job->seed, (uint32_t)job->chain);
    or_hmc_run(&mm, &c, job->form, job->seed, (uint32_t)job->chain, job->eps, job->n_md, 0, 0,
               job->n, job->n_therm, NULL, NULL);
    double *o = job->out;
    o[0] = c.n_meas; o[1] = c.n_acc; o[2] = c.sum_m; o[3] = c.sum_m2; o[4] = c.sum_E;
    o[5] = c.sum_E2; o[6] = c.sum_am; o[7] = c.sum_am2; o[8] = c.sum_dH; o[9] = c.sum_expmdH;
    free(c.psi);
    return NULL;
}

void or_hmc_run_chains(const or_model *m, int n_chains, int form, uint64_t seed,
                       const double *eps_per_chain, const double *beta_per_chain,
                       const double *C_per_chain, int n_md, int64_t n, int64_t n_therm,
                       int n_threads, double *out) {
    if (n_threads < 1) n_threads = 1;
    chain_job *jobs = (chain_job *)calloc((size_t)n_chains, sizeof(chain_job));
    pthread_t *th = (pthread_t *)calloc((size_t)n_threads, sizeof(pthread_t));
    for (int c = 0; c < n_chains; ++c) {
        jobs[c].m = m;
        jobs[c].form = form;
        jobs[c].n_md = n_md;
        jobs[c].chain = c;
        jobs[c].seed = seed;
        jobs[c].eps = eps_per_chain[c];
        jobs[c].beta = beta_per_chain ? beta_per_chain[c] : m->beta;
        jobs[c].C = C_per_chain ? C_per_chain[c] : m->C;
        jobs[c].n = n;
        jobs[c].n_therm = n_therm;
        jobs[c].out = out + 10 * c;
    }
    for (int base = 0; base < n_chains; base += n_threads) {
        int k = 0;
        for (; k < n_threads && base + k < n_chains; ++k)
            pthread_create(&th[k], NULL, chain_worker, &jobs[base + k]);
        for (int q = 0; q < k; ++q) pthread_join(th[q], NULL);
    }
    free(th);
    free(jobs);
}

/* ------------------------------------------------------------------------ */
/* Exact results.                                                            */
/* ------------------------------------------------------------------------ */
/* beta H(s) = -1/2 beta s.(JK) s - beta h.s  (Sec. 2, Eq. hamilton_matrix_notation),
 * summed over all 2^N states with a log-sum-exp shift. */
void or_brute_force(const or_model *m, double *out) {
    int64_t N = or_num_sites(m);
    int64_t nstates = (int64_t)1 << N;
    int nn = 2 * m->dim;
    int64_t *nbr = NULL;
    if (m->kind == 0) {
        nbr = (int64_t *)malloc(sizeof(int64_t) * N * nn);
        or_neighbors(m, nbr);
    }
    double *bH = (double *)malloc(sizeof(double) * nstates);
    double *s = (double *)malloc(sizeof(double) * N);
    double bHmin = INFINITY;
    for (int64_t st = 0; st < nstates; ++st) {
        for (int64_t i = 0; i < N; ++i) s[i] = ((st >> i) & 1) ? -1.0 : 1.0;
        double pair = 0.0, field = 0.0;
        for (int64_t i = 0; i < N; ++i) {
            if (m->kind == 0) {
                for (int k = 0; k < nn; ++k) pair += m->Jnn * s[i] * s[nbr[i * nn + k]];
            } else {
                for (int64_t j = 0; j < N; ++j) pair += m->J[i * N + j] * s[i] * s[j];
            }
            field += (m->h ? m->h[i] : m->h0) * s[i];
        }
        bH[st] = m->beta * (-0.5 * pair - field);
        if (bH[st] < bHmin) bHmin = bH[st];
    }
    ksum Z = {0, 0}, Zm = {0, 0}, Zam = {0, 0}, ZE = {0, 0}, Zm2 = {0, 0};
    for (int64_t st = 0; st < nstates; ++st) {
        double w = exp(-(bH[st] - bHmin));
        int64_t down = 0;
        for (int64_t i = 0; i < N; ++i) down += (st >> i) & 1;
        double mag = (double)(N - 2 * down) / (double)N;
        ks_add(&Z, w);
        ks_add(&Zm, w * mag);
        ks_add(&Zam, w * fabs(mag));
        ks_add(&ZE, w * bH[st] / (double)N);
        ks_add(&Zm2, w * mag * mag);
    }
    double z = ks_val(&Z);
    out[0] = log(z) - bHmin;
    out[1] = ks_val(&Zm) / z;
    out[2] = ks_val(&Zam) / z;
    out[3] = ks_val(&ZE) / z;
    out[4] = ks_val(&Zm2) / z;
    free(bH);
    free(s);
    free(nbr);
}

/* Periodic ring: Z = lp^N + lm^N with
 * l(+/-) = e^{bJ} cosh(bh) +/- sqrt(e^{2bJ} sinh^2(bh) + e^{-2bJ}). */
double or_ring_logZ(double beta, double J, double h, int64_t N) {
    double bJ = beta * J, bh = beta * h;
    double a = exp(bJ) * cosh(bh);
    double r = sqrt(exp(2 * bJ) * sinh(bh) * sinh(bh) + exp(-2 * bJ));
    double lp = a + r, lm = a - r;
    double ratio = lm / lp;
    double tail = pow(fabs(ratio), (double)N);
    if (ratio < 0 && (N % 2)) tail = -tail;
    return (double)N * log(lp) + log1p(tail);
}

/* Infinite-range model (appendix): beta H = -1/2 b Jh (M^2 - N) - b h M with
 * Jh = J/N and M = N - 2n; weights w_n = binom(N,n) exp(1/2 b Jh M^2 + b h M)
 * normalised among themselves; <beta eps> = 1/2 b Jh - (b/N) <1/2 Jh M^2 + h M>. */
double or_infinite_range_energy(double beta, double J, double h, int64_t N) {
    double Jh = J / (double)N;
    double *lw = (double *)malloc(sizeof(double) * (N + 1));
    double lmax = -INFINITY;
    for (int64_t n = 0; n <= N; ++n) {
        double M = (double)(N - 2 * n);
        double lbin = lgamma((double)N + 1) - lgamma((double)n + 1) - lgamma((double)(N - n) + 1);
        lw[n] = lbin + 0.5 * beta * Jh * M * M + beta * h * M;
        if (lw[n] > lmax) lmax = lw[n];
    }
    ksum Z = {0, 0}, num = {0, 0};
    for (int64_t n = 0; n <= N; ++n) {
        double M = (double)(N - 2 * n);
        double w = exp(lw[n] - lmax);
        ks_add(&Z, w);
        ks_add(&num, w * (0.5 * Jh * M * M + h * M));
    }
    free(lw);
    return 0.5 * beta * Jh - beta / (double)N * ks_val(&num) / ks_val(&Z);
}

/* ------------------------------------------------------------------------ */
/* Local Metropolis-Hastings (Sec. 4 comparator): sweeps of N single-spin     */
/* flips in site order; flip accepted with min(1, exp(-beta dH_ising)).       */
/* ------------------------------------------------------------------------ */
void or_mh_run(const or_model *m, uint64_t seed, int64_t n, int64_t n_therm, double *out,
               double *series_absm) {
    int64_t N = or_num_sites(m);
    int nn = 2 * m->dim;
    int64_t *nbr = NULL;
    if (m->kind == 0) {
        nbr = (int64_t *)malloc(sizeof(int64_t) * N * nn);
        or_neighbors(m, nbr);
    }
    double *s = (double *)malloc(sizeof(double) * N);
    for (int64_t i = 0; i < N; ++i) s[i] = 1.0;
    double nm = 0, sam = 0, sam2 = 0, sE = 0, sE2 = 0, nacc = 0, nprop = 0;
    for (int64_t sweep = 0; sweep < n; ++sweep) {
        for (int64_t i = 0; i < N; ++i) {
            double field = 0.0;
            if (m->kind == 0) {
                for (int k = 0; k < nn; ++k) field += m->Jnn * s[nbr[i * nn + k]];
            } else {
                for (int64_t j = 0; j < N; ++j) field += m->J[i * N + j] * s[j];
            }
            field += m->h ? m->h[i] : m->h0;
            double dbH = 2.0 * m->beta * s[i] * field; /* beta (H_new - H_old) */
            uint32_t x[4];
            draw(seed, (uint32_t)i, (uint32_t)sweep, 0, OR_PURPOSE_MH, x);
            double u = or_u52(x[0], x[1]);
            nprop += 1;
            if (log(u) < -dbH) {
                s[i] = -s[i];
                nacc += 1;
            }
        }
        if (sweep >= n_therm || series_absm) {
            double pair = 0.0, fld = 0.0, mag = 0.0;
            for (int64_t i = 0; i < N; ++i) {
                if (m->kind == 0) {
                    for (int k = 0; k < nn; ++k) pair += m->Jnn * s[i] * s[nbr[i * nn + k]];
                } else {
                    for (int64_t j = 0; j < N; ++j) pair += m->J[i * N + j] * s[i] * s[j];
                }
                fld += (m->h ? m->h[i] : m->h0) * s[i];
                mag += s[i];
            }
            double E = m->beta * (-0.5 * pair - fld) / (double)N;
            double am = fabs(mag) / (double)N;
            if (series_absm) series_absm[sweep] = am;
            if (sweep >= n_therm) {
                nm += 1;
                sam += am;
                sam2 += am * am;
                sE += E;
                sE2 += E * E;
            }
        }
    }
    out[0] = nm; out[1] = sam; out[2] = sam2; out[3] = sE; out[4] = sE2;
    out[5] = nacc / (nprop > 0 ? nprop : 1);
    free(s);
    free(nbr);
}

/* ------------------------------------------------------------------------ */
/* Checkerboard local Metropolis-Hastings (Sec. 4 comparator; the paper does  */
/* not fix the order of the N single-spin proposals of a sweep).  On a        */
/* lattice whose extents are all even, colour c = (x + y + z) mod 2 splits    */
/* the sites so that every bond joins the two colours: proposals of one       */
/* colour do not see each other, so one colour may be updated in any order.  */
/* A sweep updates colour 0, then colour 1, each in site order.  Site i of    */
/* colour c in sweep k draws u = u23(word (j mod 4) of Philox(j div 4,        */
/* 2k + c, chain, MH)) with j = i div 2 (the two sites 2j, 2j+1 have          */
/* different colours), and flips iff u < p in FP32, where p =                 */
/* min(1, exp(-2 beta s_i (J nb_i + h))) is formed in FP64 (nb_i the          */
/* neighbour spin sum, no contraction) and rounded to FP32.                   */
/* After each sweep k >= n_therm, with M = sum_i s_i and B = sum over bonds   */
/* s_i s_j: m = M/N, E = beta (-J B - h M) / N, and the fraction of flipped   */
/* sites, summed in the order of ising_hmc.h's ISING_SUM_* (10 values).       */
/* ------------------------------------------------------------------------ */
float or_mh_accept_prob(double beta, double J, double h, int s, int nb) {
    double f = J * (double)nb + h;
    double x = -2.0 * beta * (double)s * f;
    double p = x >= 0.0 ? 1.0 : exp(x);
    return (float)p;
}

void or_mh_checkerboard(const or_model *m, uint64_t seed, uint32_t chain, int64_t sweep0,
                        int64_t n, int64_t n_therm, int8_t *s, double *sums) {
    int64_t N = or_num_sites(m);
    int nn = 2 * m->dim;
    int64_t *nbr = (int64_t *)malloc(sizeof(int64_t) * N * nn);
    or_neighbors(m, nbr);
    int L0 = m->L[0], L1 = m->dim > 1 ? m->L[1] : 1;
    for (int64_t k = sweep0; k < sweep0 + n; ++k) {
        int64_t flips = 0;
        for (int c = 0; c < 2; ++c) {
            for (int64_t i = 0; i < N; ++i) {
                int64_t x = i % L0, y = (i / L0) % L1, z = i / ((int64_t)L0 * L1);
                if ((int)((x + y + z) & 1) != c) continue;
                int nb = 0;
                for (int d = 0; d < nn; ++d) nb += s[nbr[i * nn + d]];
                int64_t j = i / 2;
                uint32_t w[4];
                draw(seed, (uint32_t)(j / 4), (uint32_t)(2 * k + c), chain, OR_PURPOSE_MH, w);
                float u = (float)or_u23(w[j % 4]);
                if (u < or_mh_accept_prob(m->beta, m->Jnn, m->h0, s[i], nb)) {
                    s[i] = (int8_t)(-s[i]);
                    flips += 1;
                }
            }
        }
        if (k >= n_therm) {
            int64_t M = 0, B = 0;
            for (int64_t i = 0; i < N; ++i) {
                M += s[i];
                /* forward neighbours (+x, +y, +z): every bond once */
                for (int d = 0; d < m->dim; ++d) B += s[i] * s[nbr[i * nn + 2 * d]];
            }
            double mm = (double)M / (double)N;
            double E = m->beta * (-m->Jnn * (double)B - m->h0 * (double)M) / (double)N;
            sums[0] += 1.0;
            sums[1] += (double)flips / (double)N;
            sums[2] += mm;
            sums[3] += mm * mm;
            sums[4] += E;
            sums[5] += E * E;
            sums[6] += fabs(mm);
            sums[7] += mm * mm;
        }
    }
    free(nbr);
}

/* ------------------------------------------------------------------------ */
/* The paper's own parametrisation (P form).  K~ = K + C_p 1, J' = beta J,   */
/* h' = beta h (Sec. 2); action and forces as printed in Sec. 3:             */
/*  S_p = 1/2 psi.K~ psi - psi.h'/sqrt(J') - sum log cosh(sqrt(J') (K~ psi)_i)   */
/*  F_p = -K~ psi + h'/sqrt(J') + sqrt(J') K~ tanh(sqrt(J') K~ psi)          */
/* Lattice models only (uniform J).                                          */
/* ------------------------------------------------------------------------ */
static void apply_Kt(const or_model *m, double Cp, const double *x, double *y) {
    /* K~ x with the lattice adjacency, via A with beta J = 1 and C = C_p */
    or_model k = *m;
    k.beta = 1.0;
    k.Jnn = 1.0;
    k.C = Cp;
    or_apply_A(&k, x, y);
}

double or_pform_action(const or_model *m, double Cp, const double *psip) {
    int64_t N = or_num_sites(m);
    double Jp = m->beta * m->Jnn, sJ = sqrt(Jp);
    double *k = (double *)malloc(sizeof(double) * N);
    apply_Kt(m, Cp, psip, k);
    ksum S = {0, 0};
    for (int64_t i = 0; i < N; ++i) {
        ks_add(&S, 0.5 * psip[i] * k[i]);
        ks_add(&S, -psip[i] * hprime(m, i) / sJ);
        double x = fabs(sJ * k[i]);
        ks_add(&S, -(x + log1p(exp(-2.0 * x)) - M_LN2)); /* log cosh */
    }
    free(k);
    return ks_val(&S);
}

void or_pform_force(const or_model *m, double Cp, const double *psip, double *F) {
    int64_t N = or_num_sites(m);
    double Jp = m->beta * m->Jnn, sJ = sqrt(Jp);
    double *k = (double *)malloc(sizeof(double) * N);
    double *th = (double *)malloc(sizeof(double) * N);
    double *kth = (double *)malloc(sizeof(double) * N);
    apply_Kt(m, Cp, psip, k);
    for (int64_t i = 0; i < N; ++i) th[i] = tanh(sJ * k[i]);
    apply_Kt(m, Cp, th, kth);
    for (int64_t i = 0; i < N; ++i) F[i] = -k[i] + hprime(m, i) / sJ + sJ * kth[i];
    free(k);
    free(th);
    free(kth);
}

void or_pform_leapfrog(const or_model *m, double Cp, double *psip, double *p, double eps,
                       int n_md) {
    int64_t N = or_num_sites(m);
    double *F = (double *)malloc(sizeof(double) * N);
    or_pform_force(m, Cp, psip, F);
    for (int64_t i = 0; i < N; ++i) p[i] += 0.5 * eps * F[i];
    for (int step = 1; step <= n_md; ++step) {
        for (int64_t i = 0; i < N; ++i) psip[i] += eps * p[i];
        or_pform_force(m, Cp, psip, F);
        double kick = (step == n_md) ? 0.5 * eps : eps;
        for (int64_t i = 0; i < N; ++i) p[i] += kick * F[i];
    }
    free(F);
}

/* Conjugate gradients (Hestenes-Stiefel) for A x = b, A symmetric positive
 * definite.  Returns the iteration count, or -1 without convergence. */
int or_cg_solve(const or_model *m, const double *b, double *x, double tol, int max_iter) {
    int64_t N = or_num_sites(m);
    double *r = (double *)malloc(sizeof(double) * N);
    double *d = (double *)malloc(sizeof(double) * N);
    double *Ad = (double *)malloc(sizeof(double) * N);
    for (int64_t i = 0; i < N; ++i) {
        x[i] = 0.0;
        r[i] = b[i];
        d[i] = b[i];
    }
    double rr = 0, bb = 0;
    for (int64_t i = 0; i < N; ++i) {
        rr += r[i] * r[i];
        bb += b[i] * b[i];
    }
    int it = -1;
    for (int k = 0; k < max_iter; ++k) {
        if (rr <= tol * tol * bb) {
            it = k;
            break;
        }
        or_apply_A(m, d, Ad);
        double dAd = 0;
        for (int64_t i = 0; i < N; ++i) dAd += d[i] * Ad[i];
        double alpha = rr / dAd;
        double rr_new = 0;
        for (int64_t i = 0; i < N; ++i) {
            x[i] += alpha * d[i];
            r[i] -= alpha * Ad[i];
            rr_new += r[i] * r[i];
        }
        for (int64_t i = 0; i < N; ++i) d[i] = r[i] + (rr_new / rr) * d[i];
        rr = rr_new;
    }
    free(r);
    free(d);
    free(Ad);
    return it;
}
