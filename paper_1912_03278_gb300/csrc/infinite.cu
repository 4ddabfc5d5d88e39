// infinite.cu -- FP32 HMC trajectories of the infinite-range (all-to-all)
// Ising model of the appendix, one CTA per chain, whole trajectories per
// launch.
//
// Connectivity K_ij = 1/N for i != j (0 on the diagonal), so with
// kappa = beta*J/N the matrix A = beta*J*K + C*1 acts as
//     (A x)_i = kappa * (sum_j x_j - x_i) + C * x_i :
// one block-wide sum per product and an O(N) per-site update, no GEMM.
// Per force evaluation (Sec. 3, F = A (tanh(A psi + h') - psi)):
//   sweep 1:  a = A psi,  t = tanh(a + h'),  u = t - psi,  U = sum_i u_i
//   sweep 2:  F = A u (from U),  p += kick*eps*F,  psi' = psi + drift*eps*p,
//             sum_i psi'_i for the next evaluation
// Each thread owns the same sites in both sweeps (site quads q = tid + k*nt),
// so sweep 2 recomputes u from psi with the identical instructions rather
// than storing it.  The last pass of a trajectory also evaluates the
// proposal's action to FP64 accuracy in double-float arithmetic, the kinetic
// energies and the Sec. 4 estimators; the CTA takes the Metropolis decision
// itself (as the lattice kernel does).
#include <cuda_runtime.h>

#include "df32.cuh"
#include "device_common.cuh"
#include "internal.h"

namespace ihmc {
namespace {

constexpr int INF_MAX_THREADS = 256;

// Four consecutive sites 4q..4q+3 of one chain; sites at or beyond N read as
// zero and are never stored.  V4: N is a multiple of 4, so a quad is one
// aligned float4.
struct Quad {
    float v[4];
};

template <bool V4>
__device__ __forceinline__ Quad ldq(const float *__restrict__ base, int64_t i0, int64_t N) {
    Quad r;
    if constexpr (V4) {
        const float4 t = *reinterpret_cast<const float4 *>(base + i0);
        r.v[0] = t.x; r.v[1] = t.y; r.v[2] = t.z; r.v[3] = t.w;
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) r.v[k] = (i0 + k < N) ? base[i0 + k] : 0.0f;
    }
    return r;
}

template <bool V4>
__device__ __forceinline__ void stq(float *__restrict__ base, int64_t i0, int64_t N, const Quad &r) {
    if constexpr (V4) {
        *reinterpret_cast<float4 *>(base + i0) = make_float4(r.v[0], r.v[1], r.v[2], r.v[3]);
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (i0 + k < N) base[i0 + k] = r.v[k];
    }
}

// Number of valid sites in the quad starting at i0.
__device__ __forceinline__ int quad_len(int64_t i0, int64_t N) {
    const int64_t r = N - i0;
    return r >= 4 ? 4 : (int)r;
}

// Per-thread accumulators of one trajectory (same scheme as the lattice
// kernel: double-float energies with a separate low-word sum, Kahan FP32
// estimator sums).
struct Acc {
    f2 K0, K1, S;
    float K0lo, K1lo, Slo;
    float sT, cT, sAT, cAT, sHT, cHT;
    int sS;
};

__device__ __forceinline__ Acc acc_zero() {
    Acc a;
    a.K0 = a.K1 = a.S = f2{0.0f, 0.0f};
    a.K0lo = a.K1lo = a.Slo = 0.0f;
    a.sT = a.cT = a.sAT = a.cAT = a.sHT = a.cHT = 0.0f;
    a.sS = 0;
    return a;
}

// Per-chain constants: kappa = beta*J/N is stored in ChainParams::bJ.
struct InfConst {
    f2 C2, k2, hp2, beta2;
    float Cf, kf, betaf, hpf;
    bool hzero;
};

__device__ __forceinline__ InfConst inf_const(const ChainParams &prm) {
    InfConst k;
    k.C2 = df_from_double(prm.C);
    k.k2 = df_from_double(prm.bJ);
    k.hp2 = df_from_double(prm.hp);
    k.beta2 = df_from_double(prm.beta);
    k.Cf = prm.Cf;
    k.kf = prm.bJf;
    k.betaf = prm.betaf;
    k.hpf = prm.hpf;
    k.hzero = prm.hp == 0.0;
    return k;
}

__device__ __forceinline__ float field_f(const FusedArgs &A, const InfConst &kc, int64_t i) {
    return A.hdf ? kc.betaf * A.hdf[i].x : kc.hpf;
}

// t_i = tanh((A x)_i + h'_i) for the quad, with Sf = sum_j x_j in FP32: the
// one formula both the force sweeps and the estimators use.
__device__ __forceinline__ Quad quad_tanh(const FusedArgs &A, const InfConst &kc, const Quad &x,
                                          float Sf, int64_t i0, int n) {
    Quad t;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float hf = (k < n) ? field_f(A, kc, i0 + k) : 0.0f;
        const float a = fmaf(kc.Cf, x.v[k], kc.kf * (Sf - x.v[k]));
        t.v[k] = tanh_f(a + hf);
    }
    return t;
}

// Action terms of the quad's sites of S(x) (Sec. 2, Eq. phi_psi_substitution:
// S_i = 1/2 x_i a_i - |y_i| - log(1 + exp(-2|y_i|)), a = A x, y = a + h') in
// double-float arithmetic with Sx = sum_j x_j as a double-float; the Sec. 4
// estimator sums from the force-form tanh values t, and one conditional spin
// draw per site.
__device__ __forceinline__ void quad_action(const FusedArgs &A, const InfConst &kc, const Quad &x,
                                            const Quad &t, f2 Sx, int64_t i0, int n,
                                            uint32_t spin_traj, uint64_t seed, int chain,
                                            const float4 *tab, Acc &acc) {
    const float4 w = spin_u4_f32((uint32_t)(i0 >> 2), spin_traj, (uint32_t)chain, seed);
    const float su[4] = {w.x, w.y, w.z, w.w};
    const bool has_h = A.hdf || !kc.hzero;
    f2 sv{0.0f, 0.0f};
    float vT = 0.0f, vAT = 0.0f, vHT = 0.0f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (k >= n) break;
        const float ps = x.v[k];
        const f2 off = df_add_f(Sx, -ps);   // sum over j != i
        const f2 a = df_add_q(df_mul_f(kc.C2, ps), df_mul(kc.k2, off));
        f2 y = a;
        if (A.hdf) {
            const float2 hh = A.hdf[i0 + k];
            y = df_add_q(a, df_mul(kc.beta2, f2{hh.x, hh.y}));
        } else if (!kc.hzero) {
            y = df_add_q(a, kc.hp2);
        }
        const f2 ay = y.hi < 0.0f ? df_neg(y) : y;
        const f2 gl = log1pexp_neg(f2{2.0f * ay.hi, 2.0f * ay.lo}, tab);
        sv = df_add_q(sv, df_add_q(df_mul_f(a, 0.5f * ps), df_neg(df_add_q(ay, gl))));
        const float tq = t.v[k];
        vT += tq;
        vAT = fmaf(a.hi, tq, vAT);
        if (has_h) vHT = fmaf(field_f(A, kc, i0 + k), tq, vHT);
        acc.sS += (su[k] < (1.0f + tq) * 0.5f) ? 1 : -1;
    }
    acc_add(acc.S, acc.Slo, sv);
    kahan_add(acc.sT, acc.cT, vT);
    kahan_add(acc.sAT, acc.cAT, vAT);
    if (has_h) kahan_add(acc.sHT, acc.cHT, vHT);
}

__device__ __forceinline__ float *sel3(const FusedArgs &A, int i) {
    return i == 0 ? A.psi[0] : (i == 1 ? A.psi[1] : A.psi[2]);
}

// Sum of the quad's valid sites.  Every sum over a configuration adds these
// quad sums in the same order (thread t: quads t, t + nt, ...; then the block
// sum), so the sum kept while drifting equals the one recomputed from the
// stored buffer bit for bit, and the force stays a function of psi alone.
__device__ __forceinline__ float quad_sum(const Quad &v, int n) {
    const float a = v.v[0] + (n > 1 ? v.v[1] : 0.0f);
    const float b = (n > 2 ? v.v[2] : 0.0f) + (n > 3 ? v.v[3] : 0.0f);
    return a + b;
}

// sum_i x_i of one chain's buffer, identical in every thread.
template <bool V4>
__device__ double chain_sum(const float *__restrict__ x, int64_t N, double *red) {
    const int64_t nq = (N + 3) >> 2;
    f2 s{0.0f, 0.0f};
    for (int64_t q = threadIdx.x; q < nq; q += blockDim.x) {
        const int64_t i0 = 4 * q;
        s = df_add_f(s, quad_sum(ldq<V4>(x, i0, N), quad_len(i0, N)));
    }
    double r[1] = {df_to_double(s)};
    block_sum<1>(r, red);
    return r[0];
}

struct PassCfg {
    int src, dst;
    float kick, drift;   // already multiplied by eps
    uint32_t traj;
};

// One force evaluation.  Spsi: sum of the source configuration on entry, of
// the drifted one on exit (unchanged by the last pass, which does not drift).
template <bool V4, bool FIRST, bool LAST>
__device__ void inf_pass(const FusedArgs &A, const PassCfg &pc, const InfConst &kc, int chain,
                         double &Spsi, double *red, const float4 *tab, Acc &acc) {
    const int64_t N = A.g.N;
    const int64_t nq = (N + 3) >> 2;
    const int64_t cbase = (int64_t)chain * N;
    const float *__restrict__ src = sel3(A, pc.src) + cbase;
    float *__restrict__ dst = sel3(A, pc.dst) + cbase;
    float *__restrict__ gp = A.p + cbase;
    const float Sf = (float)Spsi;

    // ---- sweep 1: U = sum_i (tanh(A psi + h')_i - psi_i) ----
    f2 su{0.0f, 0.0f};
    const f2 Sdf = df_from_double(Spsi);
    for (int64_t q = threadIdx.x; q < nq; q += blockDim.x) {
        const int64_t i0 = 4 * q;
        const int n = quad_len(i0, N);
        const Quad x = ldq<V4>(src, i0, N);
        const Quad t = quad_tanh(A, kc, x, Sf, i0, n);
        float s4 = 0.0f;
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (k < n) s4 += t.v[k] - x.v[k];
        su = df_add_f(su, s4);
        // the last pass's configuration is the proposal
        if constexpr (LAST) quad_action(A, kc, x, t, Sdf, i0, n, pc.traj, A.seed, chain, tab, acc);
    }
    double r[1] = {df_to_double(su)};
    block_sum<1>(r, red);
    const float Uf = (float)r[0];

    // ---- sweep 2: kick with F = A u, drift ----
    f2 sp{0.0f, 0.0f};
    for (int64_t q = threadIdx.x; q < nq; q += blockDim.x) {
        const int64_t i0 = 4 * q;
        const int n = quad_len(i0, N);
        const Quad x = ldq<V4>(src, i0, N);
        const Quad t = quad_tanh(A, kc, x, Sf, i0, n);
        Quad pv;
        if constexpr (FIRST) {
            const float4 w = momenta4_f32((uint32_t)q, pc.traj, (uint32_t)chain, A.seed);
            pv.v[0] = w.x; pv.v[1] = w.y; pv.v[2] = w.z; pv.v[3] = w.w;
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (k < n) acc_add(acc.K0, acc.K0lo, two_prod(pv.v[k], 0.5f * pv.v[k]));
        } else {
            pv = ldq<V4>(gp, i0, N);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float u = t.v[k] - x.v[k];
            const float F = fmaf(kc.Cf, u, kc.kf * (Uf - u));
            pv.v[k] = fmaf(pc.kick, F, pv.v[k]);
        }
        stq<V4>(gp, i0, N, pv);
        if constexpr (LAST) {
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (k < n) acc_add(acc.K1, acc.K1lo, two_prod(pv.v[k], 0.5f * pv.v[k]));
        } else {
            Quad xn;
#pragma unroll
            for (int k = 0; k < 4; ++k) xn.v[k] = fmaf(pc.drift, pv.v[k], x.v[k]);
            stq<V4>(dst, i0, N, xn);
            sp = df_add_f(sp, quad_sum(xn, n));
        }
    }
    if constexpr (!LAST) {
        double w[1] = {df_to_double(sp)};
        block_sum<1>(w, red);
        Spsi = w[0];
    }
}

// Action S(sign*x) of the chain's buffer `buf` with the estimators and one
// conditional spin draw per site (evaluation of the current state, sign
// flip proposal).
template <bool V4>
__device__ void inf_action(const FusedArgs &A, const InfConst &kc, int chain, int buf, float sign,
                           uint32_t spin_traj, uint64_t seed, double *red, const float4 *tab,
                           Acc &acc) {
    const int64_t N = A.g.N;
    const int64_t nq = (N + 3) >> 2;
    const float *__restrict__ x = sel3(A, buf) + (int64_t)chain * N;
    const double Sx = (double)sign * chain_sum<V4>(x, N, red);
    const float Sf = (float)Sx;
    const f2 Sdf = df_from_double(Sx);
    for (int64_t q = threadIdx.x; q < nq; q += blockDim.x) {
        const int64_t i0 = 4 * q;
        const int n = quad_len(i0, N);
        Quad v = ldq<V4>(x, i0, N);
#pragma unroll
        for (int k = 0; k < 4; ++k) v.v[k] *= sign;
        const Quad t = quad_tanh(A, kc, v, Sf, i0, n);
        quad_action(A, kc, v, t, Sdf, i0, n, spin_traj, seed, chain, tab, acc);
    }
}

__device__ __forceinline__ int buf_loc(int start, int j) {
    if (j == 0) return start;
    return (start + ((j & 1) ? 1 : 2)) % 3;
}

__device__ __forceinline__ void set_obs(ChainState *st, const ChainParams &prm, double sT,
                                        double sAT, double sHT, double sS, double invN) {
    const double m = sT * invN;
    st->obs[0] = m;
    st->obs[1] = 0.5 * prm.C - 0.5 * sAT * invN - sHT * invN;
    st->obs[2] = fabs(sS) * invN;
    st->obs[3] = fabs(m);
}

template <bool V4>
__global__ void __launch_bounds__(INF_MAX_THREADS) infinite_kernel(FusedArgs A, Schedule S) {
    __shared__ float4 tab_s[LOG1PEXP_NODES];
    __shared__ double red[32 * 8];
    __shared__ int bcast[2];
    const int chain = A.chain0 + blockIdx.x;
    if (chain >= A.n_chains) return;
    const int64_t N = A.g.N;
    ChainState *st = A.state + chain;
    const ChainParams prm = A.params[chain];
    const double invN = 1.0 / (double)N;

    if (A.mode == MODE_MOMENTA) {
        float *gp = A.p + (int64_t)chain * N;
        for (int64_t q = threadIdx.x; q < ((N + 3) >> 2); q += blockDim.x) {
            const float4 w = momenta4_f32((uint32_t)q, A.traj0, (uint32_t)chain, A.seed);
            stq<V4>(gp, 4 * q, N, Quad{{w.x, w.y, w.z, w.w}});
        }
        return;
    }
    for (int i = threadIdx.x; i < LOG1PEXP_NODES; i += blockDim.x) tab_s[i] = A.lpe_tab[i];
    __syncthreads();
    const InfConst kc = inf_const(prm);

    if (A.mode == MODE_EVAL) {
        Acc acc = acc_zero();
        const int start = st->start;
        inf_action<V4>(A, kc, chain, start, 1.0f, TRAJ_INIT, 0, red, tab_s, acc);
        double v[5] = {acc_val(acc.S, acc.Slo), kahan_val(acc.sT, acc.cT),
                       kahan_val(acc.sAT, acc.cAT), kahan_val(acc.sHT, acc.cHT), (double)acc.sS};
        block_sum<5>(v, red);
        if (threadIdx.x == 0) {
            st->S = v[0];
            set_obs(st, prm, v[1], v[2], v[3], v[4], invN);
            st->prop = start;
        }
        return;
    }

    int start = st->start;
    // sum of the current configuration, carried from trajectory to trajectory
    double Sstart = chain_sum<V4>(sel3(A, start) + (int64_t)chain * N, N, red);
    for (int k = 0; k < A.n_traj; ++k) {
        const uint32_t traj = A.traj0 + (uint32_t)k;
        Acc acc = acc_zero();
        double Spsi = Sstart;
        // the integrator's force passes; the first draws the momenta (Sec. 3
        // refresh), the last evaluates the proposal's action
        for (int j = 0; j < S.n_pass; ++j) {
            PassCfg pc;
            pc.src = buf_loc(start, j);
            pc.dst = buf_loc(start, j + 1);
            pc.kick = (float)(S.kick[j] * prm.eps);
            pc.drift = (float)(S.drift[j] * prm.eps);
            pc.traj = traj;
            const bool first = j == 0, last = j == S.n_pass - 1;
            if (first && last) inf_pass<V4, true, true>(A, pc, kc, chain, Spsi, red, tab_s, acc);
            else if (first) inf_pass<V4, true, false>(A, pc, kc, chain, Spsi, red, tab_s, acc);
            else if (last) inf_pass<V4, false, true>(A, pc, kc, chain, Spsi, red, tab_s, acc);
            else inf_pass<V4, false, false>(A, pc, kc, chain, Spsi, red, tab_s, acc);
        }
        const int prop = buf_loc(start, S.n_pass - 1);
        double v[7] = {acc_val(acc.K0, acc.K0lo), acc_val(acc.K1, acc.K1lo),
                       acc_val(acc.S, acc.Slo), kahan_val(acc.sT, acc.cT),
                       kahan_val(acc.sAT, acc.cAT), kahan_val(acc.sHT, acc.cHT), (double)acc.sS};
        block_sum<7>(v, red);
        if (threadIdx.x == 0) {
            const double S0 = st->S;
            const double dH = (v[1] + v[2]) - (v[0] + S0);
            const double logu = accept_logu(traj, (uint32_t)chain, A.seed, PURPOSE_ACC);
            const bool accd = logu < -dH;
            st->prop = prop;
            st->rec[ISING_REC_DH] = dH;
            st->rec[ISING_REC_LOGU] = logu;
            st->rec[ISING_REC_ACCEPTED] = accd ? 1.0 : 0.0;
            st->rec[ISING_REC_K0] = v[0];
            st->rec[ISING_REC_S0] = S0;
            st->rec[ISING_REC_K1] = v[1];
            st->rec[ISING_REC_S1] = v[2];
            st->rec[ISING_REC_FLIPPED] = 0.0;
            if (accd) {
                st->start = prop;
                st->S = v[2];
                set_obs(st, prm, v[3], v[4], v[5], v[6], invN);
            }
            bcast[0] = accd ? prop : start;
        }
        __syncthreads();
        if (bcast[0] != start) Sstart = Spsi;   // accepted: the proposal's sum
        start = bcast[0];
        __syncthreads();
        // ---- optional global sign flip psi -> -psi (Sec. 3, ergodicity) ----
        if (A.flip_every > 0 && ((traj + 1) % (uint32_t)A.flip_every) == 0) {
            Acc fa = acc_zero();
            inf_action<V4>(A, kc, chain, start, -1.0f, traj, A.seed, red, tab_s, fa);
            double w[5] = {acc_val(fa.S, fa.Slo), kahan_val(fa.sT, fa.cT),
                           kahan_val(fa.sAT, fa.cAT), kahan_val(fa.sHT, fa.cHT), (double)fa.sS};
            block_sum<5>(w, red);
            if (threadIdx.x == 0) {
                const double lu = accept_logu(traj, (uint32_t)chain, A.seed, PURPOSE_FLIP);
                const bool fl = lu < -(w[0] - st->S);
                if (fl) {
                    st->S = w[0];
                    set_obs(st, prm, w[1], w[2], w[3], w[4], invN);
                    st->rec[ISING_REC_FLIPPED] = 1.0;
                }
                bcast[1] = fl ? 1 : 0;
            }
            __syncthreads();
            if (bcast[1]) {
                // -psi goes to the buffer that is neither current nor the
                // proposal, so the MD end point stays readable
                const int f = (start != prop) ? 3 - start - prop : (start + 1) % 3;
                const float *gs = sel3(A, start) + (int64_t)chain * N;
                float *gf = sel3(A, f) + (int64_t)chain * N;
                for (int64_t i = threadIdx.x; i < N; i += blockDim.x) gf[i] = -gs[i];
                start = f;
                Sstart = -Sstart;   // negation is exact in every partial sum
                if (threadIdx.x == 0) st->start = f;
            }
            __syncthreads();
        }
        // ---- measurement: a repeated configuration repeats its measurement ----
        if (threadIdx.x == 0 && (int64_t)traj >= (int64_t)A.n_therm) {
            double *sm = st->sums;
            const double dH = st->rec[ISING_REC_DH];
            sm[ISING_SUM_NMEAS] += 1.0;
            sm[ISING_SUM_NACC] += st->rec[ISING_REC_ACCEPTED];
            sm[ISING_SUM_M] += st->obs[0];
            sm[ISING_SUM_M2] += st->obs[0] * st->obs[0];
            sm[ISING_SUM_E] += st->obs[1];
            sm[ISING_SUM_E2] += st->obs[1] * st->obs[1];
            sm[ISING_SUM_ABSM] += st->obs[2];
            sm[ISING_SUM_ABSM2] += st->obs[2] * st->obs[2];
            sm[ISING_SUM_DH] += dH;
            sm[ISING_SUM_EXPMDH] += exp(-dH);
        }
        __syncthreads();
    }
}

}  // namespace

// Threads per CTA: one per site quad up to INF_MAX_THREADS, a multiple of 32.
// Fixed by N alone, so the order of every block sum (and with it every
// result) depends on nothing but the model.
int infinite_threads(int64_t N) {
    const int64_t nq = (N + 3) / 4;
    int64_t t = (nq + 31) / 32 * 32;
    if (t > INF_MAX_THREADS) t = INF_MAX_THREADS;
    if (t < 32) t = 32;
    return (int)t;
}

cudaError_t infinite_node(const FusedArgs &a, cudaKernelNodeParams *np, void **args) {
    np->func = (a.g.N % 4 == 0) ? reinterpret_cast<void *>(infinite_kernel<true>)
                                : reinterpret_cast<void *>(infinite_kernel<false>);
    np->gridDim = dim3((unsigned)(a.n_chains - a.chain0), 1, 1);
    np->blockDim = dim3((unsigned)infinite_threads(a.g.N), 1, 1);
    np->sharedMemBytes = 0;
    np->kernelParams = args;
    np->extra = nullptr;
    return cudaSuccess;
}

cudaError_t launch_infinite(const FusedArgs &a, const Schedule &sched, cudaStream_t s) {
    cudaKernelNodeParams np;
    void *args[2] = {const_cast<FusedArgs *>(&a), const_cast<Schedule *>(&sched)};
    cudaError_t e = infinite_node(a, &np, args);
    if (e != cudaSuccess) return e;
    if (np.gridDim.x == 0) return cudaSuccess;
    return cudaLaunchKernel(np.func, np.gridDim, np.blockDim, np.kernelParams, np.sharedMemBytes, s);
}

}  // namespace ihmc
