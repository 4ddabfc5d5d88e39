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
// Each thread owns the same sites in both sweeps (site quads q = tid + k*nt).
// Two variants with bit-identical results:
//  * resident (N <= 32 * threads): the thread keeps its quads' psi, p and u in
//    registers for the whole trajectory; global memory is read once per
//    launch (and after a rejection) and written once per trajectory (the
//    proposal and the end momenta);
//  * streaming (any N): psi and p are re-read from global memory every pass,
//    sweep 2 recomputes u from psi with the identical instructions.
// Every sum adds the same per-quad partial sums in the same order in both,
// and the thread count depends on N alone.  The last pass of a trajectory also evaluates the
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

// CTA-wide sums in FP32-pipe arithmetic (FP64 issues at a small fraction of
// the FP32 rate on GB300), blockDim a multiple of 32 and at most 256.  The
// order is fixed and the same in every thread: a shuffle tree to lane 0 of
// each warp, then lanes 0..7 of every warp over the per-warp totals.
struct Red {
    float *f;   // 2 x 8 floats, halves used alternately: one barrier per sum
    f2 *d;      // 8 x 8 double-floats
    int par;
};

__device__ __forceinline__ float bsum_f32(float v, Red &r) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    float *buf = r.f + 8 * r.par;
    r.par ^= 1;
    if (lane == 0) buf[warp] = v;
    __syncthreads();
    float w = lane < (int)(blockDim.x >> 5) ? buf[lane] : 0.0f;
#pragma unroll
    for (int off = 4; off > 0; off >>= 1) w += __shfl_down_sync(0xffffffffu, w, off);
    return __shfl_sync(0xffffffffu, w, 0);
}

__device__ __forceinline__ f2 shfl_down_f2(f2 v, int off) {
    return f2{__shfl_down_sync(0xffffffffu, v.hi, off), __shfl_down_sync(0xffffffffu, v.lo, off)};
}

template <int NV>
__device__ __forceinline__ void bsum_f2(f2 (&v)[NV], Red &r) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[k] = df_add(v[k], shfl_down_f2(v[k], off));
    __syncthreads();   // earlier readers of r.d are done
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) r.d[warp * NV + k] = v[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        f2 w = lane < (int)(blockDim.x >> 5) ? r.d[lane * NV + k] : f2{0.0f, 0.0f};
#pragma unroll
        for (int off = 4; off > 0; off >>= 1) w = df_add(w, shfl_down_f2(w, off));
        v[k] = f2{__shfl_sync(0xffffffffu, w.hi, 0), __shfl_sync(0xffffffffu, w.lo, 0)};
    }
}

// Sum of a configuration: the thread's partial over its quads (double-float,
// quads in increasing order) and the FP32 CTA total of the partials' high
// words, the value the force uses.  The double-float CTA total (the action's
// value) is formed from the partials only where the action needs it.
// Negation is exact in every step, so the sum of -psi is the negated sum.
struct CSum {
    f2 part;
    float Sf;
};

__device__ __forceinline__ CSum csum_make(f2 part, Red &r) { return CSum{part, bsum_f32(part.hi, r)}; }
__device__ __forceinline__ CSum csum_neg(const CSum &c) { return CSum{df_neg(c.part), -c.Sf}; }
__device__ __forceinline__ f2 csum_exact(const CSum &c, Red &r) {
    f2 v[1] = {c.part};
    bsum_f2<1>(v, r);
    return v[0];
}

// Sum of one chain's buffer.
template <bool V4>
__device__ CSum chain_sum(const float *__restrict__ x, int64_t N, Red &r) {
    const int64_t nq = (N + 3) >> 2;
    f2 s{0.0f, 0.0f};
    for (int64_t q = threadIdx.x; q < nq; q += blockDim.x) {
        const int64_t i0 = 4 * q;
        s = df_add_f(s, quad_sum(ldq<V4>(x, i0, N), quad_len(i0, N)));
    }
    return csum_make(s, r);
}

struct PassCfg {
    int src, dst;
    float kick, drift;   // already multiplied by eps
    uint32_t traj;
};

// One force evaluation.  cs: sum of the source configuration on entry, of
// the drifted one on exit (unchanged by the last pass, which does not drift).
template <bool V4, bool FIRST, bool LAST>
__device__ void inf_pass(const FusedArgs &A, const PassCfg &pc, const InfConst &kc, int chain,
                         CSum &cs, Red &red, const float4 *tab, Acc &acc) {
    const int64_t N = A.g.N;
    const int64_t nq = (N + 3) >> 2;
    const int64_t cbase = (int64_t)chain * N;
    const float *__restrict__ src = sel3(A, pc.src) + cbase;
    float *__restrict__ dst = sel3(A, pc.dst) + cbase;
    float *__restrict__ gp = A.p + cbase;
    const float Sf = cs.Sf;

    // ---- sweep 1: U = sum_i (tanh(A psi + h')_i - psi_i) ----
    float su = 0.0f;
    f2 Sdf{0.0f, 0.0f};
    if constexpr (LAST) Sdf = csum_exact(cs, red);
    for (int64_t q = threadIdx.x; q < nq; q += blockDim.x) {
        const int64_t i0 = 4 * q;
        const int n = quad_len(i0, N);
        const Quad x = ldq<V4>(src, i0, N);
        const Quad t = quad_tanh(A, kc, x, Sf, i0, n);
        Quad u;
#pragma unroll
        for (int k = 0; k < 4; ++k) u.v[k] = t.v[k] - x.v[k];
        su += quad_sum(u, n);
        // the last pass's configuration is the proposal
        if constexpr (LAST) quad_action(A, kc, x, t, Sdf, i0, n, pc.traj, A.seed, chain, tab, acc);
    }
    const float Uf = bsum_f32(su, red);

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
    if constexpr (!LAST) cs = csum_make(sp, red);
}

// Action S(sign*x) of the chain's buffer `buf` with the estimators and one
// conditional spin draw per site (evaluation of the current state, sign
// flip proposal).
template <bool V4>
__device__ void inf_action(const FusedArgs &A, const InfConst &kc, int chain, int buf, float sign,
                           uint32_t spin_traj, uint64_t seed, Red &red, const float4 *tab,
                           Acc &acc) {
    const int64_t N = A.g.N;
    const int64_t nq = (N + 3) >> 2;
    const float *__restrict__ x = sel3(A, buf) + (int64_t)chain * N;
    CSum c = chain_sum<V4>(x, N, red);
    if (sign < 0.0f) c = csum_neg(c);
    const float Sf = c.Sf;
    const f2 Sdf = csum_exact(c, red);
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

// Metropolis decision of trajectory traj (Sec. 3) from the block totals v =
// {K0, K1, S1, sum t, sum a.t, sum h'.t, sum of spins} of the proposal held
// in buffer prop; thread 0 updates the chain state.  Returns the buffer of
// the chain's current configuration afterwards (in every thread).
__device__ int metropolis(const FusedArgs &A, ChainState *st, const ChainParams &prm, int chain,
                          uint32_t traj, int start, int prop, const double (&v)[7], double invN,
                          int *bcast) {
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
    const int cur = bcast[0];
    __syncthreads();
    return cur;
}

// Sign-flip proposal psi -> -psi (Sec. 3) from the block totals w = {S(-psi),
// sum t, sum a.t, sum h'.t, sum of spins}; returns 1 (every thread) if taken.
__device__ int flip_decision(const FusedArgs &A, ChainState *st, const ChainParams &prm, int chain,
                             uint32_t traj, const double (&w)[5], double invN, int *bcast) {
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
    const int fl = bcast[1];
    __syncthreads();
    return fl;
}

// Measurement after the Metropolis step: a repeated configuration repeats its
// measurement (thread 0).
__device__ __forceinline__ void measure(const FusedArgs &A, ChainState *st, uint32_t traj) {
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

// CTA totals of a trajectory's accumulators as doubles, identical in every
// thread: {K0, K1, S, sum t, sum a.t, sum h'.t, sum of spins}.  The
// per-thread values enter as exact double-floats.
__device__ __forceinline__ f2 int_f2(int n) {
    const float hi = (float)n;
    return f2{hi, (float)(n - (int)hi)};
}

__device__ __forceinline__ void acc_totals(const Acc &acc, double (&v)[7], Red &red) {
    f2 t[7] = {df_add_f(acc.K0, acc.K0lo), df_add_f(acc.K1, acc.K1lo), df_add_f(acc.S, acc.Slo),
               two_sum(acc.sT, -acc.cT),  two_sum(acc.sAT, -acc.cAT), two_sum(acc.sHT, -acc.cHT),
               int_f2(acc.sS)};
    bsum_f2<7>(t, red);
#pragma unroll
    for (int k = 0; k < 7; ++k) v[k] = df_to_double(t[k]);
}

// The same for an action sweep: {S, sum t, sum a.t, sum h'.t, sum of spins}.
__device__ __forceinline__ void action_totals(const Acc &acc, double (&w)[5], Red &red) {
    f2 t[5] = {df_add_f(acc.S, acc.Slo), two_sum(acc.sT, -acc.cT), two_sum(acc.sAT, -acc.cAT),
               two_sum(acc.sHT, -acc.cHT), int_f2(acc.sS)};
    bsum_f2<5>(t, red);
#pragma unroll
    for (int k = 0; k < 5; ++k) w[k] = df_to_double(t[k]);
}

// ---------------------------------------------------------------- resident --
// The thread's quads q = tid + k*nt, k < QPT, held in registers: x (psi), pm
// (p); u between the two sweeps in shared memory (us[q], written and read by
// the owning thread only).  One force evaluation, the same arithmetic in the
// same order as inf_pass.  The first pass's momentum draw and the last pass's
// action run in loops that are not unrolled, through a second shared array
// (aux[q], again the owning thread's only): their code then appears once, not
// once per quad, which keeps the kernel's instruction footprint small.
template <bool V4, int QPT, bool FULL, bool FIRST, bool LAST>
__device__ __forceinline__ void res_pass(const FusedArgs &A, const InfConst &kc, int chain,
                                         uint32_t traj, float kick, float drift, Quad (&x)[QPT],
                                         Quad (&pm)[QPT], float4 *us, CSum &cs, Red &red,
                                         const float4 *tab, Acc &acc) {
    const int64_t N = A.g.N;
    const int64_t nq = (N + 3) >> 2;
    const float Sf = cs.Sf;
    float4 *aux = us + QPT * blockDim.x;
    constexpr bool ONE_PASS = FIRST && LAST;   // (never with two or more passes)
    if constexpr (FIRST && !ONE_PASS) {
#pragma unroll 1
        for (int k = 0; k < QPT; ++k) {
            const int64_t q = threadIdx.x + (int64_t)k * blockDim.x;
            if (FULL || q < nq) aux[q] = momenta4_f32((uint32_t)q, traj, (uint32_t)chain, A.seed);
        }
    }
    float su = 0.0f;
    f2 Sdf{0.0f, 0.0f};
    if constexpr (LAST) Sdf = csum_exact(cs, red);
#pragma unroll
    for (int k = 0; k < QPT; ++k) {
        const int64_t q = threadIdx.x + (int64_t)k * blockDim.x;
        if (FULL || q < nq) {
            const int64_t i0 = 4 * q;
            const int n = (FULL ? 4 : quad_len(i0, N));
            const Quad t = quad_tanh(A, kc, x[k], Sf, i0, n);
            Quad u;
#pragma unroll
            for (int e = 0; e < 4; ++e) u.v[e] = t.v[e] - x[k].v[e];
            us[q] = make_float4(u.v[0], u.v[1], u.v[2], u.v[3]);
            su += quad_sum(u, n);
            if constexpr (ONE_PASS)
                quad_action(A, kc, x[k], t, Sdf, i0, n, traj, A.seed, chain, tab, acc);
            else if constexpr (LAST)
                aux[q] = make_float4(x[k].v[0], x[k].v[1], x[k].v[2], x[k].v[3]);
        }
    }
    if constexpr (LAST && !ONE_PASS) {
        // the proposal's action, quads in the same order (t recomputed: the
        // same function of the same values)
#pragma unroll 1
        for (int k = 0; k < QPT; ++k) {
            const int64_t q = threadIdx.x + (int64_t)k * blockDim.x;
            if (FULL || q < nq) {
                const int64_t i0 = 4 * q;
                const int n = (FULL ? 4 : quad_len(i0, N));
                const float4 w = aux[q];
                const Quad xq{{w.x, w.y, w.z, w.w}};
                const Quad t = quad_tanh(A, kc, xq, Sf, i0, n);
                quad_action(A, kc, xq, t, Sdf, i0, n, traj, A.seed, chain, tab, acc);
            }
        }
    }
    const float Uf = bsum_f32(su, red);
    f2 sp{0.0f, 0.0f};
#pragma unroll
    for (int k = 0; k < QPT; ++k) {
        const int64_t q = threadIdx.x + (int64_t)k * blockDim.x;
        if (FULL || q < nq) {
            const int n = (FULL ? 4 : quad_len(4 * q, N));
            if constexpr (FIRST) {
                const float4 w = ONE_PASS ? momenta4_f32((uint32_t)q, traj, (uint32_t)chain, A.seed)
                                          : aux[q];
                pm[k].v[0] = w.x; pm[k].v[1] = w.y; pm[k].v[2] = w.z; pm[k].v[3] = w.w;
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (e < n) acc_add(acc.K0, acc.K0lo, two_prod(pm[k].v[e], 0.5f * pm[k].v[e]));
            }
            const float4 u4 = us[q];
            const float u[4] = {u4.x, u4.y, u4.z, u4.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float F = fmaf(kc.Cf, u[e], kc.kf * (Uf - u[e]));
                pm[k].v[e] = fmaf(kick, F, pm[k].v[e]);
            }
            if constexpr (LAST) {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (e < n) acc_add(acc.K1, acc.K1lo, two_prod(pm[k].v[e], 0.5f * pm[k].v[e]));
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e) x[k].v[e] = fmaf(drift, pm[k].v[e], x[k].v[e]);
                sp = df_add_f(sp, quad_sum(x[k], n));
            }
        }
    }
    if constexpr (!LAST) cs = csum_make(sp, red);
}

template <bool V4, int QPT, bool FULL>
__device__ __forceinline__ void res_load(const float *__restrict__ g, int64_t N, Quad (&x)[QPT]) {
    const int64_t nq = (N + 3) >> 2;
#pragma unroll
    for (int k = 0; k < QPT; ++k) {
        const int64_t q = threadIdx.x + (int64_t)k * blockDim.x;
        if (FULL || q < nq) x[k] = ldq<V4>(g, 4 * q, N);
    }
}

template <bool V4, int QPT, bool FULL>
__device__ __forceinline__ void res_store(float *__restrict__ g, int64_t N, const Quad (&x)[QPT]) {
    const int64_t nq = (N + 3) >> 2;
#pragma unroll
    for (int k = 0; k < QPT; ++k) {
        const int64_t q = threadIdx.x + (int64_t)k * blockDim.x;
        if (FULL || q < nq) stq<V4>(g, 4 * q, N, x[k]);
    }
}

// Whole trajectories with the chain resident in registers.  Every thread
// reads and writes only its own quads, so no barrier guards global memory.
template <bool V4, int QPT, bool FULL>
__device__ void res_trajectories(const FusedArgs &A, const Schedule &S, const ChainParams &prm,
                                 const InfConst &kc, ChainState *st, int chain, double invN,
                                 float4 *us, Red &red, int *bcast, const float4 *tab) {
    const int64_t N = A.g.N;
    const int64_t nq = (N + 3) >> 2;
    const int64_t cbase = (int64_t)chain * N;
    Quad x[QPT], pm[QPT];
#pragma unroll
    for (int k = 0; k < QPT; ++k) x[k] = pm[k] = Quad{{0.0f, 0.0f, 0.0f, 0.0f}};
    int start = st->start;
    res_load<V4, QPT, FULL>(sel3(A, start) + cbase, N, x);
    // sum of the current configuration (the order of chain_sum)
    CSum Sstart;
    {
        f2 s{0.0f, 0.0f};
#pragma unroll
        for (int k = 0; k < QPT; ++k) {
            const int64_t q = threadIdx.x + (int64_t)k * blockDim.x;
            if (FULL || q < nq) s = df_add_f(s, quad_sum(x[k], (FULL ? 4 : quad_len(4 * q, N))));
        }
        Sstart = csum_make(s, red);
    }
    for (int it = 0; it < A.n_traj; ++it) {
        const uint32_t traj = A.traj0 + (uint32_t)it;
        Acc acc = acc_zero();
        CSum cs = Sstart;
        for (int j = 0; j < S.n_pass; ++j) {
            const float kick = (float)(S.kick[j] * prm.eps);
            const float drift = (float)(S.drift[j] * prm.eps);
            const bool first = j == 0, last = j == S.n_pass - 1;
            if (first && last)
                res_pass<V4, QPT, FULL, true, true>(A, kc, chain, traj, kick, drift, x, pm, us, cs, red, tab, acc);
            else if (first)
                res_pass<V4, QPT, FULL, true, false>(A, kc, chain, traj, kick, drift, x, pm, us, cs, red, tab, acc);
            else if (last)
                res_pass<V4, QPT, FULL, false, true>(A, kc, chain, traj, kick, drift, x, pm, us, cs, red, tab, acc);
            else
                res_pass<V4, QPT, FULL, false, false>(A, kc, chain, traj, kick, drift, x, pm, us, cs, red, tab, acc);
        }
        // the proposal and the end momenta go to global memory
        const int prop = buf_loc(start, S.n_pass - 1);
        res_store<V4, QPT, FULL>(sel3(A, prop) + cbase, N, x);
        res_store<V4, QPT, FULL>(A.p + cbase, N, pm);
        double v[7];
        acc_totals(acc, v, red);
        const int cur = metropolis(A, st, prm, chain, traj, start, prop, v, invN, bcast);
        if (cur == start) res_load<V4, QPT, FULL>(sel3(A, start) + cbase, N, x);   // rejected
        else Sstart = cs;                                                   // the proposal's sum
        start = cur;
        if (A.flip_every > 0 && ((traj + 1) % (uint32_t)A.flip_every) == 0) {
            // action of -psi from the registers (the arithmetic of inf_action)
            Acc fa = acc_zero();
            const CSum neg = csum_neg(Sstart);
            const float Sf = neg.Sf;
            const f2 Sdf = csum_exact(neg, red);
#pragma unroll
            for (int k = 0; k < QPT; ++k) {
                const int64_t q = threadIdx.x + (int64_t)k * blockDim.x;
                if (FULL || q < nq) {
                    const int64_t i0 = 4 * q;
                    const int n = (FULL ? 4 : quad_len(i0, N));
                    Quad v4 = x[k];
#pragma unroll
                    for (int e = 0; e < 4; ++e) v4.v[e] *= -1.0f;
                    const Quad t = quad_tanh(A, kc, v4, Sf, i0, n);
                    quad_action(A, kc, v4, t, Sdf, i0, n, traj, A.seed, chain, tab, fa);
                }
            }
            double w[5];
            action_totals(fa, w, red);
            if (flip_decision(A, st, prm, chain, traj, w, invN, bcast)) {
                const int f = (start != prop) ? 3 - start - prop : (start + 1) % 3;
#pragma unroll
                for (int k = 0; k < QPT; ++k)
#pragma unroll
                    for (int e = 0; e < 4; ++e) x[k].v[e] = -x[k].v[e];
                res_store<V4, QPT, FULL>(sel3(A, f) + cbase, N, x);
                start = f;
                Sstart = neg;
                if (threadIdx.x == 0) st->start = f;
            }
        }
        measure(A, st, traj);
    }
}

// QPT > 0: the resident variant with QPT quads per thread (trajectories
// only); QPT = 0: streaming.  FULL (resident, N a multiple of 4 and every
// thread's QPT quads inside the chain): the bounds and quad-length checks
// fold away; the arithmetic and its order are those of the general instance.
template <bool V4, int QPT, bool FULL = false>
__global__ void __launch_bounds__(INF_MAX_THREADS, 2) infinite_kernel(FusedArgs A, Schedule S) {
    __shared__ float4 tab_s[LOG1PEXP_NODES];
    __shared__ float red_f[16];
    __shared__ f2 red_d[64];
    __shared__ int bcast[2];
    extern __shared__ float4 us[];   // resident variant: u and aux, QPT * blockDim.x quads each
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
    Red red{red_f, red_d, 0};

    if (A.mode == MODE_EVAL) {
        Acc acc = acc_zero();
        const int start = st->start;
        inf_action<V4>(A, kc, chain, start, 1.0f, TRAJ_INIT, 0, red, tab_s, acc);
        double v[5];
        action_totals(acc, v, red);
        if (threadIdx.x == 0) {
            st->S = v[0];
            set_obs(st, prm, v[1], v[2], v[3], v[4], invN);
            st->prop = start;
        }
        return;
    }
    if constexpr (QPT > 0) {
        res_trajectories<V4, QPT, FULL>(A, S, prm, kc, st, chain, invN, us, red, bcast, tab_s);
        return;
    }

    int start = st->start;
    // sum of the current configuration, carried from trajectory to trajectory
    CSum Sstart = chain_sum<V4>(sel3(A, start) + (int64_t)chain * N, N, red);
    for (int k = 0; k < A.n_traj; ++k) {
        const uint32_t traj = A.traj0 + (uint32_t)k;
        Acc acc = acc_zero();
        CSum cs = Sstart;
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
            if (first && last) inf_pass<V4, true, true>(A, pc, kc, chain, cs, red, tab_s, acc);
            else if (first) inf_pass<V4, true, false>(A, pc, kc, chain, cs, red, tab_s, acc);
            else if (last) inf_pass<V4, false, true>(A, pc, kc, chain, cs, red, tab_s, acc);
            else inf_pass<V4, false, false>(A, pc, kc, chain, cs, red, tab_s, acc);
        }
        const int prop = buf_loc(start, S.n_pass - 1);
        double v[7];
        acc_totals(acc, v, red);
        const int cur = metropolis(A, st, prm, chain, traj, start, prop, v, invN, bcast);
        if (cur != start) Sstart = cs;   // accepted: the proposal's sum
        start = cur;
        // ---- optional global sign flip psi -> -psi (Sec. 3, ergodicity) ----
        if (A.flip_every > 0 && ((traj + 1) % (uint32_t)A.flip_every) == 0) {
            Acc fa = acc_zero();
            inf_action<V4>(A, kc, chain, start, -1.0f, traj, A.seed, red, tab_s, fa);
            double w[5];
            action_totals(fa, w, red);
            if (flip_decision(A, st, prm, chain, traj, w, invN, bcast)) {
                // -psi goes to the buffer that is neither current nor the
                // proposal, so the MD end point stays readable; every thread
                // writes its own quads, as in the resident variant
                const int f = (start != prop) ? 3 - start - prop : (start + 1) % 3;
                const float *gs = sel3(A, start) + (int64_t)chain * N;
                float *gf = sel3(A, f) + (int64_t)chain * N;
                for (int64_t q = threadIdx.x; q < ((N + 3) >> 2); q += blockDim.x) {
                    Quad v4 = ldq<V4>(gs, 4 * q, N);
#pragma unroll
                    for (int e = 0; e < 4; ++e) v4.v[e] = -v4.v[e];
                    stq<V4>(gf, 4 * q, N, v4);
                }
                start = f;
                Sstart = csum_neg(Sstart);   // negation is exact in every partial sum
                if (threadIdx.x == 0) st->start = f;
            }
            __syncthreads();
        }
        measure(A, st, traj);
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

// Quads per thread of the resident variant, or 0 (streaming) when a chain
// needs more than 8 per thread.
static int infinite_qpt(int64_t N) {
    const int64_t nq = (N + 3) / 4;
    const int64_t t = infinite_threads(N);
    for (int q : {1, 2, 4, 8})
        if (nq <= (int64_t)q * t) return q;
    return 0;
}

template <bool V4, bool FULL = false>
static void *infinite_func(int qpt) {
    switch (qpt) {
        case 1: return reinterpret_cast<void *>(infinite_kernel<V4, 1, FULL>);
        case 2: return reinterpret_cast<void *>(infinite_kernel<V4, 2, FULL>);
        case 4: return reinterpret_cast<void *>(infinite_kernel<V4, 4, FULL>);
        case 8: return reinterpret_cast<void *>(infinite_kernel<V4, 8, FULL>);
        default: return reinterpret_cast<void *>(infinite_kernel<V4, 0>);
    }
}

cudaError_t infinite_node(const FusedArgs &a, cudaKernelNodeParams *np, void **args) {
    const int qpt = infinite_qpt(a.g.N);
    const int64_t nq = (a.g.N + 3) / 4;
    const bool full = a.g.N % 4 == 0 && qpt > 0 && qpt <= 4 && nq == (int64_t)qpt * infinite_threads(a.g.N);
    np->func = full ? infinite_func<true, true>(qpt)
                    : (a.g.N % 4 == 0) ? infinite_func<true>(qpt) : infinite_func<false>(qpt);
    static bool configured = false;   // room for the largest u and aux arrays above the static 20.5 KB
    if (!configured) {
        for (int q : {1, 2, 4, 8})
            for (void *f : {infinite_func<true>(q), infinite_func<false>(q), infinite_func<true, true>(q)}) {
                const cudaError_t e = cudaFuncSetAttribute(
                    f, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * 8 * INF_MAX_THREADS * 16);
                if (e != cudaSuccess) return e;
            }
        configured = true;
    }
    np->gridDim = dim3((unsigned)(a.n_chains - a.chain0), 1, 1);
    np->blockDim = dim3((unsigned)infinite_threads(a.g.N), 1, 1);
    // u and aux of the resident variant: at most 2 x 8 quads x 256 threads x 16 B = 64 KB
    np->sharedMemBytes = (unsigned)(2 * qpt * infinite_threads(a.g.N) * sizeof(float4));
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
