// fused_lattice.cu -- FP32 HMC trajectories on periodic 1D/2D/3D lattices,
// one CTA per chain, whole trajectories per launch.
//
// Per force evaluation (Sec. 3, equations of motion, in the form
// F = A (tanh(A psi + h') - psi) with A = beta*J*K + C*1):
//   a = A psi,  u = tanh(a + h') - psi,  F = A u,   p += kick*eps*F,
//   psi' = psi + drift*eps*p            (the symplectic integrator's schedule)
// The CTA streams its chain plane by plane (plane = row in 2D, xy-slab in 3D)
// through shared-memory rings: psi planes arrive by cp.async D planes ahead,
// u(z+1) is computed from psi(z..z+2), then F(z) from u(z-1..z+1).  Every
// site's psi and p cross HBM once per force evaluation: 16 B per site-step.
// The last pass of a trajectory also evaluates the FP64 action
//   S = sum_i 1/2 psi_i a_i - log 2cosh(a_i + h'_i)   (a in FP64)
// and the Sec. 4 estimators; the CTA then takes the Metropolis decision
// (Sec. 3) itself, so a launch can run many trajectories back to back.
#include <cuda_runtime.h>

#include "df32.cuh"
#include "device_common.cuh"
#include "internal.h"

namespace ihmc {
namespace {

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <int VEC>
struct Vec {
    float v[VEC];
};

template <int VEC>
__device__ __forceinline__ Vec<VEC> ldv(const float *p) {
    Vec<VEC> r;
    if constexpr (VEC == 4) {
        const float4 t = *reinterpret_cast<const float4 *>(p);
        r.v[0] = t.x; r.v[1] = t.y; r.v[2] = t.z; r.v[3] = t.w;
    } else {
#pragma unroll
        for (int k = 0; k < VEC; ++k) r.v[k] = p[k];
    }
    return r;
}
template <int VEC>
__device__ __forceinline__ void stv(float *p, const Vec<VEC> &r) {
    if constexpr (VEC == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(r.v[0], r.v[1], r.v[2], r.v[3]);
    } else {
#pragma unroll
        for (int k = 0; k < VEC; ++k) p[k] = r.v[k];
    }
}

// Sum of the nearest neighbours of the VEC sites starting at plane offset e0,
// using the current plane pc (in-plane neighbours) and the planes before and
// after (pm, pq; out-of-plane neighbours, dim >= 2).  Also returns the centre.
template <int VEC>
__device__ __forceinline__ void neighbour_sum(const Geometry &g, const float *pm, const float *pc,
                                              const float *pq, int e0, Vec<VEC> &c,
                                              Vec<VEC> &nb) {
    const int x0 = e0 % g.X;
    const int rowbase = e0 - x0;
    c = ldv<VEC>(pc + e0);
    const float left = pc[rowbase + (x0 == 0 ? g.X - 1 : x0 - 1)];
    const float right = pc[rowbase + (x0 + VEC == g.X ? 0 : x0 + VEC)];
#pragma unroll
    for (int k = 0; k < VEC; ++k) {
        const float l = (k == 0) ? left : c.v[k - 1];
        const float r = (k == VEC - 1) ? right : c.v[k + 1];
        nb.v[k] = l + r;
    }
    if (g.dim == 3) {
        const int y = rowbase / g.X;
        const int ym = (y == 0 ? g.Y - 1 : y - 1) * g.X + x0;
        const int yp = (y == g.Y - 1 ? 0 : y + 1) * g.X + x0;
        const Vec<VEC> a = ldv<VEC>(pc + ym), b = ldv<VEC>(pc + yp);
#pragma unroll
        for (int k = 0; k < VEC; ++k) nb.v[k] += a.v[k] + b.v[k];
    }
    if (g.dim >= 2) {
        const Vec<VEC> a = ldv<VEC>(pm + e0), b = ldv<VEC>(pq + e0);
#pragma unroll
        for (int k = 0; k < VEC; ++k) nb.v[k] += a.v[k] + b.v[k];
    }
}

// The same neighbour sum exactly, as a double-float (TwoSum chain), for the
// FP64-accurate action.
template <int VEC>
__device__ __forceinline__ void neighbour_sum_df(const Geometry &g, const float *pm,
                                                 const float *pc, const float *pq, int e0,
                                                 f2 (&nb)[VEC]) {
    const int x0 = e0 % g.X;
    const int rowbase = e0 - x0;
#pragma unroll
    for (int k = 0; k < VEC; ++k) {
        const int x = x0 + k;
        const int l = rowbase + (x == 0 ? g.X - 1 : x - 1);
        const int r = rowbase + (x == g.X - 1 ? 0 : x + 1);
        f2 s = two_sum(pc[l], pc[r]);
        if (g.dim == 3) {
            const int y = rowbase / g.X;
            s = df_add_f(s, pc[(y == 0 ? g.Y - 1 : y - 1) * g.X + x]);
            s = df_add_f(s, pc[(y == g.Y - 1 ? 0 : y + 1) * g.X + x]);
        }
        if (g.dim >= 2) {
            s = df_add_f(s, pm[e0 + k]);
            s = df_add_f(s, pq[e0 + k]);
        }
        nb[k] = s;
    }
}

// Per-thread accumulators of one trajectory, double-float (converted to FP64
// once, for the block reduction).
struct Acc {
    f2 K0, K1, S, sT, sAT, sHT;
    int sS;
};

__device__ __forceinline__ Acc acc_zero() {
    const f2 z{0.0f, 0.0f};
    return Acc{z, z, z, z, z, z, 0};
}

struct PassCfg {
    int src, dst;
    float kick, drift;   // already multiplied by eps
    bool first, last;    // first pass draws momenta; last pass has no drift
    bool force;          // compute F and update p (and psi unless last)
    bool action;         // accumulate action/observables of the src planes
    float sign;          // +1, or -1 to evaluate at -psi (sign-flip proposal)
    uint32_t spin_traj;  // trajectory index of the spin draw
};

__device__ __forceinline__ float *sel3(const FusedArgs &A, int i) {
    return i == 0 ? A.psi[0] : (i == 1 ? A.psi[1] : A.psi[2]);
}

template <int VEC, int D>
__device__ void run_pass(const FusedArgs &A, const PassCfg &pc, const ChainParams &prm, int chain,
                         uint32_t traj, float *smem, Acc &acc) {
    constexpr int R = D + 4;   // psi ring slots
    constexpr int RP = D + 2;  // p ring slots
    const Geometry &g = A.g;
    const int P = g.P;
    float *psi_ring = smem;
    float *p_ring = psi_ring + R * P;
    float *u_ring = p_ring + RP * P;
    const int64_t cbase = (int64_t)chain * g.N;
    const float *__restrict__ gsrc = sel3(A, pc.src) + cbase;
    float *__restrict__ gdst = sel3(A, pc.dst) + cbase;
    float *__restrict__ gp = A.p + cbase;
    const int z0 = 0, z1 = g.nplanes;
    const int nvec = P / VEC;
    const int tid = threadIdx.x, nt = blockDim.x;
    const bool load_p = pc.force && !pc.first;

    auto issue = [&](int s) {
        const int zpsi = z0 - 2 + s;
        if (zpsi <= z1 + 1) {
            const int zw = ((zpsi % g.nplanes) + g.nplanes) % g.nplanes;
            const float *src = gsrc + (int64_t)zw * P;
            float *dst = psi_ring + (s % R) * P;
            if constexpr (VEC == 4) {
                for (int v = tid; v < nvec; v += nt) cp_async16(dst + 4 * v, src + 4 * v);
            } else {
                for (int v = tid; v < P; v += nt) cp_async4(dst + v, src + v);
            }
        }
        const int zp = z0 - 4 + s;
        if (load_p && zp >= z0 && zp < z1) {
            const float *src = gp + (int64_t)zp * P;
            float *dst = p_ring + (s % RP) * P;
            if constexpr (VEC == 4) {
                for (int v = tid; v < nvec; v += nt) cp_async16(dst + 4 * v, src + 4 * v);
            } else {
                for (int v = tid; v < P; v += nt) cp_async4(dst + v, src + v);
            }
        }
        cp_commit();
    };
    auto psi_slot = [&](int z) -> const float * { return psi_ring + ((z - z0 + 2) % R) * P; };
    auto u_slot = [&](int z) -> float * { return u_ring + ((z - z0 + 3) % 3) * P; };

    for (int s = 0; s <= D + 2; ++s) issue(s);
    int s_next = D + 3;

    const float Cf = prm.Cf, bJf = prm.bJf;
    const f2 C2 = df_from_double(prm.C), bJ2 = df_from_double(prm.bJ);
    const f2 hp2 = df_from_double(prm.hp), beta2 = df_from_double(prm.beta);

    for (int it = z0 - 1; it <= z1; ++it) {
        cp_wait<D>();
        __syncthreads();
        issue(s_next++);
        // ---- u(it) = tanh(A psi + h') - psi on plane it ----
        {
            const float *pm = psi_slot(it - 1), *pcen = psi_slot(it), *pq = psi_slot(it + 1);
            float *uo = u_slot(it);
            const bool act = pc.action && it >= z0 && it < z1;
            const int zw = ((it % g.nplanes) + g.nplanes) % g.nplanes;
            for (int v = tid; v < nvec; v += nt) {
                const int e0 = v * VEC;
                Vec<VEC> c, nb;
                neighbour_sum<VEC>(g, pm, pcen, pq, e0, c, nb);
                Vec<VEC> u;
                float hpv[VEC];
#pragma unroll
                for (int k = 0; k < VEC; ++k)
                    hpv[k] = A.h32 ? prm.betaf * A.h32[(int64_t)zw * P + e0 + k] : prm.hpf;
                if (pc.force) {
#pragma unroll
                    for (int k = 0; k < VEC; ++k) {
                        const float a = fmaf(Cf, c.v[k], bJf * nb.v[k]);
                        u.v[k] = tanhf(a + hpv[k]) - c.v[k];
                    }
                    stv<VEC>(uo + e0, u);
                }
                if (act) {
                    // FP64-accurate action in double-float:
                    //   S_i = 1/2 psi_i a_i - |x_i| - log(1 + exp(-2|x_i|)),  x = a + h'
                    f2 nbd[VEC];
                    neighbour_sum_df<VEC>(g, pm, pcen, pq, e0, nbd);
                    const int64_t site0 = (int64_t)zw * P + e0;
                    float su[4];
                    if constexpr (VEC == 4) {
                        const float4 w = spin_u4_f32((uint32_t)(site0 >> 2), pc.spin_traj,
                                                     (uint32_t)chain, A.seed);
                        su[0] = w.x; su[1] = w.y; su[2] = w.z; su[3] = w.w;
                    }
#pragma unroll
                    for (int k = 0; k < VEC; ++k) {
                        const float ps = pc.sign * c.v[k];
                        const f2 hp = A.h64 ? df_mul(beta2, df_from_double(A.h64[site0 + k])) : hp2;
                        const f2 a = df_add(df_mul_f(C2, ps), df_mul(bJ2, f2{pc.sign * nbd[k].hi,
                                                                               pc.sign * nbd[k].lo}));
                        const f2 x = df_add(a, hp);
                        const f2 ax = x.hi < 0.0f ? df_neg(x) : x;
                        const f2 gl = log1pexp_neg(f2{2.0f * ax.hi, 2.0f * ax.lo}, A.lpe_tab);
                        f2 term = df_mul_f(a, 0.5f * ps);
                        term = df_add(term, df_neg(df_add(ax, gl)));
                        acc.S = df_add(acc.S, term);
                        const float t = tanhf(x.hi);
                        acc.sT = df_add_f(acc.sT, t);
                        acc.sAT = df_add_f(acc.sAT, a.hi * t);
                        acc.sHT = df_add_f(acc.sHT, hp.hi * t);
                        float uu;
                        if constexpr (VEC == 4) {
                            uu = su[k];
                        } else {
                            const float4 w = spin_u4_f32((uint32_t)((site0 + k) >> 2),
                                                         pc.spin_traj, (uint32_t)chain, A.seed);
                            const int q = (int)((site0 + k) & 3);
                            uu = q == 0 ? w.x : q == 1 ? w.y : q == 2 ? w.z : w.w;
                        }
                        acc.sS += (uu < (1.0f + t) * 0.5f) ? 1 : -1;
                    }
                }
            }
        }
        __syncthreads();
        // ---- F(z) = A u, kick and drift on plane z = it - 1 ----
        const int z = it - 1;
        if (pc.force && z >= z0 && z < z1) {
            const float *um = u_slot(z - 1), *uc = u_slot(z), *uq = u_slot(z + 1);
            const float *psz = psi_slot(z);
            const float *ppz = p_ring + ((z - z0 + 4) % RP) * P;
            for (int v = tid; v < nvec; v += nt) {
                const int e0 = v * VEC;
                Vec<VEC> uu, nb;
                neighbour_sum<VEC>(g, um, uc, uq, e0, uu, nb);
                const int64_t site0 = (int64_t)z * P + e0;
                Vec<VEC> pv;
                if (pc.first) {
                    if constexpr (VEC == 4) {
                        const float4 w = momenta4_f32((uint32_t)(site0 >> 2), traj,
                                                      (uint32_t)chain, A.seed);
                        pv.v[0] = w.x; pv.v[1] = w.y; pv.v[2] = w.z; pv.v[3] = w.w;
                    } else {
#pragma unroll
                        for (int k = 0; k < VEC; ++k) {
                            const float4 w = momenta4_f32((uint32_t)((site0 + k) >> 2), traj,
                                                          (uint32_t)chain, A.seed);
                            const int q = (int)((site0 + k) & 3);
                            pv.v[k] = q == 0 ? w.x : q == 1 ? w.y : q == 2 ? w.z : w.w;
                        }
                    }
#pragma unroll
                    for (int k = 0; k < VEC; ++k) acc.K0 = df_add(acc.K0, two_prod(pv.v[k], 0.5f * pv.v[k]));
                } else {
                    pv = ldv<VEC>(ppz + e0);
                }
#pragma unroll
                for (int k = 0; k < VEC; ++k) {
                    const float F = fmaf(Cf, uu.v[k], bJf * nb.v[k]);
                    pv.v[k] = fmaf(pc.kick, F, pv.v[k]);
                }
                stv<VEC>(gp + site0, pv);
                if (pc.last) {
#pragma unroll
                    for (int k = 0; k < VEC; ++k) acc.K1 = df_add(acc.K1, two_prod(pv.v[k], 0.5f * pv.v[k]));
                } else {
                    const Vec<VEC> ps = ldv<VEC>(psz + e0);
                    Vec<VEC> pn;
#pragma unroll
                    for (int k = 0; k < VEC; ++k) pn.v[k] = fmaf(pc.drift, pv.v[k], ps.v[k]);
                    stv<VEC>(gdst + site0, pn);
                }
            }
        }
    }
    cp_wait<0>();
    __syncthreads();
}

__device__ __forceinline__ int buf_loc(int start, int j) {
    if (j == 0) return start;
    return (start + ((j & 1) ? 1 : 2)) % 3;
}

template <int VEC, int D>
__global__ void __launch_bounds__(256) fused_lattice_kernel(FusedArgs A, Schedule S) {
    extern __shared__ float4 smem_f4[];
    float *smem = reinterpret_cast<float *>(smem_f4);
    constexpr int R = D + 4, RP = D + 2;
    const Geometry &g = A.g;
    const size_t ring_floats = (size_t)(R + RP + 3) * g.P;
    double *red = reinterpret_cast<double *>(smem + ((ring_floats + 3) & ~(size_t)3));
    int *bcast = reinterpret_cast<int *>(red + 32 * 8);

    const int chain = A.chain0 + blockIdx.x;
    if (chain >= A.n_chains) return;
    ChainState *st = A.state + chain;
    const ChainParams prm = A.params[chain];
    const double invN = 1.0 / (double)g.N;

    if (A.mode == MODE_MOMENTA) {
        float *gp = A.p + (int64_t)chain * g.N;
        for (int64_t i = threadIdx.x; i < g.N; i += blockDim.x) {
            const float4 w = momenta4_f32((uint32_t)(i >> 2), A.traj0, (uint32_t)chain, A.seed);
            const int q = (int)(i & 3);
            gp[i] = q == 0 ? w.x : q == 1 ? w.y : q == 2 ? w.z : w.w;
        }
        return;
    }

    if (A.mode == MODE_EVAL) {
        Acc acc = acc_zero();
        const int start = st->start;
        PassCfg pc{start, start, 0.f, 0.f, false, false, false, true, 1.0f, TRAJ_INIT};
        run_pass<VEC, D>(A, pc, prm, chain, TRAJ_INIT, smem, acc);
        double v[5] = {df_to_double(acc.S), df_to_double(acc.sT), df_to_double(acc.sAT),
                       df_to_double(acc.sHT), (double)acc.sS};
        block_sum<5>(v, red);
        if (threadIdx.x == 0) {
            st->S = v[0];
            const double m = v[1] * invN;
            st->obs[0] = m;
            st->obs[1] = 0.5 * prm.C - 0.5 * v[2] * invN - v[3] * invN;
            st->obs[2] = fabs(v[4]) * invN;
            st->obs[3] = fabs(m);
            st->prop = start;
        }
        return;
    }

    int start = st->start;
    for (int k = 0; k < A.n_traj; ++k) {
        const uint32_t traj = A.traj0 + (uint32_t)k;
        Acc acc = acc_zero();
        for (int j = 0; j < S.n_pass; ++j) {
            PassCfg pc;
            pc.src = buf_loc(start, j);
            pc.dst = buf_loc(start, j + 1);
            pc.kick = (float)(S.kick[j] * prm.eps);
            pc.drift = (float)(S.drift[j] * prm.eps);
            pc.first = (j == 0);
            pc.last = (j == S.n_pass - 1);
            pc.force = true;
            pc.action = pc.last;
            pc.sign = 1.0f;
            pc.spin_traj = traj;
            run_pass<VEC, D>(A, pc, prm, chain, traj, smem, acc);
        }
        double v[7] = {df_to_double(acc.K0), df_to_double(acc.K1), df_to_double(acc.S),
                       df_to_double(acc.sT), df_to_double(acc.sAT), df_to_double(acc.sHT),
                       (double)acc.sS};
        block_sum<7>(v, red);
        const int prop = buf_loc(start, S.n_pass - 1);
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
                const double m = v[3] * invN;
                st->obs[0] = m;
                st->obs[1] = 0.5 * prm.C - 0.5 * v[4] * invN - v[5] * invN;
                st->obs[2] = fabs(v[6]) * invN;
                st->obs[3] = fabs(m);
            }
            bcast[0] = accd ? prop : start;
        }
        __syncthreads();
        start = bcast[0];
        __syncthreads();
        // ---- optional global sign flip psi -> -psi (Sec. 3, ergodicity) ----
        if (A.flip_every > 0 && ((traj + 1) % (uint32_t)A.flip_every) == 0) {
            Acc fa = acc_zero();
            PassCfg pc{start, start, 0.f, 0.f, false, false, false, true, -1.0f, traj};
            run_pass<VEC, D>(A, pc, prm, chain, traj, smem, fa);
            double w[5] = {df_to_double(fa.S), df_to_double(fa.sT), df_to_double(fa.sAT),
                           df_to_double(fa.sHT), (double)fa.sS};
            block_sum<5>(w, red);
            if (threadIdx.x == 0) {
                const double lu = accept_logu(traj, (uint32_t)chain, A.seed, PURPOSE_FLIP);
                const bool fl = lu < -(w[0] - st->S);
                if (fl) {
                    st->S = w[0];
                    const double m = w[1] * invN;
                    st->obs[0] = m;
                    st->obs[1] = 0.5 * prm.C - 0.5 * w[2] * invN - w[3] * invN;
                    st->obs[2] = fabs(w[4]) * invN;
                    st->obs[3] = fabs(m);
                    st->rec[ISING_REC_FLIPPED] = 1.0;
                }
                bcast[1] = fl ? 1 : 0;
            }
            __syncthreads();
            if (bcast[1]) {
                // -psi goes to the buffer that is neither current nor the proposal,
                // so the MD end point stays readable
                const int f = (start != prop) ? 3 - start - prop : (start + 1) % 3;
                const float *gs = sel3(A, start) + (int64_t)chain * g.N;
                float *gf = sel3(A, f) + (int64_t)chain * g.N;
                for (int64_t i = threadIdx.x; i < g.N; i += blockDim.x) gf[i] = -gs[i];
                start = f;
                if (threadIdx.x == 0) st->start = f;
            }
            __syncthreads();
        }
        // ---- measurement: a repeated configuration repeats its measurement ----
        if (threadIdx.x == 0) {
            if ((int64_t)traj >= (int64_t)A.n_therm) {
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
        }
        __syncthreads();
    }
}

template <int VEC, int D>
cudaError_t launch_vd(const FusedArgs &a, const Schedule &s, int threads, cudaStream_t st) {
    const int smem = fused_lattice_smem_bytes(a.g, D, VEC);
    static bool configured[2] = {false, false};
    auto kern = fused_lattice_kernel<VEC, D>;
    int dev = 0;
    cudaGetDevice(&dev);
    if (!configured[dev & 1]) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             227 * 1024);
        if (e != cudaSuccess) return e;
        configured[dev & 1] = true;
    }
    const int grid = a.n_chains - a.chain0;
    if (grid <= 0) return cudaSuccess;
    kern<<<grid, threads, smem, st>>>(a, s);
    return cudaGetLastError();
}

}  // namespace

int fused_lattice_smem_bytes(const Geometry &g, int depth, int vec) {
    (void)vec;
    const size_t ring = (size_t)(depth + 4 + depth + 2 + 3) * g.P;
    const size_t floats = ((ring + 3) & ~(size_t)3);
    return (int)(floats * 4 + 32 * 8 * 8 + 16);
}

int fused_lattice_pick(const Geometry &g, int *threads, int *depth) {
    const int vec = (g.X % 4 == 0 && g.P % 4 == 0) ? 4 : 1;
    int t = (g.P / vec + 31) / 32 * 32;
    if (t > 256) t = 256;
    if (t < 32) t = 32;
    *threads = t;
    const int limit = 200 * 1024;
    int d = 4;
    while (d > 1 && fused_lattice_smem_bytes(g, d, vec) > limit) d = (d == 4) ? 2 : 1;
    if (fused_lattice_smem_bytes(g, d, vec) > 227 * 1024) return -1;
    *depth = d;
    return vec;
}

cudaError_t launch_fused_lattice(const FusedArgs &a, const Schedule &sched, int threads,
                                 int depth, cudaStream_t s) {
    const int vec = (a.g.X % 4 == 0 && a.g.P % 4 == 0) ? 4 : 1;
    if (vec == 4) {
        if (depth >= 4) return launch_vd<4, 4>(a, sched, threads, s);
        if (depth >= 2) return launch_vd<4, 2>(a, sched, threads, s);
        return launch_vd<4, 1>(a, sched, threads, s);
    }
    if (depth >= 4) return launch_vd<1, 4>(a, sched, threads, s);
    if (depth >= 2) return launch_vd<1, 2>(a, sched, threads, s);
    return launch_vd<1, 1>(a, sched, threads, s);
}

}  // namespace ihmc
