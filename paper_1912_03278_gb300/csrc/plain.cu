// plain.cu -- the plain FP64 form of the HS-field HMC: FP64 state and force,
// one chain per launch, one unfused kernel per elementary operation
// (a = A psi; u = tanh(a + h') - psi; F = A u; p += k eps F; psi += d eps p).
// It is the reference point of the throughput comparison and the
// straightforward GPU statement of Sec. 3's algorithm.
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "internal.h"

namespace ihmc {
namespace {

constexpr int TPB = 256;
constexpr int NSLOT = 7;  // K0, K1, S, sum t, sum a t, sum h' t, sum s

__device__ __forceinline__ int64_t lattice_nbr_sum_index(const Geometry &g, int64_t i, int which) {
    // neighbours in the order (+x, -x, +y, -y, +z, -z)
    const int64_t x = i % g.X;
    const int64_t y = (i / g.X) % g.Y;
    const int64_t z = i / ((int64_t)g.X * g.Y);
    int64_t xx = x, yy = y, zz = z;
    switch (which) {
        case 0: xx = (x + 1) % g.X; break;
        case 1: xx = (x + g.X - 1) % g.X; break;
        case 2: yy = (y + 1) % g.Y; break;
        case 3: yy = (y + g.Y - 1) % g.Y; break;
        case 4: zz = (z + 1) % g.Z; break;
        default: zz = (z + g.Z - 1) % g.Z; break;
    }
    return xx + (int64_t)g.X * (yy + (int64_t)g.Y * zz);
}

// y = A x on a periodic lattice, A = beta J K + C 1.
__global__ void k_apply_A_lattice(const double *__restrict__ x, double *__restrict__ y, Geometry g,
                                  const ChainParams *prm) {
    const double bJ = prm->bJ, C = prm->C;
    const int nn = 2 * g.dim;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.N;
         i += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int k = 0; k < nn; ++k) s += x[lattice_nbr_sum_index(g, i, k)];
        y[i] = bJ * s + C * x[i];
    }
}

// y = A x with dense couplings, A = beta Jmat + C 1; one warp per row.
__global__ void k_apply_A_dense(const double *__restrict__ J, const double *__restrict__ x,
                                double *__restrict__ y, int64_t N, const ChainParams *prm) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = warp; r < N; r += nwarps) {
        const double *row = J + r * N;
        double s = 0.0;
        for (int64_t j = lane; j < N; j += 32) s += row[j] * x[j];
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (lane == 0) y[r] = prm->beta * s + prm->C * x[r];
    }
}

__device__ __forceinline__ double hprime(const double *h64, const ChainParams *prm, int64_t i) {
    return h64 ? prm->beta * h64[i] : prm->hp;
}

// u = tanh(a + h') - psi
__global__ void k_u(const double *__restrict__ a, const double *__restrict__ psi,
                    double *__restrict__ u, const double *h64, int64_t N, const ChainParams *prm) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x)
        u[i] = tanh(a[i] + hprime(h64, prm, i)) - psi[i];
}

// y += coef * eps * x
__global__ void k_axpy(double *__restrict__ y, const double *__restrict__ x, double coef, int64_t N,
                       const ChainParams *prm) {
    const double al = coef * prm->eps;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x)
        y[i] += al * x[i];
}

__global__ void k_copy(double *__restrict__ dst, const double *__restrict__ src, int64_t N) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

// FP64 momenta: pair q -> sites 2q, 2q+1.
__global__ void k_momenta(double *__restrict__ p, int64_t N, uint64_t seed, uint32_t traj,
                          uint32_t chain) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; 2 * q < N;
         q += (int64_t)gridDim.x * blockDim.x) {
        double z0, z1;
        momenta2_f64((uint32_t)q, traj, chain, seed, z0, z1);
        p[2 * q] = z0;
        if (2 * q + 1 < N) p[2 * q + 1] = z1;
    }
}

// Per-block partial sums of 1/2 p^2 into slot `slot`.
__global__ void k_kinetic_partials(const double *__restrict__ p, int64_t N, double *partials,
                                   int slot) {
    __shared__ double red[32];
    double v[1] = {0.0};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x)
        v[0] += 0.5 * p[i] * p[i];
    block_sum<1>(v, red);
    if (threadIdx.x == 0) partials[(int64_t)slot * gridDim.x + blockIdx.x] = v[0];
}

// Per-block partial sums of the action and estimators of sign*psi (a = A psi given).
__global__ void k_action_partials(const double *__restrict__ psi, const double *__restrict__ a,
                                  const double *h64, int64_t N, const ChainParams *prm,
                                  double sign, uint64_t seed, uint32_t spin_traj, uint32_t chain,
                                  double *partials) {
    __shared__ double red[32 * 5];
    double v[5] = {0, 0, 0, 0, 0};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double ai = sign * a[i];
        const double hp = hprime(h64, prm, i);
        const double x = ai + hp;
        v[0] += 0.5 * (sign * psi[i]) * ai - log2cosh_f64(x);
        const double t = tanh(x);
        v[1] += t;
        v[2] += ai * t;
        v[3] += hp * t;
        const u32x4 r = philox((uint32_t)(i >> 1), spin_traj, chain, PURPOSE_SPIN, seed);
        const double uu = (i & 1) ? u52(r.z, r.w) : u52(r.x, r.y);
        v[4] += (uu < (1.0 + t) * 0.5) ? 1.0 : -1.0;
    }
    block_sum<5>(v, red);
    if (threadIdx.x == 0) {
        for (int k = 0; k < 5; ++k) partials[(int64_t)(2 + k) * gridDim.x + blockIdx.x] = v[k];
    }
}

__device__ void sum_partials(const double *partials, int nb, double (&v)[NSLOT]) {
    for (int k = 0; k < NSLOT; ++k) {
        double s = 0.0;
        for (int b = 0; b < nb; ++b) s += partials[(int64_t)k * nb + b];
        v[k] = s;
    }
}

__device__ void set_obs(ChainState *st, const ChainParams *prm, const double (&v)[NSLOT],
                        double invN) {
    const double m = v[3] * invN;
    st->obs[0] = m;
    st->obs[1] = 0.5 * prm->C - 0.5 * v[4] * invN - v[5] * invN;
    st->obs[2] = fabs(v[6]) * invN;
    st->obs[3] = fabs(m);
}

__device__ void accumulate(ChainState *st) {
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

// Energy splitting, Metropolis test (Sec. 3) and, without a pending flip, the
// measurement.  flag[0] = accepted.
__global__ void k_finalize_traj(const double *partials, int nb, ChainState *st,
                                const ChainParams *prm, int64_t N, uint64_t seed, uint32_t traj,
                                uint32_t chain, int measure, int flip_pending, int *flag) {
    double v[NSLOT];
    sum_partials(partials, nb, v);
    const double S0 = st->S;
    const double dH = (v[1] + v[2]) - (v[0] + S0);
    const double logu = accept_logu(traj, chain, seed, PURPOSE_ACC);
    const bool acc = logu < -dH;
    st->rec[ISING_REC_DH] = dH;
    st->rec[ISING_REC_LOGU] = logu;
    st->rec[ISING_REC_ACCEPTED] = acc ? 1.0 : 0.0;
    st->rec[ISING_REC_K0] = v[0];
    st->rec[ISING_REC_S0] = S0;
    st->rec[ISING_REC_K1] = v[1];
    st->rec[ISING_REC_S1] = v[2];
    st->rec[ISING_REC_FLIPPED] = 0.0;
    if (acc) {
        st->S = v[2];
        set_obs(st, prm, v, 1.0 / (double)N);
    }
    flag[0] = acc ? 1 : 0;
    if (measure && !flip_pending) accumulate(st);
}

__global__ void k_finalize_flip(const double *partials, int nb, ChainState *st,
                                const ChainParams *prm, int64_t N, uint64_t seed, uint32_t traj,
                                uint32_t chain, int measure, int *flag) {
    double v[NSLOT];
    sum_partials(partials, nb, v);
    const double lu = accept_logu(traj, chain, seed, PURPOSE_FLIP);
    const bool fl = lu < -(v[2] - st->S);
    if (fl) {
        st->S = v[2];
        set_obs(st, prm, v, 1.0 / (double)N);
        st->rec[ISING_REC_FLIPPED] = 1.0;
    }
    flag[1] = fl ? 1 : 0;
    if (measure) accumulate(st);
}

__global__ void k_finalize_eval(const double *partials, int nb, ChainState *st,
                                const ChainParams *prm, int64_t N) {
    double v[NSLOT];
    sum_partials(partials, nb, v);
    st->S = v[2];
    set_obs(st, prm, v, 1.0 / (double)N);
}

__global__ void k_select(double *cur, const double *prop, int64_t N,
                         const int *flag, int which, double scale) {
    if (!flag[which]) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x)
        cur[i] = scale * prop[i];
}

int grid_for(int64_t N) {
    int64_t b = (N + TPB - 1) / TPB;
    if (b > 1184) b = 1184;
    if (b < 1) b = 1;
    return (int)b;
}

cudaError_t apply_A(const PlainArgs &a, const double *x, double *y, cudaStream_t s) {
    if (a.kind == ISING_KIND_DENSE) {
        int64_t warps = a.g.N;
        int64_t blocks = (warps * 32 + TPB - 1) / TPB;
        if (blocks > 1184) blocks = 1184;
        k_apply_A_dense<<<(int)blocks, TPB, 0, s>>>(a.J, x, y, a.g.N, a.params);
    } else {
        k_apply_A_lattice<<<grid_for(a.g.N), TPB, 0, s>>>(x, y, a.g, a.params);
    }
    return cudaGetLastError();
}

}  // namespace

int plain_partial_blocks(int64_t N) { return grid_for(N); }

#define CK(x)                                  \
    do {                                       \
        cudaError_t e_ = (x);                  \
        if (e_ != cudaSuccess) return e_;      \
    } while (0)

// One trajectory of one chain (Sec. 3 algorithm).
cudaError_t plain_trajectory(const PlainArgs &a, const Schedule &sched, uint64_t seed,
                             uint32_t traj, int measure, int flip, cudaStream_t s,
                             int64_t *launches) {
    const int64_t N = a.g.N;
    const int gb = grid_for(N);
    int64_t n = 0;
    k_copy<<<gb, TPB, 0, s>>>(a.psi, a.psi_cur, N); ++n;
    k_momenta<<<grid_for((N + 1) / 2), TPB, 0, s>>>(a.p, N, seed, traj, a.chain); ++n;
    k_kinetic_partials<<<gb, TPB, 0, s>>>(a.p, N, a.partials, 0); ++n;
    for (int j = 0; j < sched.n_pass; ++j) {
        CK(apply_A(a, a.psi, a.a, s)); ++n;
        k_u<<<gb, TPB, 0, s>>>(a.a, a.psi, a.u, a.h64, N, a.params); ++n;
        CK(apply_A(a, a.u, a.F, s)); ++n;
        k_axpy<<<gb, TPB, 0, s>>>(a.p, a.F, (double)sched.kick[j], N, a.params); ++n;
        if (j + 1 < sched.n_pass) {
            k_axpy<<<gb, TPB, 0, s>>>(a.psi, a.p, (double)sched.drift[j], N, a.params); ++n;
        }
    }
    k_kinetic_partials<<<gb, TPB, 0, s>>>(a.p, N, a.partials, 1); ++n;
    CK(apply_A(a, a.psi, a.a, s)); ++n;
    k_action_partials<<<gb, TPB, 0, s>>>(a.psi, a.a, a.h64, N, a.params, 1.0, seed, traj, a.chain,
                                         a.partials); ++n;
    k_finalize_traj<<<1, 1, 0, s>>>(a.partials, gb, a.state, a.params, N, seed, traj, a.chain,
                                    measure, flip, a.flag); ++n;
    k_select<<<gb, TPB, 0, s>>>(a.psi_cur, a.psi, N, a.flag, 0, 1.0); ++n;
    if (flip) {
        CK(apply_A(a, a.psi_cur, a.a, s)); ++n;
        k_action_partials<<<gb, TPB, 0, s>>>(a.psi_cur, a.a, a.h64, N, a.params, -1.0, seed, traj,
                                             a.chain, a.partials); ++n;
        k_finalize_flip<<<1, 1, 0, s>>>(a.partials, gb, a.state, a.params, N, seed, traj, a.chain,
                                        measure, a.flag); ++n;
        k_select<<<gb, TPB, 0, s>>>(a.psi_cur, a.psi_cur, N, a.flag, 1, -1.0); ++n;
    }
    *launches += n;
    return cudaGetLastError();
}

cudaError_t plain_eval(const PlainArgs &a, cudaStream_t s, int64_t *launches) {
    const int64_t N = a.g.N;
    const int gb = grid_for(N);
    CK(apply_A(a, a.psi_cur, a.a, s));
    k_action_partials<<<gb, TPB, 0, s>>>(a.psi_cur, a.a, a.h64, N, a.params, 1.0, 0, TRAJ_INIT,
                                         a.chain, a.partials);
    k_finalize_eval<<<1, 1, 0, s>>>(a.partials, gb, a.state, a.params, N);
    *launches += 3;
    return cudaGetLastError();
}

cudaError_t plain_momenta(const PlainArgs &a, uint64_t seed, uint32_t traj, cudaStream_t s,
                          int64_t *launches) {
    k_momenta<<<grid_for((a.g.N + 1) / 2), TPB, 0, s>>>(a.p, a.g.N, seed, traj, a.chain);
    *launches += 1;
    return cudaGetLastError();
}

}  // namespace ihmc
