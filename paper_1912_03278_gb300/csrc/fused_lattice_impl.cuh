// fused_lattice_impl.cuh -- FP32 HMC trajectories on periodic 1D/2D/3D lattices,
// one CTA per chain, whole trajectories per launch.
//
// Per force evaluation (Sec. 3, equations of motion, in the form
// F = A (tanh(A psi + h') - psi) with A = beta*J*K + C*1):
//   a = A psi,  u = tanh(a + h') - psi,  F = A u,   p += kick*eps*F,
//   psi' = psi + drift*eps*p            (the symplectic integrator's schedule)
// The CTA streams its chain plane by plane (plane = row in 2D, xy-slab in 3D)
// through shared-memory rings: psi and p planes arrive by cp.async D planes
// ahead, u(z+1) is computed from psi(z..z+2), then F(z) from u(z-1..z+1).
// Every site's psi and p cross HBM once per force evaluation: 16 B per
// site-step.  The last pass of a trajectory also evaluates the action
//   S = sum_i 1/2 psi_i a_i - log 2cosh(a_i + h'_i)
// to FP64 accuracy in double-float arithmetic, the kinetic energies and the
// Sec. 4 estimators; the CTA then takes the Metropolis decision (Sec. 3)
// itself, so one launch can run many trajectories back to back.
//
// Work layout inside a plane: a thread owns up to NVMAX vectors of VEC
// consecutive sites, fixed for the whole launch, so every neighbour offset is
// computed once.
//
// A chain may be split over a thread-block cluster of CS CTAs (launch
// attribute; CS = 1 is a plain launch): CTA r streams the slab of planes
// [r*nz/CS, (r+1)*nz/CS) and reads the two planes beyond each end of its slab
// (the previous pass's psi, in global memory) to form the u values its force
// needs, so the CTAs of a chain only meet at one cluster barrier after every
// force pass.  The per-chain sums of a trajectory are exchanged through
// distributed shared memory and added in rank order by every CTA, so all of
// them take the same Metropolis decision.
#pragma once
#include <cuda_runtime.h>

#include "df32.cuh"
#include "device_common.cuh"
#include "internal.h"
#include "mbarrier.cuh"

namespace ihmc {
namespace {

constexpr int NVMAX = 4;
// Threads per CTA: up to 256 (two CTAs per SM) for a chain on one CTA, up to
// 512 (16 warps for the large planes, which hold one CTA per SM) for a chain
// split over a cluster; both give a cap of 128 registers per thread.
constexpr int MAX_THREADS = 512;
constexpr int MAX_THREADS_UNSPLIT = 256;
constexpr int MAX_CS = 8;                    // CTAs per chain (portable cluster size)
constexpr int XCH_WORDS = 8;                 // per-CTA sums exchanged in a cluster
constexpr int MAX_BARS = 16;                 // copy-group mbarriers (one per psi ring slot)
// block reduction (32 warps x 8 doubles), broadcast words, two exchange
// buffers, the copy-group mbarriers
constexpr int RED_BYTES = 32 * 8 * 8 + 16 + 2 * XCH_WORDS * 8 + MAX_BARS * 8;

// F(z) trails u by LAG planes: with LAG = 1 a plane's force reads only u
// planes finished in earlier iterations, so one barrier per plane suffices.
#ifndef IHMC_FL_LAG
#define IHMC_FL_LAG 1
#endif
constexpr int LAG = IHMC_FL_LAG;

// Shared memory of a launch: the plane rings (psi D+4+LAG, p D+2+LAG, u
// 3+LAG slots), optionally the log(1 + e^-y) table, the reduction words.
__host__ __device__ inline size_t ring_bytes(int P, int D) {
    return (((size_t)(2 * D + 9 + 3 * LAG) * P + 3) & ~(size_t)3) * 4;
}

// Thread-block cluster: size and rank of this CTA, barrier, and an FP64 read
// of another CTA's shared memory.
__device__ __forceinline__ int cluster_size() {
    unsigned n;
    asm("mov.u32 %0, %%cluster_nctarank;" : "=r"(n));
    return (int)n;
}
__device__ __forceinline__ int cluster_rank() {
    unsigned r;
    asm("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return (int)r;
}
// Every thread of every CTA of the cluster; orders this thread's earlier
// global and shared writes before the other CTAs' later reads.
__device__ __forceinline__ void cluster_barrier() {
    __syncwarp();
    asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
                 "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ double ld_cluster_f64(const double *local, int rank) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(local);
    unsigned ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
    double v;
    asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(ra) : "memory");
    return v;
}

// Chain-wide sum of NV per-thread values: the CTA's fixed-order block sum,
// then (cs > 1) the CTAs' block sums added in rank order through the
// exchange buffer xch (NV <= XCH_WORDS doubles in every CTA's shared memory;
// two alternating buffers so a buffer is rewritten only after a later
// cluster barrier).  Every CTA's thread 0 ends with the same totals in v.
template <int NV, bool CL>
__device__ __forceinline__ void chain_sum(double (&v)[NV], double *red, double *xch, int cs) {
    static_assert(NV <= XCH_WORDS, "exchange buffer");
    block_sum<NV>(v, red);
    if (!CL || cs == 1) return;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) xch[k] = v[k];
    }
    cluster_barrier();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double t = 0.0;
            for (int r = 0; r < cs; ++r) t += ld_cluster_f64(xch + k, r);
            v[k] = t;
        }
    }
}

// Periodic plane index of an absolute plane z in [-2, nz + 1] (any nz >= 1):
// at most two additions or subtractions of nz, no division in the loop.
__device__ __forceinline__ int wrap_plane(int z, int nz) {
    z = z < 0 ? z + nz : z;
    z = z < 0 ? z + nz : z;
    z = z >= nz ? z - nz : z;
    z = z >= nz ? z - nz : z;
    return z;
}

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

// One thread's vectors in a plane: plane offset e0 and column x0 of the first
// site; loads of inactive slots use the last vector (in bounds), stores skip.
struct Slots {
    int e0[NVMAX];
    int x0[NVMAX];
    bool valid[NVMAX];
    int nwarp;   // number of k with any active lane in this warp
};

template <int VEC>
__device__ __forceinline__ Slots make_slots(const Geometry &g) {
    Slots s;
    const int nvec = g.P / VEC;
    const int nt = blockDim.x;
    const int wbase = threadIdx.x & ~31;
    s.nwarp = 0;
#pragma unroll
    for (int k = 0; k < NVMAX; ++k) {
        const int v = threadIdx.x + k * nt;
        s.valid[k] = v < nvec;
        const int vc = v < nvec ? v : nvec - 1;
        s.e0[k] = vc * VEC;
        s.x0[k] = (vc * VEC) % g.X;
        if (wbase + k * nt < nvec) s.nwarp = k + 1;
    }
    return s;
}

// Neighbour sum of the VEC sites at (e0, x0) of plane pc, with planes pm/pq
// before/after (dim >= 2).  The centre values are returned in c and the
// individual neighbour values in the arrays (for the exact df sum).
template <int DIM, int VEC>
struct Nbr {
    Vec<VEC> c, nb;
    float lw, rx;           // x-neighbours of the first and last site
    Vec<VEC> ym, yp, zm, zp;
};

// Loads of a gather: from shared memory, or (GL) from global memory through
// L2 only, so that planes another CTA of the cluster rewrote are never served
// from a stale L1 line.
template <int VEC, bool GL>
__device__ __forceinline__ Vec<VEC> ldg_or_s(const float *p) {
    if constexpr (!GL) {
        return ldv<VEC>(p);
    } else {
        Vec<VEC> r;
        if constexpr (VEC == 4) {
            const float4 t = __ldcg(reinterpret_cast<const float4 *>(p));
            r.v[0] = t.x; r.v[1] = t.y; r.v[2] = t.z; r.v[3] = t.w;
        } else {
#pragma unroll
            for (int k = 0; k < VEC; ++k) r.v[k] = __ldcg(p + k);
        }
        return r;
    }
}
template <bool GL>
__device__ __forceinline__ float ld1(const float *p) {
    if constexpr (GL) return __ldcg(p);
    else return *p;
}

template <int DIM, int VEC, bool GL = false>
__device__ __forceinline__ void gather(const Geometry &g, const float *pm, const float *pc,
                                       const float *pq, int e0, int x0, Nbr<DIM, VEC> &n) {
    const int X = g.X;
    n.c = ldg_or_s<VEC, GL>(pc + e0);
    // x-neighbours of the end sites straight from shared memory (measured
    // faster than lane shuffles with the wrap fix-ups)
    const int lidx = (x0 == 0) ? e0 + X - 1 : e0 - 1;
    const int ridx = (x0 + VEC == X) ? e0 + VEC - X : e0 + VEC;
    n.lw = ld1<GL>(pc + lidx);
    n.rx = ld1<GL>(pc + ridx);
#pragma unroll
    for (int k = 0; k < VEC; ++k) {
        const float l = (k == 0) ? n.lw : n.c.v[k - 1];
        const float r = (k == VEC - 1) ? n.rx : n.c.v[k + 1];
        n.nb.v[k] = l + r;
    }
    if constexpr (DIM == 3) {
        const int P = g.P;
        const int ym = (e0 < X) ? e0 + P - X : e0 - X;
        const int yp = (e0 + X >= P) ? e0 + X - P : e0 + X;
        n.ym = ldg_or_s<VEC, GL>(pc + ym);
        n.yp = ldg_or_s<VEC, GL>(pc + yp);
#pragma unroll
        for (int k = 0; k < VEC; ++k) n.nb.v[k] += n.ym.v[k] + n.yp.v[k];
    }
    if constexpr (DIM >= 2) {
        n.zm = ldg_or_s<VEC, GL>(pm + e0);
        n.zp = ldg_or_s<VEC, GL>(pq + e0);
#pragma unroll
        for (int k = 0; k < VEC; ++k) n.nb.v[k] += n.zm.v[k] + n.zp.v[k];
    }
}

// Exact neighbour sum of site k as a double-float (TwoSum chain).
template <int DIM, int VEC>
__device__ __forceinline__ f2 exact_nb(const Nbr<DIM, VEC> &n, int k) {
    const float l = (k == 0) ? n.lw : n.c.v[k - 1];
    const float r = (k == VEC - 1) ? n.rx : n.c.v[k + 1];
    f2 s = two_sum(l, r);
    if constexpr (DIM == 3) {
        s = df_add_f(s, n.ym.v[k]);
        s = df_add_f(s, n.yp.v[k]);
    }
    if constexpr (DIM >= 2) {
        s = df_add_f(s, n.zm.v[k]);
        s = df_add_f(s, n.zp.v[k]);
    }
    return s;
}

// Per-thread accumulators of one trajectory.  Energies: the high words are
// summed as double-floats, the low words of the addends in a separate FP32
// sum (their magnitude is ~2^-24 of the terms).  Estimators: Kahan FP32 sums.
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

struct PassCfg {
    int src, dst;
    float kick, drift;   // already multiplied by eps
    bool first, last;    // first pass draws p and sums K0; last pass has no drift, sums K1
                         // and evaluates the action of its configuration
    uint32_t traj;       // trajectory index (momenta and spin draws)
};

__device__ __forceinline__ float *sel3(const FusedArgs &A, int i) {
    return i == 0 ? A.psi[0] : (i == 1 ? A.psi[1] : A.psi[2]);
}

// Per-chain constants of the action in double-float form.
struct ActConst {
    f2 C2, bJ2, hp2, beta2;
    float Cf, bJf, betaf, hpf;
    bool hzero;
};

__device__ __forceinline__ ActConst act_const(const ChainParams &prm) {
    ActConst k;
    k.C2 = df_from_double(prm.C);
    k.bJ2 = df_from_double(prm.bJ);
    k.hp2 = df_from_double(prm.hp);
    k.beta2 = df_from_double(prm.beta);
    k.Cf = prm.Cf;
    k.bJf = prm.bJf;
    k.betaf = prm.betaf;
    k.hpf = prm.hpf;
    k.hzero = prm.hp == 0.0;
    return k;
}

// Action terms of the VEC sites site0.. of S(sign*psi), whose neighbourhood n
// has been gathered:  S_i = 1/2 psi_i a_i - |x_i| - log(1 + exp(-2|x_i|)),
// x = a + h', a = A psi, in double-float arithmetic; the Sec. 4 estimators
// (tanh(x) sums, x in FP32 exactly as the force pass forms it, so a force
// pass may hand over its tanh values in tpre) and one conditional spin draw
// per site.
template <int DIM, int VEC>
__device__ __forceinline__ void vector_action(const FusedArgs &A, const ActConst &kc,
                                              const Nbr<DIM, VEC> &n, int64_t site0, float sign,
                                              uint32_t spin_traj, uint64_t seed, int chain,
                                              const float4 *tab, Acc &acc,
                                              const Vec<VEC> *tpre = nullptr) {
    float su[4];
    if constexpr (VEC == 4) {
        const float4 w = spin_u4_f32((uint32_t)(site0 >> 2), spin_traj, (uint32_t)chain, seed);
        su[0] = w.x; su[1] = w.y; su[2] = w.z; su[3] = w.w;
    }
    f2 sv{0.0f, 0.0f};
    float vT = 0.0f, vAT = 0.0f, vHT = 0.0f;   // estimator sums over the vector
    const bool has_h = A.hdf || !kc.hzero;
#pragma unroll
    for (int q = 0; q < VEC; ++q) {
        const float ps = sign * n.c.v[q];
        const f2 nbd = exact_nb<DIM, VEC>(n, q);
        const f2 a = df_add_q(df_mul_f(kc.C2, ps), df_mul(kc.bJ2, f2{sign * nbd.hi, sign * nbd.lo}));
        f2 x = a;
        if (A.hdf) {
            const float2 hh = A.hdf[site0 + q];
            const f2 hp = df_mul(kc.beta2, f2{hh.x, hh.y});
            x = df_add_q(a, hp);
        } else if (!kc.hzero) {
            x = df_add_q(a, kc.hp2);
        }
        const f2 ax = x.hi < 0.0f ? df_neg(x) : x;
        const f2 gl = log1pexp_neg(f2{2.0f * ax.hi, 2.0f * ax.lo}, tab);
        // S_i for this site, summed over the vector first (short chains)
        const f2 si = df_add_q(df_mul_f(a, 0.5f * ps), df_neg(df_add_q(ax, gl)));
        sv = df_add_q(sv, si);
        const float hf = A.hdf ? kc.betaf * A.hdf[site0 + q].x : kc.hpf;
        const float tq = tpre ? tpre->v[q]
                              : tanh_f(fmaf(kc.Cf, ps, fmaf(sign * kc.bJf, n.nb.v[q], hf)));
        vT += tq;
        vAT = fmaf(a.hi, tq, vAT);
        if (has_h) vHT = fmaf(hf, tq, vHT);
        float uu;
        if constexpr (VEC == 4) {
            uu = su[q];
        } else {
            const float4 w = spin_u4_f32((uint32_t)((site0 + q) >> 2), spin_traj, (uint32_t)chain,
                                         seed);
            const int qq = (int)((site0 + q) & 3);
            uu = qq == 0 ? w.x : qq == 1 ? w.y : qq == 2 ? w.z : w.w;
        }
        acc.sS += (uu < (1.0f + tq) * 0.5f) ? 1 : -1;
    }
    acc_add(acc.S, acc.Slo, sv);
    kahan_add(acc.sT, acc.cT, vT);
    kahan_add(acc.sAT, acc.cAT, vAT);
    if (has_h) kahan_add(acc.sHT, acc.cHT, vHT);
}

// FP32 momenta of the VEC sites site0.. (Sec. 3 momentum refresh): the same
// Philox draws as the momentum sweep.
template <int VEC>
__device__ __forceinline__ Vec<VEC> draw_momenta(int64_t site0, uint32_t traj, int chain,
                                                 uint64_t seed) {
    Vec<VEC> pv;
    if constexpr (VEC == 4) {
        const float4 w = momenta4_f32((uint32_t)(site0 >> 2), traj, (uint32_t)chain, seed);
        pv.v[0] = w.x; pv.v[1] = w.y; pv.v[2] = w.z; pv.v[3] = w.w;
    } else {
#pragma unroll
        for (int q = 0; q < VEC; ++q) {
            const float4 w = momenta4_f32((uint32_t)((site0 + q) >> 2), traj, (uint32_t)chain, seed);
            const int qq = (int)((site0 + q) & 3);
            pv.v[q] = qq == 0 ? w.x : qq == 1 ? w.y : qq == 2 ? w.z : w.w;
        }
    }
    return pv;
}

// FIRST: the first pass of the trajectory (draws the momenta, sums K0);
// LAST: the final pass (no drift; sums K1 and evaluates the proposal's
// action).  Both are compiled apart so the other passes keep a lean loop.
// The pass covers the slab of planes [z0, z0 + nzs) of the chain; plane
// indices inside are slab-local, site indices (random-number counters)
// absolute.
// eacc (first pass only, may be null): also accumulate the action and
// estimators of the start configuration (psi read by this pass) with the
// spin draw of a configuration set from outside -- the same per-site code, in
// the same per-thread order, as the evaluation sweep.
// Staging.  Bulk (BULK instances, VEC = 4: every plane a whole number of 16-byte
// vectors): one lane of warp 0 issues a copy group as one or two bulk copies
// (psi plane, p plane) that complete on the mbarrier of the group's psi slot,
// and every thread waits on it; `phase` holds the parity each slot's barrier is at (the same in every
// thread, carried from pass to pass).  A wait that runs out flags
// KERR_TIMEOUT and sets `dead`: no copy is issued or waited for after that
// except that thread 0, at the end of the pass, waits once more (bounded) for
// the copies it issued and has not seen complete; the launch finishes on
// whatever the rings hold and the host reports the error.  Otherwise every thread copies its share of each plane with 16-byte
// (VEC = 4) or 4-byte cp.async, which suits small planes better: there the
// copies are short and the issuing warp's extra work is on every plane's
// critical path.
template <int DIM, int VEC, int D, bool BULK, bool FIRST, bool LAST, bool EV = false>
__device__ void run_pass(const FusedArgs &A, const PassCfg &pc, const ChainParams &prm, int chain,
                         const Slots &sl, float *smem, const float4 *tab, Acc &acc, int z0,
                         int nzs, uint64_t *bars, uint32_t &phase, volatile int *dead,
                         Acc *eacc = nullptr) {
    constexpr int R = D + 4 + LAG;   // psi ring slots
    constexpr int RP = D + 2 + LAG;  // p ring slots
    constexpr int RU = 3 + LAG;      // u ring slots
    static_assert(R <= MAX_BARS, "one mbarrier per psi ring slot");
    constexpr bool bulk = BULK;
    static_assert(!BULK || VEC == 4, "bulk staging copies whole 16-byte vectors");
    // warp index as a value the compiler sees as the same in every lane
    const int warp = __shfl_sync(0xffffffffu, (int)(threadIdx.x >> 5), 0);
    const Geometry &g = A.g;
    const int P = g.P;
    float *psi_ring = smem;
    float *p_ring = psi_ring + R * P;
    float *u_ring = p_ring + RP * P;
    const int64_t cbase = (int64_t)chain * g.N;
    const float *__restrict__ gsrc = sel3(A, pc.src) + cbase;
    float *__restrict__ gdst = sel3(A, pc.dst) + cbase + (int64_t)z0 * P;
    float *__restrict__ gp = A.p + cbase + (int64_t)z0 * P;
    const int nz = g.nplanes;
    const int nvec = P / VEC;
    const int tid = threadIdx.x, nt = blockDim.x;

    // copy group s: psi plane z0 + s - 2 (periodic) into psi slot s % R and
    // p plane z0 + s - 4 into p slot s % RP (slots passed in: the loop below
    // advances them without a division)
    const uint32_t pbytes = (uint32_t)P * 4u;
    // copy groups [drain0, drain1] were in flight when a wait ran out (groups
    // are issued and awaited in order: the one that ran out and those issued
    // after it); none otherwise
    int drain0 = 0, drain1 = -1;
    int s_next = 0;     // next copy group to issue
    int issued = 0;     // warp 0: copy groups actually issued (bulk)
    auto issue = [&](int s, int slot_psi, int slot_p) {
        const int zpsi = s - 2;
        if constexpr (bulk) {
            // groups past psi plane nzs + 1 are empty (their p plane is
            // past the slab as well) and take no barrier phase; warp 0
            // forms the (warp-uniform) addresses, one elected lane issues
            if (zpsi > nzs + 1 || warp != 0 || *dead) return;
            const int zp = s - 4;
            const bool with_p = !FIRST && zp >= 0 && zp < nzs;   // the first pass draws p
            uint64_t *bar = bars + slot_psi;
            const float *src_psi = gsrc + (int64_t)wrap_plane(z0 + zpsi, nz) * P;
            if (mb::elect_one()) {
                mb::expect_tx(bar, with_p ? 2u * pbytes : pbytes);
                mb::bulk_g2s(psi_ring + slot_psi * P, src_psi, pbytes, bar);
                if (with_p) mb::bulk_g2s(p_ring + slot_p * P, gp + (int64_t)zp * P, pbytes, bar);
            }
            issued = s + 1;
            __syncwarp();
            return;
        }
        if (zpsi <= nzs + 1) {
            const int zw = wrap_plane(z0 + zpsi, nz);
            const float *src = gsrc + (int64_t)zw * P;
            float *dst = psi_ring + slot_psi * P;
            if constexpr (VEC == 4) {
                for (int v = tid; v < nvec; v += nt) cp_async16(dst + 4 * v, src + 4 * v);
            } else {
                for (int v = tid; v < P; v += nt) cp_async4(dst + v, src + v);
            }
        }
        const int zp = s - 4;
        if (zp >= 0 && zp < nzs && !FIRST) {   // the first pass draws p itself
            const float *src = gp + (int64_t)zp * P;
            float *dst = p_ring + slot_p * P;
            if constexpr (VEC == 4) {
                for (int v = tid; v < nvec; v += nt) cp_async16(dst + 4 * v, src + 4 * v);
            } else {
                for (int v = tid; v < P; v += nt) cp_async4(dst + v, src + v);
            }
        }
        cp_commit();
    };
    // ring slots: psi plane z (slab-local, z >= -2) lives in slot (z + 2) % R,
    // u plane z (z >= -1) in (z + 4) % RU, the p plane of copy group s in s % RP
    auto u_slot = [&](int z) -> float * { return u_ring + (unsigned)(z + 4) % RU * P; };
    auto wrapR = [](int x) { return x >= R ? x - R : (x < 0 ? x + R : x); };
    auto wrapRP = [](int x) { return x >= RP ? x - RP : x; };

    // copy group s (s <= nzs + 3) completes on the barrier of psi slot s % R
    auto wait_group = [&](int slot, int group) {
        if (!*dead) {
            if (mb::wait(bars + slot, (phase >> slot) & 1u)) {
                phase ^= 1u << slot;
                return;
            }
            *dead = 1;
            atomicOr(A.err, KERR_TIMEOUT);
        }
        // a wait ran out (here or in another thread): this group's phase and
        // those of the groups issued after it stay expected
        if (drain1 < drain0) {
            drain0 = group;
            drain1 = issued - 1;   // (in thread 0, the issuing warp's count)
        }
    };

    for (; s_next <= D + 2; ++s_next) issue(s_next, s_next % R, s_next % RP);
    if constexpr (bulk) {
        wait_group(0, 0);   // psi planes -2 and -1; plane 0 is waited for at it = -1
        wait_group(1, 1);
    }
    // at iteration it: sq = slot of psi plane it + 1, sp = p slot of copy group
    // it + D + 4 (the group issued in that iteration)
    int sq = 2 % R, sp = (D + 3) % RP;

    const float Cf = prm.Cf, bJf = prm.bJf;
    ActConst kc;
    if constexpr (LAST || EV) kc = act_const(prm);

    for (int it = -1; it <= nzs + LAG; ++it) {
        if constexpr (bulk) {
            if (it <= nzs) wait_group(sq, it + 3);   // group it + 3: psi plane it + 1, p plane it - 1
        } else {
            cp_wait<D>();
        }
        __syncthreads();
        // group it + D + 4 takes the psi slot of plane it - 3 (used last by the
        // previous iteration's drift) and the p slot it + 1
        issue(s_next++, wrapR(sq - 4), sp);
        // ---- u(it) = tanh(A psi + h') - psi on plane it ----
        if (it <= nzs) {
            const float *pm = psi_ring + wrapR(sq - 2) * P;
            const float *pcen = psi_ring + wrapR(sq - 1) * P;
            const float *pq = psi_ring + sq * P;
            float *uo = u_slot(it);
            const int zw = A.hdf ? wrap_plane(z0 + it, nz) : 0;
#pragma unroll
            for (int k = 0; k < NVMAX; ++k) {
                if (k >= sl.nwarp) break;
                const int e0 = sl.e0[k];
                Nbr<DIM, VEC> n;
                gather<DIM, VEC>(g, pm, pcen, pq, e0, sl.x0[k], n);
                float hpv[VEC];
#pragma unroll
                for (int q = 0; q < VEC; ++q)
                    hpv[q] = A.hdf ? prm.betaf * A.hdf[(int64_t)zw * P + e0 + q].x : prm.hpf;
                Vec<VEC> t;
#pragma unroll
                for (int q = 0; q < VEC; ++q)
                    t.v[q] = tanh_f(fmaf(Cf, n.c.v[q], fmaf(bJf, n.nb.v[q], hpv[q])));
                if (sl.valid[k]) {
                    Vec<VEC> u;
#pragma unroll
                    for (int q = 0; q < VEC; ++q) u.v[q] = t.v[q] - n.c.v[q];
                    stv<VEC>(uo + e0, u);
                    // the last pass's configuration is the proposal: its action
                    // from the neighbourhood already gathered (each plane once)
                    if constexpr (LAST) {
                        if (it >= 0 && it < nzs)
                            vector_action<DIM, VEC>(A, kc, n, (int64_t)(z0 + it) * P + e0, 1.0f,
                                                    pc.traj, A.seed, chain, tab, acc, &t);
                    }
                    if constexpr (FIRST && EV) {
                        if (it >= 0 && it < nzs)
                            vector_action<DIM, VEC>(A, kc, n, (int64_t)(z0 + it) * P + e0, 1.0f,
                                                    TRAJ_INIT, 0, chain, tab, *eacc, &t);
                    }
                }
            }
        }
        if constexpr (LAG == 0) __syncthreads();
        // ---- F(z) = A u, kick and drift on plane z = it - 1 - LAG ----
        const int z = it - 1 - LAG;
        if (z >= 0 && z < nzs) {
            const float *um = u_slot(z - 1), *uc = u_slot(z), *uq = u_slot(z + 1);
            const float *psz = psi_ring + wrapR(sq - 1 - LAG - 1) * P;   // psi plane z
            const float *ppz = p_ring + wrapRP(sp + 1) * P;   // p plane z: group z + 4
            float *gpz = gp + (int64_t)z * P;
            float *gdz = gdst + (int64_t)z * P;
#pragma unroll
            for (int k = 0; k < NVMAX; ++k) {
                if (k >= sl.nwarp) break;
                const int e0 = sl.e0[k];
                Nbr<DIM, VEC> n;
                gather<DIM, VEC>(g, um, uc, uq, e0, sl.x0[k], n);
                Vec<VEC> pv;
                if constexpr (FIRST)
                    pv = draw_momenta<VEC>((int64_t)(z0 + z) * P + e0, pc.traj, chain, A.seed);
                else
                    pv = ldv<VEC>(ppz + e0);
                if (FIRST && sl.valid[k]) {
#pragma unroll
                    for (int q = 0; q < VEC; ++q)
                        acc_add(acc.K0, acc.K0lo, two_prod(pv.v[q], 0.5f * pv.v[q]));
                }
#pragma unroll
                for (int q = 0; q < VEC; ++q) {
                    const float F = fmaf(Cf, n.c.v[q], bJf * n.nb.v[q]);
                    pv.v[q] = fmaf(pc.kick, F, pv.v[q]);
                }
                if (sl.valid[k]) {
                    stv<VEC>(gpz + e0, pv);
                    if constexpr (LAST) {
#pragma unroll
                        for (int q = 0; q < VEC; ++q)
                            acc_add(acc.K1, acc.K1lo, two_prod(pv.v[q], 0.5f * pv.v[q]));
                    } else {
                        const Vec<VEC> ps = ldv<VEC>(psz + e0);
                        Vec<VEC> pnew;
#pragma unroll
                        for (int q = 0; q < VEC; ++q) pnew.v[q] = fmaf(pc.drift, pv.v[q], ps.v[q]);
                        stv<VEC>(gdz + e0, pnew);
                    }
                }
            }
        }
        sq = wrapR(sq + 1);
        sp = wrapRP(sp + 1);
    }
    if constexpr (bulk) {
        // after a wait ran out: thread 0 waits once more, bounded, for the
        // copies it issued and has not seen complete, so none is still
        // writing this CTA's shared memory when the launch ends
        if (threadIdx.x == 0)
            for (int gi = drain0; gi <= drain1; ++gi) mb::wait(bars + gi % R, (phase >> (gi % R)) & 1u);
        // the next pass's bulk copies read the planes written here
        mb::fence_global_to_async();
    } else {
        cp_wait<0>();
    }
    __syncthreads();
}

// Momentum refresh (Sec. 3): p ~ N(0,1) for every site of the chain, written
// to global memory.  No barriers: every thread streams its own vectors.
template <int VEC>
__device__ void momenta_sweep(const FusedArgs &A, int chain, uint32_t traj, const Slots &sl,
                              int z0, int z1) {
    const Geometry &g = A.g;
    float *gp = A.p + (int64_t)chain * g.N;
    for (int z = z0; z < z1; ++z) {
#pragma unroll
        for (int k = 0; k < NVMAX; ++k) {
            if (k >= sl.nwarp) break;
            if (!sl.valid[k]) continue;
            const int64_t site0 = (int64_t)z * g.P + sl.e0[k];
            Vec<VEC> pv;
            if constexpr (VEC == 4) {
                const float4 w = momenta4_f32((uint32_t)(site0 >> 2), traj, (uint32_t)chain, A.seed);
                pv.v[0] = w.x; pv.v[1] = w.y; pv.v[2] = w.z; pv.v[3] = w.w;
            } else {
#pragma unroll
                for (int q = 0; q < VEC; ++q) {
                    const float4 w = momenta4_f32((uint32_t)((site0 + q) >> 2), traj,
                                                  (uint32_t)chain, A.seed);
                    const int qq = (int)((site0 + q) & 3);
                    pv.v[q] = qq == 0 ? w.x : qq == 1 ? w.y : qq == 2 ? w.z : w.w;
                }
            }
            stv<VEC>(gp + site0, pv);
        }
    }
}

// Action S(sign*psi) (Sec. 2, Eq. phi_psi_substitution in the form
// S = 1/2 psi.A psi - sum_i log 2cosh((A psi)_i + h'_i)) to FP64 accuracy in
// double-float arithmetic, and the Sec. 4 estimators with one conditional
// spin draw, over the planes [z0, z1) of the chain stored in buffer `buf`.
// No barriers: every thread streams its own vectors, neighbours come from
// global memory (L1/L2).
// (The proposal's action at the end of a trajectory is evaluated inside the
// last force pass instead; this sweep serves the sign flip and the current
// state.)
template <int DIM, int VEC, bool GL>
__device__ void action_sweep(const FusedArgs &A, const ChainParams &prm, int chain, int buf,
                             float sign, uint32_t spin_traj, uint64_t seed, const Slots &sl,
                             const float4 *tab, Acc &acc, int z0, int z1) {
    const Geometry &g = A.g;
    const int P = g.P, nz = g.nplanes;
    const float *psi = sel3(A, buf) + (int64_t)chain * g.N;
    const ActConst kc = act_const(prm);
    for (int z = z0; z < z1; ++z) {
        const float *pc = psi + (int64_t)z * P;
        const float *pm = psi + (int64_t)(z == 0 ? nz - 1 : z - 1) * P;
        const float *pq = psi + (int64_t)(z == nz - 1 ? 0 : z + 1) * P;
#pragma unroll
        for (int k = 0; k < NVMAX; ++k) {
            if (k >= sl.nwarp) break;
            if (!sl.valid[k]) continue;
            const int e0 = sl.e0[k];
            Nbr<DIM, VEC> n;
            gather<DIM, VEC, GL>(g, pm, pc, pq, e0, sl.x0[k], n);
            vector_action<DIM, VEC>(A, kc, n, (int64_t)z * P + e0, sign, spin_traj, seed, chain,
                                    tab, acc);
        }
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

// CL: compiled for chains split over a cluster (launched with a cluster
// size); the unsplit instance carries no cluster instructions at all.
template <int DIM, int VEC, int D, bool CL, bool BULK>
__global__ void __launch_bounds__(CL ? MAX_THREADS : MAX_THREADS_UNSPLIT, CL ? 1 : 2)
    fused_lattice_kernel(FusedArgs A, Schedule S) {
    extern __shared__ float4 smem_f4[];
    float *smem = reinterpret_cast<float *>(smem_f4);
    const Geometry &g = A.g;
    const size_t rb = ring_bytes(g.P, D);
    // The launch's shared-memory size says where the log(1 + e^-y) table
    // lives: copied into shared memory when the host gave room for it (it
    // does when that costs no resident CTAs), else read through L1 from
    // global memory.
    uint32_t dsm;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dsm));
    const bool tab_in_smem = dsm >= rb + LOG1PEXP_NODES * 16 + RED_BYTES;
    float4 *tab_s = reinterpret_cast<float4 *>(smem + rb / 4);
    const float4 *tab = tab_in_smem ? tab_s : A.lpe_tab;
    double *red = reinterpret_cast<double *>(smem + rb / 4 + (tab_in_smem ? LOG1PEXP_NODES * 4 : 0));
    int *bcast = reinterpret_cast<int *>(red + 32 * 8);   // [0], [1] broadcasts, [2] dead flag
    double *xch = red + 32 * 8 + 2;   // two exchange buffers of XCH_WORDS
    uint64_t *bars = reinterpret_cast<uint64_t *>(xch + 2 * XCH_WORDS);

    // CTAs per chain (the launch's cluster size) and this CTA's slab
    const int cs = CL ? cluster_size() : 1, cr = CL ? cluster_rank() : 0;
    const int chain = A.chain0 + (int)(blockIdx.x / (unsigned)cs);
    if (chain >= A.n_chains) return;   // uniform over the cluster
    if (cs != A.cs && threadIdx.x == 0 && cr == 0) atomicOr(A.err, KERR_BOUNDS);
    const int nz = g.nplanes;
    const int z0 = (int)((int64_t)cr * nz / cs), z1 = (int)((int64_t)(cr + 1) * nz / cs);
    const bool lead = cr == 0;   // writes the chain's state
    ChainState *st = A.state + chain;
    const ChainParams prm = A.params[chain];
    const double invN = 1.0 / (double)g.N;
    const Slots sl = make_slots<VEC>(g);

    if (A.mode == MODE_MOMENTA) {
        momenta_sweep<VEC>(A, chain, A.traj0, sl, z0, z1);
        return;
    }
    if (tab_in_smem)
        for (int i = threadIdx.x; i < LOG1PEXP_NODES; i += blockDim.x) tab_s[i] = A.lpe_tab[i];
    if (threadIdx.x == 0) {
        bcast[2] = 0;
        if constexpr (BULK) {
            for (int i = 0; i < D + 4 + LAG; ++i) mb::init(bars + i, 1);
            mb::init_fence();
        }
    }
    __syncthreads();
    uint32_t phase = 0;   // parity of each copy-group barrier

    if (A.mode == MODE_EVAL) {
        Acc acc = acc_zero();
        const int start = st->start;
        action_sweep<DIM, VEC, CL>(A, prm, chain, start, 1.0f, TRAJ_INIT, 0, sl, tab, acc, z0, z1);
        double v[5] = {acc_val(acc.S, acc.Slo), kahan_val(acc.sT, acc.cT),
                       kahan_val(acc.sAT, acc.cAT), kahan_val(acc.sHT, acc.cHT), (double)acc.sS};
        chain_sum<5, CL>(v, red, xch, cs);
        if (threadIdx.x == 0 && lead) {
            st->S = v[0];
            set_obs(st, prm, v[1], v[2], v[3], v[4], invN);
            st->prop = start;
        }
        if (CL && cs > 1) cluster_barrier();   // no CTA leaves while its buffer may be read
        return;
    }

    // the chain's state as every CTA of the cluster tracks it (the same
    // values in all of them: they add the same sums in the same order)
    int start = st->start;
    double S_cur = st->S;
    for (int k = 0; k < A.n_traj; ++k) {
        const uint32_t traj = A.traj0 + (uint32_t)k;
        Acc acc = acc_zero();
        // a configuration set from outside: its action and observables come
        // from the first force pass of the first trajectory
        const bool eval_start = k == 0 && A.eval_start;
        Acc ea = acc_zero();
        // the integrator's force passes; the first draws the momenta (Sec. 3
        // refresh), the last evaluates the proposal's action
        for (int j = 0; j < S.n_pass; ++j) {
            PassCfg pc;
            pc.src = buf_loc(start, j);
            pc.dst = buf_loc(start, j + 1);
            pc.kick = (float)(S.kick[j] * prm.eps);
            pc.drift = (float)(S.drift[j] * prm.eps);
            pc.first = (j == 0);
            pc.last = (j == S.n_pass - 1);
            pc.traj = traj;
            // (n_pass >= 2: the first pass is never the last)
            const int nzs = z1 - z0;
            if (pc.first && eval_start)
                run_pass<DIM, VEC, D, BULK, true, false, true>(A, pc, prm, chain, sl, smem, tab, acc, z0,
                                                         nzs, bars, phase, bcast + 2, &ea);
            else if (pc.first)
                run_pass<DIM, VEC, D, BULK, true, false>(A, pc, prm, chain, sl, smem, tab, acc, z0, nzs,
                                                   bars, phase, bcast + 2);
            else if (pc.last)
                run_pass<DIM, VEC, D, BULK, false, true>(A, pc, prm, chain, sl, smem, tab, acc, z0, nzs,
                                                   bars, phase, bcast + 2);
            else
                run_pass<DIM, VEC, D, BULK, false, false>(A, pc, prm, chain, sl, smem, tab, acc, z0, nzs,
                                                    bars, phase, bcast + 2);
            // the next pass reads (and the one after rewrites) the planes
            // beyond this slab's ends, written by the neighbouring CTAs
            if (CL && cs > 1) cluster_barrier();
        }
        if (eval_start) {
            double ev[5] = {acc_val(ea.S, ea.Slo), kahan_val(ea.sT, ea.cT),
                            kahan_val(ea.sAT, ea.cAT), kahan_val(ea.sHT, ea.cHT), (double)ea.sS};
            chain_sum<5, CL>(ev, red, xch + XCH_WORDS, cs);
            if (threadIdx.x == 0) {
                S_cur = ev[0];
                if (lead) {
                    st->S = ev[0];
                    set_obs(st, prm, ev[1], ev[2], ev[3], ev[4], invN);
                    st->prop = start;
                }
            }
        }
        const int prop = buf_loc(start, S.n_pass - 1);
        double v[7] = {acc_val(acc.K0, acc.K0lo), acc_val(acc.K1, acc.K1lo),
                       acc_val(acc.S, acc.Slo), kahan_val(acc.sT, acc.cT),
                       kahan_val(acc.sAT, acc.cAT), kahan_val(acc.sHT, acc.cHT), (double)acc.sS};
        chain_sum<7, CL>(v, red, xch, cs);
        if (threadIdx.x == 0) {
            const double S0 = S_cur;
            const double dH = (v[1] + v[2]) - (v[0] + S0);
            const double logu = accept_logu(traj, (uint32_t)chain, A.seed, PURPOSE_ACC);
            const bool accd = logu < -dH;
            if (lead) {
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
            }
            if (accd) S_cur = v[2];
            bcast[0] = accd ? prop : start;
        }
        __syncthreads();
        start = bcast[0];
        __syncthreads();
        // ---- optional global sign flip psi -> -psi (Sec. 3, ergodicity) ----
        if (A.flip_every > 0 && ((traj + 1) % (uint32_t)A.flip_every) == 0) {
            Acc fa = acc_zero();
            action_sweep<DIM, VEC, CL>(A, prm, chain, start, -1.0f, traj, A.seed, sl, tab, fa, z0, z1);
            double w[5] = {acc_val(fa.S, fa.Slo), kahan_val(fa.sT, fa.cT),
                           kahan_val(fa.sAT, fa.cAT), kahan_val(fa.sHT, fa.cHT), (double)fa.sS};
            chain_sum<5, CL>(w, red, xch + XCH_WORDS, cs);
            if (threadIdx.x == 0) {
                const double lu = accept_logu(traj, (uint32_t)chain, A.seed, PURPOSE_FLIP);
                const bool fl = lu < -(w[0] - S_cur);
                if (fl) {
                    S_cur = w[0];
                    if (lead) {
                        st->S = w[0];
                        set_obs(st, prm, w[1], w[2], w[3], w[4], invN);
                        st->rec[ISING_REC_FLIPPED] = 1.0;
                    }
                }
                bcast[1] = fl ? 1 : 0;
            }
            __syncthreads();
            if (bcast[1]) {
                // -psi goes to the buffer that is neither current nor the proposal,
                // so the MD end point stays readable
                const int f = (start != prop) ? 3 - start - prop : (start + 1) % 3;
                const int64_t off = (int64_t)chain * g.N + (int64_t)z0 * g.P;
                const int64_t cnt = (int64_t)(z1 - z0) * g.P;
                const float *gs = sel3(A, start) + off;
                float *gf = sel3(A, f) + off;
                for (int64_t i = threadIdx.x; i < cnt; i += blockDim.x) gf[i] = -gs[i];
                if constexpr (BULK) mb::fence_global_to_async();   // read by the next pass's copies
                start = f;
                if (threadIdx.x == 0 && lead) st->start = f;
                if (CL && cs > 1) cluster_barrier();   // the next pass reads the other slabs' planes
            }
            __syncthreads();
        }
        // ---- measurement: a repeated configuration repeats its measurement ----
        if (threadIdx.x == 0 && lead && (int64_t)traj >= (int64_t)A.n_therm) {
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
    if (CL && cs > 1) cluster_barrier();   // no CTA leaves while its exchange buffers may be read
}

// Shared-memory size of a launch: with the table if that leaves as many CTAs
// resident per SM as without it (the occupancy calculator decides), else
// without.  The last answers are cached per thread.
template <class K>
static int launch_smem(K kern, const Geometry &g, int D, int threads) {
    struct Memo {
        const void *kern;
        int P, D, threads, smem;
    };
    thread_local Memo memo[8] = {};
    thread_local int next = 0;
    for (const Memo &m : memo)
        if (m.smem && m.kern == reinterpret_cast<const void *>(kern) && m.P == g.P && m.D == D &&
            m.threads == threads)
            return m.smem;
    const int base = (int)(ring_bytes(g.P, D) + RED_BYTES);
    const int with_tab = base + LOG1PEXP_NODES * 16;
    int n_with = 0, n_without = 0;
    int smem = base;
    if (with_tab <= 227 * 1024 &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n_with, kern, threads, with_tab) == cudaSuccess &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n_without, kern, threads, base) == cudaSuccess &&
        n_with >= n_without)
        smem = with_tab;
    cudaGetLastError();
    memo[next] = Memo{reinterpret_cast<const void *>(kern), g.P, D, threads, smem};
    next = (next + 1) % 8;
    return smem;
}

template <int DIM, int VEC, int D, bool CL, bool BULK = false>
cudaError_t kernel_node(const FusedArgs &a, int threads, cudaKernelNodeParams *np, void **args) {
    static bool configured = false;
    auto kern = fused_lattice_kernel<DIM, VEC, D, CL, BULK>;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             227 * 1024);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const int smem = launch_smem(kern, a.g, D, threads);
    np->func = reinterpret_cast<void *>(kern);
    np->gridDim = dim3((unsigned)((a.n_chains - a.chain0) * a.cs), 1, 1);
    np->blockDim = dim3((unsigned)threads, 1, 1);
    np->sharedMemBytes = (unsigned)smem;
    np->kernelParams = args;
    np->extra = nullptr;
    return cudaSuccess;
}

template <int DIM, bool CL>
cudaError_t node_dim(const FusedArgs &a, int threads, int depth, int vec, cudaKernelNodeParams *np,
                     void **args) {
    if (vec == 4) {
        // the staging is a compile-time choice: one kernel carrying both
        // paths measured slower in either mode (register allocation)
        if (a.bulk) {
            if (depth >= 4) return kernel_node<DIM, 4, 4, CL, true>(a, threads, np, args);
            if (depth >= 2) return kernel_node<DIM, 4, 2, CL, true>(a, threads, np, args);
            return kernel_node<DIM, 4, 1, CL, true>(a, threads, np, args);
        }
        if (depth >= 4) return kernel_node<DIM, 4, 4, CL>(a, threads, np, args);
        if (depth >= 2) return kernel_node<DIM, 4, 2, CL>(a, threads, np, args);
        return kernel_node<DIM, 4, 1, CL>(a, threads, np, args);
    }
    if (depth >= 4) return kernel_node<DIM, 1, 4, CL>(a, threads, np, args);
    if (depth >= 2) return kernel_node<DIM, 1, 2, CL>(a, threads, np, args);
    return kernel_node<DIM, 1, 1, CL>(a, threads, np, args);
}

}  // namespace

// Kernel-node parameters of one dimension's instances (one translation unit
// each, compiled in parallel); CL selects the cluster-split instances.
cudaError_t fused_node_1d(const FusedArgs &a, int threads, int depth, int vec,
                          cudaKernelNodeParams *np, void **args);
cudaError_t fused_node_2d(const FusedArgs &a, int threads, int depth, int vec,
                          cudaKernelNodeParams *np, void **args);
cudaError_t fused_node_2d_cl(const FusedArgs &a, int threads, int depth, int vec,
                             cudaKernelNodeParams *np, void **args);
cudaError_t fused_node_3d(const FusedArgs &a, int threads, int depth, int vec,
                          cudaKernelNodeParams *np, void **args);
cudaError_t fused_node_3d_cl(const FusedArgs &a, int threads, int depth, int vec,
                             cudaKernelNodeParams *np, void **args);

}  // namespace ihmc
