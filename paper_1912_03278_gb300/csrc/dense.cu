// dense.cu -- dense all-to-all couplings on the tensor cores.
//
// For a block of chains Psi (chains x sites, chain-major) the force of Sec. 3,
// F = A (tanh(A psi + h') - psi) with A = beta*J + C*1, is two BF16 tcgen05
// GEMMs per force evaluation, G = J Psi^T, with fused FP32 epilogues:
//   pass 1:  a = beta G + C psi,  u = tanh(a + h') - psi      -> U (FP32, BF16)
//   pass 2:  F = beta (J U^T) + C u,  p += kick F,  psi += drift p  (FP32, BF16)
// beta and C stay in the FP32 epilogue, so one BF16 copy of J serves every
// chain's beta.  The action of the end point needs a = A psi to FP64
// accuracy: a double-float GEMM on the FP32 pipe (exact products through FMA,
// compensated sums) followed by a per-chain kernel that evaluates S, the Sec. 4
// estimators, dH and the Metropolis test (Sec. 3).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include "df32.cuh"
#include "device_common.cuh"
#include "internal.h"
#include "tc_gemm.cuh"

namespace ihmc {
namespace {

// ---------------------------------------------------------------- GEMM tests
struct StoreEpi {
    static constexpr int W = 16;
    float *out;
    int M;
    __device__ int a_off(int) const { return 0; }
    __device__ int b_off(int) const { return 0; }
    __device__ __forceinline__ void operator()(int m, int n0, const float (&v)[W], int) const {
#pragma unroll
        for (int j = 0; j < W; ++j) out[(int64_t)(n0 + j) * M + m] = v[j];
    }
};


template <bool PAIR>
__global__ void __launch_bounds__(tc::THREADS, 1)
    gemm_store_kernel(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb,
                      float *out, int M, int N, int K, int *err) {
    StoreEpi epi{out, M};
    using Md = tc::Mode<PAIR>;
    tc::gemm_persistent<PAIR>(&ta, &tb, M / Md::TILE_M, N / Md::TILE_N, K / tc::BK, 1, epi, err);
}

// ------------------------------------------------------- force epilogues
// Each epilogue call handles W chains n0.. of one site m per thread; a warp
// covers 32 consecutive sites, so every load and store below is one 128-byte
// (64-byte for BF16) coalesced access per warp.  The kernel's pointers live in
// registers; lane j < W reads chain n0+j's (beta, C, eps, h') as one float4
// and the other lanes take it by shuffle.  All loads are issued before the
// first store, so each thread keeps its W (or 3W) reads in flight at once.
template <int W>
__device__ __forceinline__ float4 chain_coef(const ChainParams *params, int n0, int n_chains) {
    const int n = n0 + (int)(threadIdx.x & (W - 1));
    return n < n_chains ? *reinterpret_cast<const float4 *>(&params[n].betaf)
                        : make_float4(0.f, 0.f, 0.f, 0.f);
}

// Low-precision GEMM operands: BF16, or FP8 E4M3 holding x / FP8_OP_SCALE
// (a fixed scale, so the force stays a function of psi alone and the
// integrator reversible; values beyond +-FP8_OP_RANGE saturate).  With FP8 the
// accumulator of row m is scaled by the row's J scale times FP8_OP_SCALE.
template <bool FP8>
struct Low {
    using T = __nv_bfloat16;
    static __device__ __forceinline__ T from(float x) { return __float2bfloat16_rn(x); }
};
template <>
struct Low<true> {
    using T = uint8_t;
    static __device__ __forceinline__ T from(float x) {
        return (T)__nv_cvt_float_to_fp8(x * (1.0f / FP8_OP_SCALE), __NV_SATFINITE, __NV_E4M3);
    }
};

// u = tanh(beta G + C psi + h') - psi  ->  U (FP32 and low precision).  One
// load per element, so 32 columns per chunk keep enough reads in flight.
template <bool FP8>
struct Epi1 {
    static constexpr int W = 32;
    const float *psi;
    float *u32;
    typename Low<FP8>::T *ulow;
    const float *row_scale;   // FP8: per-row scale of J
    const float2 *hdf;
    const ChainParams *params;
    int N, n_chains;
    __device__ int a_off(int) const { return 0; }
    __device__ int b_off(int) const { return 0; }
    __device__ __forceinline__ void operator()(int m, int n0, const float (&v)[W], int) const {
        const float4 cf = chain_coef<W>(params, n0, n_chains);
        const int64_t base = (int64_t)n0 * N + m;   // column j sits j*N further (N*W < 2^31)
        const float *ps_in = psi + base;
        float ps[W];
#pragma unroll
        for (int j = 0; j < W; ++j) ps[j] = (n0 + j < n_chains) ? ps_in[j * N] : 0.0f;
        const float hm = hdf ? hdf[m].x : 0.0f;
        const float gs = FP8 ? row_scale[m] * FP8_OP_SCALE : 1.0f;
#pragma unroll
        for (int j = 0; j < W; ++j) {
            const float bj = __shfl_sync(0xffffffffu, cf.x, j);
            const float cj = __shfl_sync(0xffffffffu, cf.y, j);
            const float hj = __shfl_sync(0xffffffffu, cf.w, j);
            const float a = fmaf(bj, FP8 ? v[j] * gs : v[j], cj * ps[j]);
            const float u = tanh_f(a + (hdf ? bj * hm : hj)) - ps[j];
            if (n0 + j < n_chains) {
                u32[base + j * N] = u;
                ulow[base + j * N] = Low<FP8>::from(u);
            }
        }
    }
};

// F = beta (J U) + C u;  p += kick eps F;  psi += drift eps p (FP32 and low
// precision).
template <bool FP8>
struct Epi2 {
    static constexpr int W = 16;
    const float *u32;
    float *p, *psi;
    typename Low<FP8>::T *psilow;
    const float *row_scale;   // FP8: per-row scale of J
    const ChainParams *params;
    int N, n_chains;
    float kick, drift;   // schedule coefficients (times each chain's eps)
    bool do_drift;
    __device__ int a_off(int) const { return 0; }
    __device__ int b_off(int) const { return 0; }
    __device__ __forceinline__ void operator()(int m, int n0, const float (&v)[W], int) const {
        const float4 cf = chain_coef<W>(params, n0, n_chains);
        const int64_t base = (int64_t)n0 * N + m;   // column j sits j*N further (N*W < 2^31)
        const float *u_in = u32 + base;
        float *p_io = p + base, *ps_io = psi + base;
        float uu[W], pp[W], ps[W];
        const float gs = FP8 ? row_scale[m] * FP8_OP_SCALE : 1.0f;
#pragma unroll
        for (int j = 0; j < W; ++j) {
            const bool live = n0 + j < n_chains;
            uu[j] = live ? u_in[j * N] : 0.0f;
            pp[j] = live ? p_io[j * N] : 0.0f;
            ps[j] = (live && do_drift) ? ps_io[j * N] : 0.0f;
        }
#pragma unroll
        for (int j = 0; j < W; ++j) {
            const float bj = __shfl_sync(0xffffffffu, cf.x, j);
            const float cj = __shfl_sync(0xffffffffu, cf.y, j);
            const float ej = __shfl_sync(0xffffffffu, cf.z, j);
            if (n0 + j >= n_chains) continue;
            const float F = fmaf(bj, FP8 ? v[j] * gs : v[j], cj * uu[j]);
            const float pn = fmaf(kick * ej, F, pp[j]);
            p_io[j * N] = pn;
            if (do_drift) {
                const float psn = fmaf(drift * ej, pn, ps[j]);
                ps_io[j * N] = psn;
                psilow[base + j * N] = Low<FP8>::from(psn);
            }
        }
    }
};

template <bool FP8>
__device__ __forceinline__ typename Low<FP8>::T *low_psi(const DenseArgs &d) {
    if constexpr (FP8) return d.psi8; else return d.psi16;
}
template <bool FP8>
__device__ __forceinline__ typename Low<FP8>::T *low_u(const DenseArgs &d) {
    if constexpr (FP8) return d.u8; else return d.u16;
}

template <bool PAIR, bool FP8>
__global__ void __launch_bounds__(tc::THREADS, 1)
    force1_kernel(const __grid_constant__ CUtensorMap tj, const __grid_constant__ CUtensorMap tpsi,
                  const __grid_constant__ DenseArgs d) {
    Epi1<FP8> epi{d.psi, d.u32, low_u<FP8>(d), d.sJ8, d.hdf, d.params, d.N, d.n_chains};
    using Md = tc::Mode<PAIR>;
    tc::gemm_persistent<PAIR, Epi1<FP8>, FP8>(&tj, &tpsi, d.N / Md::TILE_M, d.b_pad / Md::TILE_N,
                                              d.N / tc::Elem<FP8>::BK_ELEMS, 1, epi, d.err);
}

template <bool PAIR, bool FP8>
__global__ void __launch_bounds__(tc::THREADS, 1)
    force2_kernel(const __grid_constant__ CUtensorMap tj, const __grid_constant__ CUtensorMap tu,
                  const __grid_constant__ DenseArgs d, float kick, float drift, int do_drift) {
    Epi2<FP8> epi{d.u32,  d.p,        d.psi, low_psi<FP8>(d), d.sJ8,   d.params,
                  d.N,    d.n_chains, kick,  drift,           do_drift != 0};
    using Md = tc::Mode<PAIR>;
    tc::gemm_persistent<PAIR, Epi2<FP8>, FP8>(&tj, &tu, d.N / Md::TILE_M, d.b_pad / Md::TILE_N,
                                              d.N / tc::Elem<FP8>::BK_ELEMS, 1, epi, d.err);
}

// ------------------------------------------ FP64-accurate G = J Psi^T (action)
// Exact digit products on the tensor cores.  Each row i of J is scaled by
// 2^e_i and each chain c of Psi by 2^f_c so that all entries lie in
// [-1/2, 1/2], then written in base 128 with ACT_DIGITS = 6 signed digits in
// [-64, 64] (exact in BF16):  J_ij = 2^e_i sum_s d_s 2^(-7(s+1)),
// psi_cj = 2^f_c sum_t q_t 2^(-7(t+1)).  One digit-plane product sums N terms
// of magnitude <= 2^12, so for N <= 4096 every partial sum is an integer
// of magnitude <= 2^24 and the FP32 accumulator holds it exactly.  The
// epilogue adds the ACT_PAIRS = 21 products with s + t <= 5 exactly, as
// 64-bit integers (no FP64 arithmetic, which is slow on this GPU):
//   G_int = sum_{s+t<=5} 2^(7(5-s-t)) sum_j d_s,ij q_t,cj   (|G_int| < 2^60),
//   (J psi)_ic = 2^(e_i + f_c - 49) G_int.
// The dropped products (s+t >= 6) and the digit truncation weigh below
// 2^-40 of 2^(e_i+f_c), far under the accuracy the action needs (Sec. 3:
// dH decides the Metropolis test).
__constant__ int c_pair_s[ACT_PAIRS] = {0, 0, 1, 0, 1, 2, 0, 1, 2, 3, 0,
                                        1, 2, 3, 4, 0, 1, 2, 3, 4, 5};
__constant__ int c_pair_t[ACT_PAIRS] = {0, 1, 0, 2, 1, 0, 3, 2, 1, 0, 4,
                                        3, 2, 1, 0, 5, 4, 3, 2, 1, 0};

struct EpiG {
    static constexpr int W = 32;   // 32 reads of 8 bytes in flight per thread
    long long *G;
    int N, n_chains, b_pad;
    __device__ int a_off(int r) const { return c_pair_s[r] * N; }
    __device__ int b_off(int r) const { return c_pair_t[r] * b_pad; }
    __device__ __forceinline__ void operator()(int m, int n0, const float (&v)[W], int r) const {
        const int sh = ACT_BITS * (ACT_DIGITS - 1 - c_pair_s[r] - c_pair_t[r]);
        long long *g = G + (int64_t)n0 * N + m;
        if (r == 0) {
#pragma unroll
            for (int j = 0; j < W; ++j)
                if (n0 + j < n_chains) g[j * N] = (long long)__float2int_rn(v[j]) << sh;
        } else {
            long long old[W];
#pragma unroll
            for (int j = 0; j < W; ++j) old[j] = (n0 + j < n_chains) ? g[j * N] : 0;
#pragma unroll
            for (int j = 0; j < W; ++j)
                if (n0 + j < n_chains) g[j * N] = old[j] + ((long long)__float2int_rn(v[j]) << sh);
        }
    }
};

template <bool PAIR>
__global__ void __launch_bounds__(tc::THREADS, 1)
    action_kernel(const __grid_constant__ CUtensorMap tjd, const __grid_constant__ CUtensorMap tpd,
                  const __grid_constant__ DenseArgs d) {
    EpiG epi{d.Gint, d.N, d.n_chains, d.b_pad};
    using Md = tc::Mode<PAIR>;
    tc::gemm_persistent<PAIR>(&tjd, &tpd, d.N / Md::TILE_M, d.b_pad / Md::TILE_N, d.N / tc::BK,
                              ACT_PAIRS, epi, d.err);
}

// Digits of Psi (chain c = block): f_c from max |psi_c|, then ACT_DIGITS
// base-128 digits in [-64, 64] of X = round(psi 2^(42 - f_c)), the integer
// taken from the FP32 bit pattern, per site; each digit plane is b_pad x N
// (padding chains get zero digits).  |psi 2^-f_c| < 1/2, so |X| <= 2^41 and
// six digits represent it exactly.
__global__ void __launch_bounds__(256) k_psi_digits(const float *__restrict__ psi,
                                                    __nv_bfloat16 *__restrict__ dig,
                                                    int *__restrict__ chain_exp, int N,
                                                    int n_chains, int b_pad) {
    __shared__ float red[8];
    const int n = blockIdx.x;
    const bool live = n < n_chains;
    float mx = 0.0f;
    if (live)
        for (int m = threadIdx.x; m < N; m += blockDim.x)
            mx = fmaxf(mx, fabsf(psi[(int64_t)n * N + m]));
    for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    mx = 0.0f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mx = fmaxf(mx, red[w]);
    const int f = mx > 0.0f ? ilogbf(mx) + 2 : 0;   // max |psi| * 2^-f < 1/2
    if (threadIdx.x == 0) chain_exp[n] = f;
    constexpr int FRAC = ACT_BITS * ACT_DIGITS;   // 42 fraction bits
    for (int m = threadIdx.x; m < N; m += blockDim.x) {
        long long X = 0;
        if (live) {
            const uint32_t b = __float_as_uint(psi[(int64_t)n * N + m]);
            const int be = (int)((b >> 23) & 0xFF);
            if (be) {   // normal (subnormals lie far below the last digit)
                const long long M = (long long)((b & 0x7FFFFFu) | 0x800000u);
                const int sh = be - 150 - f + FRAC;   // psi 2^(FRAC-f) = M 2^sh
                if (sh >= 0)
                    X = M << sh;
                else if (sh > -40)
                    X = (M + (1ll << (-sh - 1))) >> (-sh);
                if (b >> 31) X = -X;
            }
        }
        // low digits in [-64, 63]; the top digit takes the rest, |rest| <= 64
#pragma unroll
        for (int t = ACT_DIGITS - 1; t >= 1; --t) {
            const int q = (int)(((X + 64) & 127) - 64);
            X = (X - q) >> ACT_BITS;
            dig[((int64_t)t * b_pad + n) * N + m] = __float2bfloat16_rn((float)q);
        }
        dig[(int64_t)n * N + m] = __float2bfloat16_rn((float)(int)X);
    }
}

// ------------------------------------------------------------- state helpers
__global__ void k_copy_state(const float *__restrict__ src, float *__restrict__ dst,
                             __nv_bfloat16 *__restrict__ dst16, uint8_t *__restrict__ dst8,
                             int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float v = src[i];
        dst[i] = v;
        if (dst16) dst16[i] = Low<false>::from(v);
        if (dst8) dst8[i] = Low<true>::from(v);
    }
}

// p ~ N(0,1), FP32 form: sites 4q..4q+3 of chain n from one Philox call.
__global__ void k_dense_momenta(float *__restrict__ p, int N, int n_chains, int b_pad,
                                uint64_t seed, uint32_t traj) {
    const int64_t nq = (int64_t)b_pad * (N / 4);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nq;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int n = (int)(i / (N / 4));
        const int q = (int)(i % (N / 4));
        float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        if (n < n_chains) z = momenta4_f32((uint32_t)q, traj, (uint32_t)n, seed);
        reinterpret_cast<float4 *>(p)[i] = z;
    }
}

// ------------------------------------------- FP64-accurate G = J Psi^T on FP32
// Double-float GEMM: J = Jhi + Jlo (two FP32), psi exact in FP32; every product
// Jhi*psi is split exactly by an FMA, Jlo*psi is added to the error word, and
// the running sum is kept as a TwoSum pair.  Tile 64 sites x 64 chains, 256
// threads with 4 x 4 outputs each, K slabs of 16 in shared memory.
constexpr int DG_T = 64, DG_K = 16;

__global__ void __launch_bounds__(256) k_df_gemm(const float *__restrict__ Jhi,
                                                 const float *__restrict__ Jlo,
                                                 const float *__restrict__ psi, float *__restrict__ Ghi,
                                                 float *__restrict__ Glo, int N) {
    __shared__ float sJh[DG_K][DG_T + 4], sJl[DG_K][DG_T + 4], sP[DG_K][DG_T + 4];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int m0 = blockIdx.x * DG_T, n0 = blockIdx.y * DG_T;
    float s[4][4], c[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) s[i][j] = c[i][j] = 0.0f;
    for (int k0 = 0; k0 < N; k0 += DG_K) {
        // 64 rows x 16 k of each operand: 1024 values, 4 per thread
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int e = threadIdx.x + r * 256;
            const int row = e >> 4, kk = e & 15;
            sJh[kk][row] = Jhi[(int64_t)(m0 + row) * N + k0 + kk];
            sJl[kk][row] = Jlo[(int64_t)(m0 + row) * N + k0 + kk];
            sP[kk][row] = psi[(int64_t)(n0 + row) * N + k0 + kk];
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < DG_K; ++kk) {
            float ah[4], al[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                ah[i] = sJh[kk][ty * 4 + i];
                al[i] = sJl[kk][ty * 4 + i];
                b[i] = sP[kk][tx * 4 + i];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float p = __fmul_rn(ah[i], b[j]);
                    float e = __fmaf_rn(ah[i], b[j], -p);
                    e = __fmaf_rn(al[i], b[j], e);
                    const f2 t = two_sum(s[i][j], p);
                    s[i][j] = t.hi;
                    c[i][j] = __fadd_rn(c[i][j], __fadd_rn(t.lo, e));
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const f2 r = fast_two_sum(s[i][j], c[i][j]);
            const int64_t idx = (int64_t)(n0 + tx * 4 + j) * N + (m0 + ty * 4 + i);
            Ghi[idx] = r.hi;
            Glo[idx] = r.lo;
        }
}

// ----------------------------------------- per-chain action, dH, Metropolis
// mode 0: end of a trajectory (psi_w = proposal, p = end momenta, K0 from the
// regenerated momenta, Metropolis test, copy to psi_cur on accept);
// mode 1: evaluate S and the estimators of psi_cur (G computed from psi_cur);
// mode 2: global sign flip (Sec. 3): S and the estimators of -psi_cur (G
// computed from psi_cur, so A(-psi) = -A psi), the flip's Metropolis test
// against S(psi_cur), psi_cur negated on acceptance.
// Modes 0 and 2 add the measurement of the trajectory when `measure` is set
// (a flip trajectory measures after the flip, in mode 2).
__global__ void __launch_bounds__(256, 4) k_dense_finalize(DenseArgs d, int mode, uint32_t traj,
                                                        uint64_t seed, int measure) {
    __shared__ float4 tab[LOG1PEXP_NODES];
    __shared__ double red[32 * 8];
    __shared__ int bcast;
    const int n = blockIdx.x;
    if (n >= d.n_chains) return;
    for (int i = threadIdx.x; i < LOG1PEXP_NODES; i += blockDim.x) tab[i] = d.lpe_tab[i];
    __syncthreads();
    const ChainParams pr = d.params[n];
    ChainState *st = d.state + n;
    const float *psi = (mode == 0 ? d.psi : d.psi_cur) + (int64_t)n * d.N;
    const f2 beta2 = df_from_double(pr.beta), C2 = df_from_double(pr.C), hp2 = df_from_double(pr.hp);
    f2 S{0.f, 0.f}, K0{0.f, 0.f}, K1{0.f, 0.f};
    float Slo = 0.f, K0lo = 0.f, K1lo = 0.f;
    float sT = 0.f, cT = 0.f, sAT = 0.f, cAT = 0.f, sHT = 0.f, cHT = 0.f;
    int sS = 0;
    const uint32_t spin_traj = mode == 1 ? TRAJ_INIT : traj;
    const uint64_t spin_seed = mode == 1 ? 0 : seed;
    const float sg = mode == 2 ? -1.0f : 1.0f;   // the configuration is sg * psi
    for (int q = threadIdx.x; q < d.N / 4; q += blockDim.x) {
        const float4 su = spin_u4_f32((uint32_t)q, spin_traj, (uint32_t)n, spin_seed);
        const float suv[4] = {su.x, su.y, su.z, su.w};
        float4 p0 = make_float4(0.f, 0.f, 0.f, 0.f);
        if (mode == 0) p0 = momenta4_f32((uint32_t)q, traj, (uint32_t)n, seed);
        const float p0v[4] = {p0.x, p0.y, p0.z, p0.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int m = 4 * q + k;
            const int64_t idx = (int64_t)n * d.N + m;
            const float ps = sg * psi[m];
            f2 G;
            if (d.action_tc) {   // exact integer digit sum -> double-float (48 bits)
                const long long gi = d.Gint[idx];
                const float ghi = __ll2float_rn(gi);
                const float glo = __ll2float_rn(gi - __float2ll_rn(ghi));
                const int sh = d.row_exp[m] + d.chain_exp[n] - ACT_BITS * (ACT_DIGITS + 1);
                G = f2{ldexpf(ghi, sh), ldexpf(glo, sh)};
            } else {
                G = f2{d.Ghi[idx], d.Glo[idx]};
            }
            if (mode == 2) G = df_neg(G);
            const f2 a = df_add(df_mul(beta2, G), df_mul_f(C2, ps));
            f2 x = a;
            float hq = pr.hpf;
            if (d.hdf) {
                const f2 hp = df_mul(beta2, f2{d.hdf[m].x, d.hdf[m].y});
                x = df_add(a, hp);
                hq = hp.hi;
            } else if (pr.hp != 0.0) {
                x = df_add(a, hp2);
            }
            const f2 ax = x.hi < 0.0f ? df_neg(x) : x;
            const f2 gl = log1pexp_neg(f2{2.0f * ax.hi, 2.0f * ax.lo}, tab);
            acc_add(S, Slo, df_mul_f(a, 0.5f * ps));
            acc_add(S, Slo, df_neg(ax));
            acc_add(S, Slo, df_neg(gl));
            const float t = tanh_f(x.hi);
            kahan_add(sT, cT, t);
            kahan_add(sAT, cAT, a.hi * t);
            kahan_add(sHT, cHT, hq * t);
            sS += (suv[k] < (1.0f + t) * 0.5f) ? 1 : -1;
            if (mode == 0) {
                const float p1 = d.p[idx];
                acc_add(K1, K1lo, two_prod(p1, 0.5f * p1));
                acc_add(K0, K0lo, two_prod(p0v[k], 0.5f * p0v[k]));
            }
        }
    }
    double v[8] = {acc_val(K0, K0lo), acc_val(K1, K1lo), acc_val(S, Slo), kahan_val(sT, cT),
                   kahan_val(sAT, cAT), kahan_val(sHT, cHT), (double)sS, 0.0};
    block_sum<8>(v, red);
    const double invN = 1.0 / (double)d.N;
    if (threadIdx.x == 0) {
        auto set_obs = [&]() {
            const double m = v[3] * invN;
            st->obs[0] = m;
            st->obs[1] = 0.5 * pr.C - 0.5 * v[4] * invN - v[5] * invN;
            st->obs[2] = fabs(v[6]) * invN;
            st->obs[3] = fabs(m);
        };
        auto add_measurement = [&]() {
            const double dH = st->rec[ISING_REC_DH];
            double *sm = st->sums;
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
        };
        if (mode == 1) {
            st->S = v[2];
            set_obs();
            bcast = 0;
        } else if (mode == 2) {
            const double lu = accept_logu(traj, (uint32_t)n, seed, PURPOSE_FLIP);
            const bool fl = lu < -(v[2] - st->S);
            if (fl) {
                st->S = v[2];
                set_obs();
                st->rec[ISING_REC_FLIPPED] = 1.0;
            }
            if (measure) add_measurement();
            bcast = fl ? 1 : 0;
        } else {
            const double S0 = st->S;
            const double dH = (v[1] + v[2]) - (v[0] + S0);
            const double logu = accept_logu(traj, (uint32_t)n, seed, PURPOSE_ACC);
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
                set_obs();
            }
            if (measure) add_measurement();
            bcast = acc ? 1 : 0;
        }
    }
    __syncthreads();
    if (bcast) {
        // mode 0: the proposal becomes current; mode 2: psi_cur = -psi_cur
        float *dst = d.psi_cur + (int64_t)n * d.N;
        for (int m = threadIdx.x; m < d.N; m += blockDim.x) dst[m] = sg * psi[m];
    }
}

// CTA-pair tiles (256 x 256) where both GEMM output dimensions allow them,
// else single-CTA 128 x 128 tiles.
#ifndef IHMC_NO_PAIR
static bool use_pair(int M, int N) { return M % 256 == 0 && N % 256 == 0; }
#else
static bool use_pair(int, int) { return false; }
#endif

// ------------------------------------------------- set-up of the dense form
// y = J x in FP64 (Lanczos estimate of lambda_min at creation), one warp per row.
__global__ void k_matvec_f64(const double *__restrict__ J, const double *__restrict__ x,
                             double *__restrict__ y, int64_t N) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = warp; r < N; r += nwarps) {
        const double *row = J + r * N;
        double acc = 0.0;
        for (int64_t j = lane; j < N; j += 32) acc = fma(row[j], x[j], acc);
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if (lane == 0) y[r] = acc;
    }
}

__device__ __forceinline__ uint16_t bf16_bits(float f) {
    return __bfloat16_as_ushort(__float2bfloat16_rn(f));
}

// Per row i of the FP64 couplings (one CTA): the BF16 copy (round to nearest
// even of the FP32 value) and either the ACT_DIGITS base-128 digit planes of
// J_i. 2^-e_i, e_i = ilogb(max_j |J_ij|) + 2 (so every entry lies in
// (-1/2, 1/2)), from X = round(J_ij 2^(42 - e_i)) taken from the FP64 bit
// pattern with integer arithmetic, or the double-float pair (N > 4096).
__global__ void __launch_bounds__(256) k_dense_prepare(const double *__restrict__ J, int64_t N,
                                                       uint16_t *__restrict__ J16,
                                                       uint16_t *__restrict__ dig,
                                                       int *__restrict__ row_exp,
                                                       float *__restrict__ Jhi,
                                                       float *__restrict__ Jlo,
                                                       uint8_t *__restrict__ J8,
                                                       float *__restrict__ sJ8) {
    __shared__ double red[8];
    const int64_t i = blockIdx.x;
    const double *row = J + i * N;
    double mx = 0.0;
    for (int64_t j = threadIdx.x; j < N; j += blockDim.x) mx = fmax(mx, fabs(row[j]));
    for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    mx = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mx = fmax(mx, red[w]);
    const int e = mx > 0.0 ? ilogb(mx) + 2 : 0;
    if (threadIdx.x == 0 && row_exp) row_exp[i] = e;
    // FP8 row scale: the row's largest |J| maps to 448, the largest E4M3 value
    const float s8 = mx > 0.0 ? (float)(mx / 448.0) : 1.0f;
    if (threadIdx.x == 0 && sJ8) sJ8[i] = s8;
    constexpr int FRAC = ACT_BITS * ACT_DIGITS;   // 42 fraction bits
    const int64_t nn = N * N;
    for (int64_t j = threadIdx.x; j < N; j += blockDim.x) {
        const double x = row[j];
        if (J16) J16[i * N + j] = bf16_bits((float)x);
        if (J8)
            J8[i * N + j] = (uint8_t)__nv_cvt_float_to_fp8((float)x / s8, __NV_SATFINITE, __NV_E4M3);
        if (dig) {
            const unsigned long long b = (unsigned long long)__double_as_longlong(x);
            const int be = (int)((b >> 52) & 0x7FF);
            long long X = 0;
            if (be) {   // normal (subnormals lie far below the last digit)
                const long long M = (long long)((b & 0xFFFFFFFFFFFFFull) | (1ull << 52));
                const int sh = be - 1075 - e + FRAC;   // x 2^(FRAC-e) = M 2^sh, sh < -11
                if (sh > -63) X = (M + (1ll << (-sh - 1))) >> (-sh);
                if (b >> 63) X = -X;
            }
            // low digits in [-64, 63]; the top digit takes the rest, |rest| <= 64
#pragma unroll
            for (int t = ACT_DIGITS - 1; t >= 1; --t) {
                const int q = (int)(((X + 64) & 127) - 64);
                X = (X - q) >> ACT_BITS;
                dig[(int64_t)t * nn + i * N + j] = bf16_bits((float)q);
            }
            dig[i * N + j] = bf16_bits((float)(int)X);
        }
        if (Jhi) {
            const float hi = (float)x;
            Jhi[i * N + j] = hi;
            Jlo[i * N + j] = (float)(x - (double)hi);
        }
    }
}

// Cluster of cn CTAs; with pdl, programmatic dependent launch (the kernel
// waits on the previous grid itself, after its set-up).
static cudaLaunchConfig_t cluster_config(cudaLaunchAttribute *at, int cn, int grid, cudaStream_t s,
                                         bool pdl = false) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(tc::THREADS);
    cfg.dynamicSmemBytes = tc::SMEM_BYTES;
    cfg.stream = s;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)cn;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 2 : 1;
    return cfg;
}

// How many clusters of cn CTAs of kern fit on the GPU at once (one CTA per SM).
template <class K>
cudaError_t max_clusters(K kern, int cn, int *out) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         tc::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute at[2];
    cudaLaunchConfig_t cfg = cluster_config(at, cn, cn, 0);
    e = cudaOccupancyMaxActiveClusters(out, kern, &cfg);
    if (e == cudaSuccess && *out < 1) e = cudaErrorInvalidConfiguration;
    return e;
}

#ifndef IHMC_PDL
#define IHMC_PDL true
#endif
// Persistent launch in clusters of cn CTAs: as many clusters as fit at once
// (nclu), at most one per tile.
template <class... KArgs, class... Args>
cudaError_t launch_gemm(void (*kern)(KArgs...), int cn, int nclu, int units, cudaStream_t s,
                        Args... args) {
    cudaLaunchAttribute at[2];
    cudaLaunchConfig_t cfg = cluster_config(at, cn, (units < nclu ? units : nclu) * cn, s, IHMC_PDL);
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

}  // namespace

// Tensor map of a row-major BF16 matrix (rows x cols, cols contiguous) read in
// boxes of box_rows x 64 with 128-byte swizzling.
cudaError_t make_tmap_2d(CUtensorMap *map, const void *base, int64_t rows, int64_t cols,
                         int box_rows, int elem_bytes) {
    // the driver entry point is looked up through the runtime, so the library
    // does not link the driver library itself
    using encode_fn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                   const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                   const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static encode_fn encode = nullptr;
    if (!encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                         cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
        encode = reinterpret_cast<encode_fn>(fn);
    }
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)cols * (cuuint64_t)elem_bytes};
    const cuuint32_t box[2] = {(cuuint32_t)(128 / elem_bytes), (cuuint32_t)box_rows};   // 128-byte rows
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = encode(map, elem_bytes == 1 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                        2, const_cast<void *>(base), dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <bool PAIR>
static cudaError_t gemm_store_mode(const CUtensorMap &ta, const CUtensorMap &tb, float *D, int M,
                                   int N, int K, int *err, cudaStream_t s) {
    using Md = tc::Mode<PAIR>;
    const int cs = PAIR ? 2 : 1;
    int nclu = 0;
    cudaError_t e = max_clusters(gemm_store_kernel<PAIR>, cs, &nclu);
    if (e != cudaSuccess) return e;
    return launch_gemm(gemm_store_kernel<PAIR>, cs, nclu, (M / Md::TILE_M) * (N / Md::TILE_N), s,
                       ta, tb, D, M, N, K, err);
}

cudaError_t launch_gemm_store(const void *A, const void *B, float *D, int M, int N, int K, int *err,
                              cudaStream_t s) {
    CUtensorMap ta, tb;
    cudaError_t e = make_tmap_2d(&ta, A, M, K, tc::BM, 2);
    if (e == cudaSuccess) e = make_tmap_2d(&tb, B, N, K, tc::BR, 2);
    if (e != cudaSuccess) return e;
    return use_pair(M, N) ? gemm_store_mode<true>(ta, tb, D, M, N, K, err, s)
                          : gemm_store_mode<false>(ta, tb, D, M, N, K, err, s);
}

template <bool PAIR>
static cudaError_t force_clusters(int *nclu) {
    const int cs = PAIR ? 2 : 1;
    int a = 0, b = 0, c = 0, a8 = 0, b8 = 0;
    cudaError_t e = max_clusters(force1_kernel<PAIR, false>, cs, &a);
    if (e == cudaSuccess) e = max_clusters(force2_kernel<PAIR, false>, cs, &b);
    if (e == cudaSuccess) e = max_clusters(force1_kernel<PAIR, true>, cs, &a8);
    if (e == cudaSuccess) e = max_clusters(force2_kernel<PAIR, true>, cs, &b8);
    if (e == cudaSuccess) e = max_clusters(action_kernel<PAIR>, cs, &c);
    int m = a;
    for (int x : {b, c, a8, b8}) m = x < m ? x : m;
    *nclu = m;
    return e;
}

cudaError_t dense_setup(DenseArgs &d) {
    d.pair = use_pair(d.N, d.b_pad) ? 1 : 0;
    cudaError_t e = d.pair ? force_clusters<true>(&d.nclu) : force_clusters<false>(&d.nclu);
    const int eb = d.fp8 ? 1 : 2;
    if (e == cudaSuccess)
        e = make_tmap_2d(&d.tm_J, d.fp8 ? (const void *)d.J8 : (const void *)d.J16, d.N, d.N, tc::BM, eb);
    if (e == cudaSuccess)
        e = make_tmap_2d(&d.tm_psi, d.fp8 ? (const void *)d.psi8 : (const void *)d.psi16, d.b_pad,
                         d.N, tc::BR, eb);
    if (e == cudaSuccess)
        e = make_tmap_2d(&d.tm_u, d.fp8 ? (const void *)d.u8 : (const void *)d.u16, d.b_pad, d.N,
                         tc::BR, eb);
    if (e == cudaSuccess && d.action_tc) {
        e = make_tmap_2d(&d.tm_Jdig, d.Jdig, (int64_t)ACT_DIGITS * d.N, d.N, tc::BM, 2);
        if (e == cudaSuccess)
            e = make_tmap_2d(&d.tm_psidig, d.psidig, (int64_t)ACT_DIGITS * d.b_pad, d.N, tc::BR, 2);
    }
    return e;
}

// G = J psi to FP64 accuracy for the chains' psi (proposal or current).
static cudaError_t launch_action_product(DenseArgs &d, const float *psi, cudaStream_t s,
                                         int64_t *n) {
    if (!d.action_tc) {
        k_df_gemm<<<dim3(d.N / DG_T, d.b_pad / DG_T), 256, 0, s>>>(d.Jhi, d.Jlo, psi, d.Ghi, d.Glo,
                                                                  d.N);
        ++*n;
        return cudaGetLastError();
    }
    k_psi_digits<<<d.b_pad, 256, 0, s>>>(psi, d.psidig, d.chain_exp, d.N, d.n_chains, d.b_pad);
    ++*n;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    ++*n;
    if (d.pair)
        return launch_gemm(action_kernel<true>, 2, d.nclu, (d.N / 256) * (d.b_pad / 256), s,
                           d.tm_Jdig, d.tm_psidig, d);
    return launch_gemm(action_kernel<false>, 1, d.nclu, (d.N / 128) * (d.b_pad / 128), s, d.tm_Jdig,
                       d.tm_psidig, d);
}

// G = J Psi^T with the pass-1 epilogue (u), then G = J U^T with the pass-2
// epilogue (kick, drift).
template <bool PAIR, bool FP8>
static cudaError_t launch_force_t(const DenseArgs &d, int pass, float kick, float drift,
                                  int do_drift, cudaStream_t s) {
    const int t = PAIR ? 256 : 128;
    const int units = (d.N / t) * (d.b_pad / t);
    const int cs = PAIR ? 2 : 1;
    return pass == 0 ? launch_gemm(force1_kernel<PAIR, FP8>, cs, d.nclu, units, s, d.tm_J, d.tm_psi, d)
                     : launch_gemm(force2_kernel<PAIR, FP8>, cs, d.nclu, units, s, d.tm_J, d.tm_u, d,
                                   kick, drift, do_drift);
}

static cudaError_t launch_force(const DenseArgs &d, int pass, float kick, float drift, int do_drift,
                                cudaStream_t s) {
    if (d.pair)
        return d.fp8 ? launch_force_t<true, true>(d, pass, kick, drift, do_drift, s)
                     : launch_force_t<true, false>(d, pass, kick, drift, do_drift, s);
    return d.fp8 ? launch_force_t<false, true>(d, pass, kick, drift, do_drift, s)
                 : launch_force_t<false, false>(d, pass, kick, drift, do_drift, s);
}

static int grid_elems(int64_t n) {
    int64_t b = (n + 255) / 256;
    return (int)(b > 4096 ? 4096 : (b < 1 ? 1 : b));
}

cudaError_t dense_trajectory(DenseArgs &d, const Schedule &sched, uint64_t seed, uint32_t traj,
                             int measure, int flip, cudaStream_t s, int64_t *launches) {
    const int64_t nel = (int64_t)d.b_pad * d.N;
    int64_t n = 0;
    k_copy_state<<<grid_elems(nel), 256, 0, s>>>(d.psi_cur, d.psi, d.fp8 ? nullptr : d.psi16,
                                                  d.fp8 ? d.psi8 : nullptr, nel);
    ++n;
    k_dense_momenta<<<grid_elems(nel / 4), 256, 0, s>>>(d.p, d.N, d.n_chains, d.b_pad, seed, traj); ++n;
    for (int j = 0; j < sched.n_pass; ++j) {
        cudaError_t e = launch_force(d, 0, 0.f, 0.f, 0, s); ++n;
        const bool drift = j + 1 < sched.n_pass;
        if (e == cudaSuccess)
            e = launch_force(d, 1, (float)sched.kick[j], (float)sched.drift[j], drift ? 1 : 0, s);
        ++n;
        if (e != cudaSuccess) {
            *launches += n;
            return e;
        }
    }
    cudaError_t e = launch_action_product(d, d.psi, s, &n);
    if (e != cudaSuccess) {
        *launches += n;
        return e;
    }
    k_dense_finalize<<<d.n_chains, 256, 0, s>>>(d, 0, traj, seed, flip ? 0 : measure); ++n;
    if (flip) {
        // sign-flip proposal of the current configuration: its A psi first
        e = cudaGetLastError();
        if (e == cudaSuccess) e = launch_action_product(d, d.psi_cur, s, &n);
        if (e != cudaSuccess) {
            *launches += n;
            return e;
        }
        k_dense_finalize<<<d.n_chains, 256, 0, s>>>(d, 2, traj, seed, measure); ++n;
    }
    *launches += n;
    return cudaGetLastError();
}

cudaError_t dense_eval(DenseArgs &d, cudaStream_t s, int64_t *launches) {
    int64_t n = 0;
    cudaError_t e = launch_action_product(d, d.psi_cur, s, &n);
    if (e == cudaSuccess) {
        k_dense_finalize<<<d.n_chains, 256, 0, s>>>(d, 1, 0, 0, 0);
        ++n;
        e = cudaGetLastError();
    }
    *launches += n;
    return e;
}

cudaError_t dense_momenta(DenseArgs &d, uint64_t seed, uint32_t traj, cudaStream_t s,
                          int64_t *launches) {
    const int64_t nel = (int64_t)d.b_pad * d.N;
    k_dense_momenta<<<grid_elems(nel / 4), 256, 0, s>>>(d.p, d.N, d.n_chains, d.b_pad, seed, traj);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t dense_matvec_f64(const double *J, const double *x, double *y, int64_t N,
                             cudaStream_t s) {
    const int64_t blocks = (N + 7) / 8;   // 8 warps (rows) per block
    k_matvec_f64<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(J, x, y, N);
    return cudaGetLastError();
}

cudaError_t dense_prepare(const double *J, int64_t N, uint16_t *J16, uint16_t *dig, int *row_exp,
                          float *Jhi, float *Jlo, uint8_t *J8, float *sJ8, cudaStream_t s) {
    k_dense_prepare<<<(unsigned)N, 256, 0, s>>>(J, N, J16, dig, row_exp, Jhi, Jlo, J8, sJ8);
    return cudaGetLastError();
}

// One force evaluation of the dense path alone (two GEMMs with epilogues), for
// timing the tensor-core kernels.
cudaError_t dense_force_once(DenseArgs &d, cudaStream_t s) {
    cudaError_t e = launch_force(d, 0, 0.f, 0.f, 0, s);
    return e == cudaSuccess ? launch_force(d, 1, 0.f, 0.f, 0, s) : e;
}

}  // namespace ihmc
