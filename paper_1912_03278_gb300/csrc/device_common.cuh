// device_common.cuh -- device helpers shared by the kernels of the GB300
// HS-field HMC library: counter-based random numbers, Box-Muller, and
// deterministic block reductions.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ihmc {

// Philox purposes (fourth counter word).
enum : uint32_t { PURPOSE_MOM = 1, PURPOSE_ACC = 2, PURPOSE_SPIN = 3, PURPOSE_FLIP = 4 };

// Trajectory index used for the measurement of a configuration set from outside.
constexpr uint32_t TRAJ_INIT = 0xffffffffu;

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of
//   (x0,x1,x2,x3) -> (hi(M1*x2)^x1^k0, lo(M1*x2), hi(M0*x0)^x3^k1, lo(M0*x0))
// with the key advanced by the Weyl increments (W0, W1) after every round.
// Counter = (index, trajectory, chain, purpose); key = (seed lo, seed hi).
struct u32x4 { uint32_t x, y, z, w; };

__device__ __forceinline__ u32x4 philox(uint32_t idx, uint32_t traj, uint32_t chain,
                                        uint32_t purpose, uint64_t seed) {
    uint32_t c0 = idx, c1 = traj, c2 = chain, c3 = purpose;
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c0;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0;
        const uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return u32x4{c0, c1, c2, c3};
}

// Uniform in (0,1): ((x >> 9) + 1/2) * 2^-23, exact in FP32.
__device__ __forceinline__ float u23(uint32_t x) {
    return ((float)(x >> 9) + 0.5f) * 1.1920928955078125e-07f;
}
// Uniform in (0,1) from 52 bits: ((a >> 6) 2^26 + (b >> 6) + 1/2) 2^-52, exact in FP64.
__device__ __forceinline__ double u52(uint32_t a, uint32_t b) {
    return ((double)(a >> 6) * 67108864.0 + (double)(b >> 6) + 0.5) * 2.220446049250313e-16;
}

// Box-Muller (1958): r = sqrt(-2 ln u1), z0 = r cos(2 pi u2), z1 = r sin(2 pi u2).
// FP32 form: the angle 2 pi u2 - pi lies in [-pi, pi), where the hardware
// sine and cosine are accurate to ~4e-7 absolute; cos(t + pi) = -cos t and
// sin(t + pi) = -sin t restore the angle 2 pi u2.
__device__ __forceinline__ void box_muller_f32(float u1, float u2, float &z0, float &z1) {
    const float r = sqrtf(-2.0f * logf(u1));
    const float th = fmaf(6.2831853071795865f, u2, -3.1415926535897932f);
    float s, c;
    __sincosf(th, &s, &c);
    z0 = -r * c;
    z1 = -r * s;
}
__device__ __forceinline__ void box_muller_f64(double u1, double u2, double &z0, double &z1) {
    const double r = sqrt(-2.0 * log(u1));
    double s, c;
    sincospi(2.0 * u2, &s, &c);
    z0 = r * c;
    z1 = r * s;
}

// Four FP32 momenta for sites 4*q .. 4*q+3 of a chain (FP32 form).
__device__ __forceinline__ float4 momenta4_f32(uint32_t q, uint32_t traj, uint32_t chain,
                                               uint64_t seed) {
    const u32x4 x = philox(q, traj, chain, PURPOSE_MOM, seed);
    float4 z;
    box_muller_f32(u23(x.x), u23(x.y), z.x, z.y);
    box_muller_f32(u23(x.z), u23(x.w), z.z, z.w);
    return z;
}
// Four spin uniforms for sites 4*q .. 4*q+3 (FP32 form).
__device__ __forceinline__ float4 spin_u4_f32(uint32_t q, uint32_t traj, uint32_t chain,
                                              uint64_t seed) {
    const u32x4 x = philox(q, traj, chain, PURPOSE_SPIN, seed);
    return make_float4(u23(x.x), u23(x.y), u23(x.z), u23(x.w));
}
// Two FP64 momenta for sites 2*q, 2*q+1 (FP64 form).
__device__ __forceinline__ void momenta2_f64(uint32_t q, uint32_t traj, uint32_t chain,
                                             uint64_t seed, double &z0, double &z1) {
    const u32x4 x = philox(q, traj, chain, PURPOSE_MOM, seed);
    box_muller_f64(u52(x.x, x.y), u52(x.z, x.w), z0, z1);
}

__device__ __forceinline__ double accept_logu(uint32_t traj, uint32_t chain, uint64_t seed,
                                              uint32_t purpose) {
    const u32x4 x = philox(0, traj, chain, purpose, seed);
    return log(u52(x.x, x.y));
}

// tanh x = 1 - 2/(1 + e^{2x}) on |x| with the sign restored: e^{2|x|} from
// the hardware exp2, 1/(1+e) from the hardware reciprocal (1 ulp; a Newton
// step would lower the measured maximum error only from 1.7e-7 to 1.4e-7).
// Absolute error below 3e-7 for all x, odd to the bit (see the self-test).
__device__ __forceinline__ float tanh_f(float x) {
    const float ax = fminf(fabsf(x), 20.0f);
    float e, r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(ax * 2.8853900817779268f));  // 2 log2(e)
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(e + 1.0f));
    return copysignf(fmaf(-2.0f, r, 1.0f), x);
}

// log(2 cosh x) = |x| + log1p(exp(-2|x|)) in FP64.
__device__ __forceinline__ double log2cosh_f64(double x) {
    const double ax = fabs(x);
    return ax + log1p(exp(-2.0 * ax));
}

// Deterministic sum over the block of NV doubles per thread: xor-butterfly in
// each warp, then warp 0 adds the per-warp totals in warp order.  Result valid
// in every thread.  scratch: >= 32*NV doubles of shared memory.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double *scratch) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], off);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) scratch[warp * NV + k] = v[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double s = 0.0;
        for (int w = 0; w < nwarps; ++w) s += scratch[w * NV + k];
        v[k] = s;
    }
    __syncthreads();
}

}  // namespace ihmc
