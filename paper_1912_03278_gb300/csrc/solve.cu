// solve.cu -- A x = b for one chain's A = beta*J*K + C*1 (Sec. 2) by conjugate
// gradients (Hestenes and Stiefel 1952) in FP64 on the device.  It serves the
// paper's own parametrisation: its field is psi_p = sqrt(J') (psi + A^-1 h')
// and its observables carry the constant h'^T Kt^-1 h' = J' h'^T A^-1 h'
// (Kt = K + C_p*1 = A / J'), both of which need A^-1 h' when h varies from
// site to site.
//
// A set-up computation, not a hot path: one CTA runs the whole iteration, so
// every product with A and every dot product is a CTA-wide loop with barriers
// between the dependent steps and no inter-CTA synchronisation; the CTA-wide
// sums are taken in a fixed order, so the result is deterministic.  The
// iteration count is bounded by max_iter.
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "internal.h"

namespace ihmc {
namespace {

constexpr int SOLVE_THREADS = 1024;

struct SolveArgs {
    const double *J;   // dense couplings (N x N, row-major) or null
    const double *b;
    double *x, *r, *d, *Ad;
    int64_t N;
    int kind, dim, X, Y, Z;
    double bJ, C;   // beta*J (lattice), kappa = beta*J/N (infinite range) or beta (dense);
                    // the shift
    double tol;
    int max_iter;
    int *iters;     // out: iterations taken (max_iter if the tolerance was not reached)
    double *resid;  // out: ||b - A x|| / ||b|| of the recursive residual
};

// CTA-wide dot product u.v, identical in every thread.
__device__ double dot(const double *u, const double *v, int64_t N, double *red) {
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) s = fma(u[i], v[i], s);
    double w[1] = {s};
    block_sum<1>(w, red);
    return w[0];
}

// out = A v.  Lattice: periodic nearest neighbours; infinite range: every
// other site with weight kappa; dense: beta J v, one warp per row (lanes
// stride the row, then a fixed-order shuffle sum).
__device__ void apply_A(const SolveArgs &a, const double *v, double *out, double *red) {
    const int64_t N = a.N;
    if (a.kind == ISING_KIND_DENSE) {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
        for (int64_t i = warp; i < N; i += nw) {
            const double *row = a.J + i * N;
            double s = 0.0;
            for (int64_t j = lane; j < N; j += 32) s = fma(row[j], v[j], s);
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) out[i] = a.C * v[i] + a.bJ * s;
        }
        return;
    }
    if (a.kind == ISING_KIND_INFINITE) {
        double s = 0.0;
        for (int64_t i = threadIdx.x; i < N; i += blockDim.x) s += v[i];
        double w[1] = {s};
        block_sum<1>(w, red);
        for (int64_t i = threadIdx.x; i < N; i += blockDim.x)
            out[i] = a.C * v[i] + a.bJ * (w[0] - v[i]);
        return;
    }
    const int64_t X = a.X, Y = a.Y, Z = a.Z, XY = X * Y;
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
        const int64_t x = i % X, y = (i / X) % Y, z = i / XY;
        double nb = v[x > 0 ? i - 1 : i + X - 1] + v[x + 1 < X ? i + 1 : i - (X - 1)];
        if (a.dim >= 2)
            nb += v[y > 0 ? i - X : i + (Y - 1) * X] + v[y + 1 < Y ? i + X : i - (Y - 1) * X];
        if (a.dim == 3)
            nb += v[z > 0 ? i - XY : i + (Z - 1) * XY] + v[z + 1 < Z ? i + XY : i - (Z - 1) * XY];
        out[i] = a.C * v[i] + a.bJ * nb;
    }
}

__global__ void __launch_bounds__(SOLVE_THREADS) cg_kernel(SolveArgs a) {
    __shared__ double red[32];
    const int64_t N = a.N;
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
        a.x[i] = 0.0;
        a.r[i] = a.b[i];
        a.d[i] = a.b[i];
    }
    __syncthreads();
    double rr = dot(a.r, a.r, N, red);
    const double bb = rr;
    int k = 0;
    for (; k < a.max_iter; ++k) {
        if (rr <= a.tol * a.tol * bb) break;
        apply_A(a, a.d, a.Ad, red);
        __syncthreads();
        const double alpha = rr / dot(a.d, a.Ad, N, red);
        for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
            a.x[i] = fma(alpha, a.d[i], a.x[i]);
            a.r[i] = fma(-alpha, a.Ad[i], a.r[i]);
        }
        __syncthreads();
        const double rr_new = dot(a.r, a.r, N, red);
        const double beta = rr_new / rr;
        for (int64_t i = threadIdx.x; i < N; i += blockDim.x) a.d[i] = fma(beta, a.d[i], a.r[i]);
        __syncthreads();
        rr = rr_new;
    }
    if (threadIdx.x == 0) {
        *a.iters = k;
        *a.resid = bb > 0 ? sqrt(rr / bb) : 0.0;
    }
}

}  // namespace

cudaError_t solve_A(const double *b_dev, double *x_dev, double *work /* 3N */, int64_t N, int kind,
                    int dim, const int L[3], double bJ, double C, double tol, int max_iter,
                    int *iters_dev, double *resid_dev, cudaStream_t s, const double *J) {
    SolveArgs a{};
    a.J = J;
    a.b = b_dev;
    a.x = x_dev;
    a.r = work;
    a.d = work + N;
    a.Ad = work + 2 * N;
    a.N = N;
    a.kind = kind;
    a.dim = dim;
    a.X = L[0];
    a.Y = L[1];
    a.Z = L[2];
    a.bJ = bJ;
    a.C = C;
    a.tol = tol;
    a.max_iter = max_iter;
    a.iters = iters_dev;
    a.resid = resid_dev;
    cg_kernel<<<1, SOLVE_THREADS, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace ihmc
