// noalloc.cu -- the plain FP64 form's energy arithmetic in kernels that
// allocate no memory: S(psi) and 1/2 p.p of periodic-lattice configurations, with the
// per-block partial sums in a fixed, file-scope device array instead of a
// buffer allocated by a simulation handle.  For callers that cannot call
// cudaMalloc (see ising_hmc_energy_noalloc in ising_hmc.h).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "device_common.cuh"
#include "internal.h"

namespace ihmc {
namespace {

constexpr int NOALLOC_BLOCKS = 256;   // partial-sum blocks per configuration
constexpr int NOALLOC_THREADS = 256;

// Scratch shared by every call: two partial sums (S, K) per block and
// configuration.  Every slot a call reads is written by the same call first,
// so nothing needs clearing between calls.
static __device__ __align__(256) double g_energy_scratch[ISING_NOALLOC_MAX_CHAINS * NOALLOC_BLOCKS * 2];

struct LatticeParams {
    Geometry g;
    double bJ, C, hp;
};

__device__ __forceinline__ int64_t nbr_index(const Geometry &g, int64_t i, int which) {
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

// Per block: sum over its sites of 1/2 psi_i a_i - log 2cosh(a_i + h') with
// a = A psi computed on the fly, and of 1/2 p_i^2 (Sec. 3, HMC Hamiltonian).
__global__ void k_energy_partials(const double *__restrict__ psi, const double *__restrict__ p,
                                  LatticeParams lp, double *scratch) {
    __shared__ double red[32 * 2];
    const int c = blockIdx.y;
    const Geometry &g = lp.g;
    const double *x = psi + (int64_t)c * g.N;
    const double *pc = p ? p + (int64_t)c * g.N : nullptr;
    const int nn = 2 * g.dim;
    double v[2] = {0.0, 0.0};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.N;
         i += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int k = 0; k < nn; ++k) s += x[nbr_index(g, i, k)];
        const double a = lp.bJ * s + lp.C * x[i];
        v[0] += 0.5 * x[i] * a - log2cosh_f64(a + lp.hp);
        if (pc) v[1] += 0.5 * pc[i] * pc[i];
    }
    block_sum<2>(v, red);
    if (threadIdx.x == 0) {
        double *slot = scratch + ((int64_t)c * gridDim.x + blockIdx.x) * 2;
        slot[0] = v[0];
        slot[1] = v[1];
    }
}

// Per configuration: the block partials added in block order.
__global__ void k_energy_finalize(const double *scratch, int nblocks, double *out) {
    const int c = blockIdx.x;
    if (threadIdx.x != 0) return;
    double S = 0.0, K = 0.0;
    for (int b = 0; b < nblocks; ++b) {
        S += scratch[((int64_t)c * nblocks + b) * 2];
        K += scratch[((int64_t)c * nblocks + b) * 2 + 1];
    }
    out[2 * c] = S;
    out[2 * c + 1] = K;
}

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
double *g_scratch_addr[MAX_DEVICES] = {nullptr};
thread_local char g_noalloc_err[256];

ising_status err(ising_status st, const char *msg, const char *detail = "") {
    std::snprintf(g_noalloc_err, sizeof g_noalloc_err, "%s%s", msg, detail);
    return st;
}

}  // namespace

const char *noalloc_last_error() { return g_noalloc_err; }

}  // namespace ihmc

using namespace ihmc;

extern "C" ising_status ising_hmc_energy_noalloc(int dim, const int L[3], double beta, double Jnn,
                                                 double C, double h0, int n_chains,
                                                 const double *psi, const double *p, double *out,
                                                 void *stream) {
    g_noalloc_err[0] = 0;
    if (!L || !psi || !out) return err(ISING_EINVAL, "energy_noalloc: null L, psi or out");
    if (dim < 1 || dim > 3) return err(ISING_EINVAL, "energy_noalloc: dim must be 1..3");
    if (n_chains < 1 || n_chains > ISING_NOALLOC_MAX_CHAINS)
        return err(ISING_EINVAL, "energy_noalloc: n_chains must be 1..ISING_NOALLOC_MAX_CHAINS (64)");
    Geometry g{};
    g.dim = dim;
    g.X = L[0];
    g.Y = dim > 1 ? L[1] : 1;
    g.Z = dim > 2 ? L[2] : 1;
    int64_t N = 1;
    for (int d = 0; d < dim; ++d) {
        if (L[d] < 3) return err(ISING_EINVAL, "energy_noalloc: each lattice extent must be >= 3");
        N *= L[d];
    }
    if (N > ((int64_t)1 << 31)) return err(ISING_EINVAL, "energy_noalloc: too many sites");
    g.N = N;
    // an error pending from earlier work belongs to the caller: leave it in
    // place and do not launch, so the status below is this call's own
    const cudaError_t pending = cudaPeekAtLastError();
    if (pending != cudaSuccess)
        return err(ISING_ECUDA, "energy_noalloc: a CUDA error from earlier work is pending: ",
                   cudaGetErrorString(pending));
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES)
        return err(ISING_ECUDA, "energy_noalloc: no usable CUDA device");
    double *scratch;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_scratch_addr[dev]) {
            void *ptr = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&ptr, g_energy_scratch);
            if (e != cudaSuccess)
                return err(ISING_ECUDA, "energy_noalloc: cudaGetSymbolAddress failed: ",
                           cudaGetErrorString(e));
            g_scratch_addr[dev] = static_cast<double *>(ptr);
        }
        scratch = g_scratch_addr[dev];
    }
    LatticeParams lp{g, beta * Jnn, C, beta * h0};
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    k_energy_partials<<<dim3(NOALLOC_BLOCKS, n_chains), NOALLOC_THREADS, 0, s>>>(psi, p, lp, scratch);
    k_energy_finalize<<<n_chains, 32, 0, s>>>(scratch, NOALLOC_BLOCKS, out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return err(ISING_ECUDA, "energy_noalloc: launch failed: ", cudaGetErrorString(e));
    return ISING_OK;
}

extern "C" const char *ising_hmc_energy_noalloc_error(void) { return g_noalloc_err; }
