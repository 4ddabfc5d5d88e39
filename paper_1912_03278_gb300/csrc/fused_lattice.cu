// fused_lattice.cu -- host side of the fused FP32 lattice kernel (launch
// shape, validity, launches, graph nodes) and the 1D instances; the kernel
// itself is in fused_lattice_impl.cuh, its 2D and 3D instances in
// fused_lattice_{2d,3d}{,_cl}.cu.
#include "fused_lattice_impl.cuh"

namespace ihmc {

cudaError_t fused_node_1d(const FusedArgs &a, int threads, int depth, int vec,
                          cudaKernelNodeParams *np, void **args) {
    return node_dim<1, false>(a, threads, depth, vec, np, args);
}

namespace {

// tanh self-test kernel
__global__ void tanh_selftest_kernel(const float *x, float *y, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        y[i] = tanh_f(x[i]);
}

__global__ void log1pexp_selftest_kernel(const double *y, double *out, int64_t n,
                                         const float4 *tab) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = df_to_double(log1pexp_neg(df_from_double(y[i]), tab));
}

}  // namespace

// Least shared memory a launch needs (the table read from global memory).
int fused_lattice_smem_bytes(const Geometry &g, int depth, int vec) {
    (void)vec;
    return (int)(ring_bytes(g.P, depth) + RED_BYTES);
}

// Launch shape: VEC = 4 when rows split into float4s; threads = one per vector
// up to 256, each thread owning at most NVMAX vectors per plane; prefetch
// depth 1 plane (with the force plane trailing, the resident CTAs cover the
// copy latency: the autotuner picks depth 1 for 2D L = 256 and 1024 as well).
// Returns VEC, or -1 if the plane does not fit on chip.
int fused_lattice_pick(const Geometry &g, int *threads, int *depth) {
    const int vec = (g.X % 4 == 0 && g.P % 4 == 0) ? 4 : 1;
    const int nvec = g.P / vec;
    int t = (nvec + 31) / 32 * 32;
    if (t > 256) t = 256;
    if (t < 32) t = 32;
    if ((nvec + t - 1) / t > NVMAX) return -1;
    *threads = t;
    if (fused_lattice_smem_bytes(g, 1, vec) > 227 * 1024) return -1;
    *depth = 1;
    return vec;
}

cudaError_t fused_lattice_node(const FusedArgs &a, int threads, int depth,
                               cudaKernelNodeParams *np, void **args) {
    const int vec = (a.g.X % 4 == 0 && a.g.P % 4 == 0) ? 4 : 1;
    const bool cl = a.cs > 1;
    if (a.g.dim == 3)
        return cl ? fused_node_3d_cl(a, threads, depth, vec, np, args)
                  : fused_node_3d(a, threads, depth, vec, np, args);
    if (a.g.dim == 2)
        return cl ? fused_node_2d_cl(a, threads, depth, vec, np, args)
                  : fused_node_2d(a, threads, depth, vec, np, args);
    if (cl) return cudaErrorInvalidValue;   // 1D chains have one plane: no split
    return fused_node_1d(a, threads, depth, vec, np, args);
}

static int valid_shape(const Geometry &g, int threads, int depth, int max_threads) {
    const int vec = (g.X % 4 == 0 && g.P % 4 == 0) ? 4 : 1;
    const int nvec = g.P / vec;
    if (threads < 32 || threads > max_threads || threads % 32) return 0;
    if ((nvec + threads - 1) / threads > NVMAX) return 0;
    if (depth != 1 && depth != 2 && depth != 4) return 0;
    return fused_lattice_smem_bytes(g, depth, vec) <= 227 * 1024;
}

int fused_lattice_valid_launch(const Geometry &g, int threads, int depth) {
    return valid_shape(g, threads, depth, MAX_THREADS_UNSPLIT);
}

// A chain split over cs CTAs: cs in {1, 2, 4, 8}, a 2D or 3D lattice with at
// least two planes per slab, up to 512 threads per CTA, and a cluster of cs
// such CTAs must fit on the device (asked of the occupancy calculator).
int fused_lattice_valid_split(const Geometry &g, int threads, int depth, int cs) {
    if (cs == 1) return fused_lattice_valid_launch(g, threads, depth);
    if (cs != 2 && cs != 4 && cs != MAX_CS) return 0;
    if (g.dim < 2 || g.nplanes < 2 * cs) return 0;
    if (!valid_shape(g, threads, depth, MAX_THREADS)) return 0;
    FusedArgs a{};
    a.g = g;
    a.n_chains = 1;
    a.cs = cs;
    Schedule sched{};
    cudaKernelNodeParams np;
    void *args[2] = {&a, &sched};
    if (fused_lattice_node(a, threads, depth, &np, args) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)cs, 1, 1);
    cfg.blockDim = np.blockDim;
    cfg.dynamicSmemBytes = np.sharedMemBytes;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    const cudaError_t e = cudaOccupancyMaxActiveClusters(&n, np.func, &cfg);
    cudaGetLastError();
    return e == cudaSuccess && n >= 1;
}

cudaError_t launch_fused_lattice(const FusedArgs &a, const Schedule &sched, int threads,
                                 int depth, cudaStream_t s) {
    cudaKernelNodeParams np;
    void *args[2] = {const_cast<FusedArgs *>(&a), const_cast<Schedule *>(&sched)};
    cudaError_t e = fused_lattice_node(a, threads, depth, &np, args);
    if (e != cudaSuccess) return e;
    if (np.gridDim.x == 0) return cudaSuccess;
    if (a.cs == 1)
        return cudaLaunchKernel(np.func, np.gridDim, np.blockDim, np.kernelParams,
                                np.sharedMemBytes, s);
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)a.cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = np.gridDim;
    cfg.blockDim = np.blockDim;
    cfg.dynamicSmemBytes = np.sharedMemBytes;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, np.func, np.kernelParams);
}

namespace {
// Copy by the SMs themselves: every thread moves 16-byte words with a grid
// stride, so a source in pinned host memory is read over the coherent
// CPU-GPU link by all SMs at once instead of by one copy engine.
__global__ void copy16_kernel(const uint4 *__restrict__ src, uint4 *__restrict__ dst, int64_t n) {
    // four independent 16-byte loads in flight per thread (the link's latency
    // is long); the ragged tail one word at a time
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (; i + 3 * stride < n; i += 4 * stride) {
        const uint4 a = src[i], b = src[i + stride], c = src[i + 2 * stride], d = src[i + 3 * stride];
        dst[i] = a;
        dst[i + stride] = b;
        dst[i + 2 * stride] = c;
        dst[i + 3 * stride] = d;
    }
    for (; i < n; i += stride) dst[i] = src[i];
}

__global__ void reset_chain_start_kernel(ChainState *st, int n) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n) {
        st[c].start = 0;
        st[c].prop = 0;
    }
}
}  // namespace

cudaError_t launch_copy16(const void *src, void *dst, size_t bytes, cudaStream_t s) {
    if (bytes == 0) return cudaSuccess;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    copy16_kernel<<<nsm * 4, 512, 0, s>>>(static_cast<const uint4 *>(src), static_cast<uint4 *>(dst),
                                          (int64_t)(bytes / 16));
    return cudaGetLastError();
}

cudaError_t launch_reset_chain_start(ChainState *st, int n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    reset_chain_start_kernel<<<(n + 255) / 256, 256, 0, s>>>(st, n);
    return cudaGetLastError();
}

cudaError_t fused_lattice_node_cluster(cudaGraphNode_t node, int cs) {
    cudaLaunchAttributeValue v{};
    v.clusterDim.x = (unsigned)cs;
    v.clusterDim.y = 1;
    v.clusterDim.z = 1;
    return cudaGraphKernelNodeSetAttribute(node, cudaLaunchAttributeClusterDimension, &v);
}

cudaError_t launch_tanh_selftest(const float *x, float *y, int64_t n, cudaStream_t s) {
    tanh_selftest_kernel<<<148, 256, 0, s>>>(x, y, n);
    return cudaGetLastError();
}

cudaError_t launch_log1pexp_selftest(const double *y, double *out, int64_t n, const float4 *tab,
                                     cudaStream_t s) {
    log1pexp_selftest_kernel<<<148, 256, 0, s>>>(y, out, n, tab);
    return cudaGetLastError();
}

}  // namespace ihmc
