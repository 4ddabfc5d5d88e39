// fused_lattice_2d_cl.cu -- the 2D instances of the fused FP32 lattice
// kernel split over a thread-block cluster (fused_lattice_impl.cuh).
#include "fused_lattice_impl.cuh"

namespace ihmc {

cudaError_t fused_node_2d_cl(const FusedArgs &a, int threads, int depth, int vec,
                          cudaKernelNodeParams *np, void **args) {
    return node_dim<2, true>(a, threads, depth, vec, np, args);
}

}  // namespace ihmc
