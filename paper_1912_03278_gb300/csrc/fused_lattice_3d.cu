// fused_lattice_3d.cu -- the 3D instances of the fused FP32 lattice
// kernel (fused_lattice_impl.cuh).
#include "fused_lattice_impl.cuh"

namespace ihmc {

cudaError_t fused_node_3d(const FusedArgs &a, int threads, int depth, int vec,
                          cudaKernelNodeParams *np, void **args) {
    return node_dim<3, false>(a, threads, depth, vec, np, args);
}

}  // namespace ihmc
