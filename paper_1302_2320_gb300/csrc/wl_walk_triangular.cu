// wl_walk_triangular.cu -- walker instantiations for the periodic triangular lattice.
#include "wl_walk_inst.cuh"

namespace wl {

cudaError_t launch_walk_triangular(int S, bool det, bool idx16, dim3 grid, dim3 block, size_t smem,
                              cudaStream_t s, const WalkArgs& a, int* bps)
{
    return walk_dispatch<kTriangular>(S, det, idx16, grid, block, smem, s, a, bps);
}

}  // namespace wl
