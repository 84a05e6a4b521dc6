// wl_walk_square_p2.cu -- walker instantiations for the periodic square lattice
// with L a power of two (site coordinates by shift and mask).
#include "wl_walk_inst.cuh"

namespace wl {

cudaError_t launch_walk_square_p2(int S, bool det, bool idx16, dim3 grid, dim3 block, size_t smem,
                                  cudaStream_t s, const WalkArgs& a, int* bps)
{
    return walk_dispatch<kSquareP2>(S, det, idx16, grid, block, smem, s, a, bps);
}

}  // namespace wl
