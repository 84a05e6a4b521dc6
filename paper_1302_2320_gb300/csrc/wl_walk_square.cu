// wl_walk_square.cu -- walker instantiations for the periodic square lattice.
#include "wl_walk_inst.cuh"

namespace wl {

cudaError_t launch_walk_square(int S, bool det, bool idx16, dim3 grid, dim3 block, size_t smem,
                              cudaStream_t s, const WalkArgs& a, int* bps)
{
    return walk_dispatch<kSquare>(S, det, idx16, grid, block, smem, s, a, bps);
}

}  // namespace wl
