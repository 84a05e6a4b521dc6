// wl_walk_square_open.cu -- walker instantiations for the square lattice with
// open boundaries.
#include "wl_walk_inst.cuh"

namespace wl {

cudaError_t launch_walk_square_open(int S, bool det, bool idx16, dim3 grid, dim3 block, size_t smem,
                                    cudaStream_t s, const WalkArgs& a, int* bps)
{
    return walk_dispatch<kSquareOpen>(S, det, idx16, grid, block, smem, s, a, bps);
}

}  // namespace wl
