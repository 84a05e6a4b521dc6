// wl_walk_inst.cuh -- instantiates the walker for one lattice over every
// (lanes per walker, acceptance mode, list index width) and dispatches at run
// time.  Included once per lattice by wl_walk_<lattice>.cu so the lattices
// compile in parallel.
#pragma once

#include "wl_kernels.cuh"
#include "wl_walk.cuh"

namespace wl {

template <int LAT, int S, bool DET, typename IDX, bool TBL>
cudaError_t walk_one(dim3 grid, dim3 block, size_t smem, cudaStream_t s, const WalkArgs& a,
                     int* bps)
{
    auto* fn = walk_kernel<LAT, S, DET, IDX, TBL>;
    // The dynamic shared-memory limit is a property of the kernel function,
    // shared by every handle: raise it to the device maximum (outside stream
    // capture) and never lower it, so a captured launch of one handle stays
    // valid whatever shape another handle uses.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (!bps) {
        cudaError_t e = cudaStreamIsCapturing(s, &cap);
        if (e != cudaSuccess) return e;
    }
    if (cap == cudaStreamCaptureStatusNone) {
        int dev = 0, optin = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     optin > (int)smem ? optin : (int)smem);
        if (e != cudaSuccess) return e;
    }
    if (bps) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, fn, (int)block.x, smem);
    clear_stale_error();
    fn<<<grid, block, smem, s>>>(a);
    return cudaGetLastError();
}

// The conflict-filter form (a.tbl_mask != 0) exists for 32 lanes per walker.
template <int LAT, int S>
cudaError_t walk_s(bool det, bool idx16, dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                   const WalkArgs& a, int* bps)
{
    if (S == 32 && a.tbl_mask != 0) {
        if (det) {
            if (idx16) return walk_one<LAT, S, true, uint16_t, true>(grid, block, smem, s, a, bps);
            return walk_one<LAT, S, true, uint32_t, true>(grid, block, smem, s, a, bps);
        }
        if (idx16) return walk_one<LAT, S, false, uint16_t, true>(grid, block, smem, s, a, bps);
        return walk_one<LAT, S, false, uint32_t, true>(grid, block, smem, s, a, bps);
    }
    if (a.tbl_mask != 0) return cudaErrorInvalidValue;
    if (det) {
        if (idx16) return walk_one<LAT, S, true, uint16_t, false>(grid, block, smem, s, a, bps);
        return walk_one<LAT, S, true, uint32_t, false>(grid, block, smem, s, a, bps);
    }
    if (idx16) return walk_one<LAT, S, false, uint16_t, false>(grid, block, smem, s, a, bps);
    return walk_one<LAT, S, false, uint32_t, false>(grid, block, smem, s, a, bps);
}

template <int LAT>
cudaError_t walk_dispatch(int S, bool det, bool idx16, dim3 grid, dim3 block, size_t smem,
                          cudaStream_t s, const WalkArgs& a, int* bps)
{
    switch (S) {
    case 1: return walk_s<LAT, 1>(det, idx16, grid, block, smem, s, a, bps);
    case 2: return walk_s<LAT, 2>(det, idx16, grid, block, smem, s, a, bps);
    case 4: return walk_s<LAT, 4>(det, idx16, grid, block, smem, s, a, bps);
    case 8: return walk_s<LAT, 8>(det, idx16, grid, block, smem, s, a, bps);
    case 16: return walk_s<LAT, 16>(det, idx16, grid, block, smem, s, a, bps);
    case 32: return walk_s<LAT, 32>(det, idx16, grid, block, smem, s, a, bps);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace wl
