// wl_kernels.cuh -- launch interface between the host runtime (wl_api.cu) and
// the kernels (wl_kernels.cu, wl_walk_*.cu).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "wl_device.cuh"

namespace wl {

struct InitArgs {
    Geo g;
    const LineDesc* desc;
    LineState* st;
    void* perm;
    uint32_t* spins;
    int64_t* lng;
    hist_t* hist;
    int32_t pstride;
    int32_t nlines;
    uint32_t seed;
    int64_t F0;
};

struct Summary {
    int64_t moves, accepts, checks, batches;
    int32_t active, converged, overflow, min_stage, max_stage, flags;
};

// Launch wrappers report the status of their own launch: an error left by an
// earlier runtime call (e.g. a not-ready query of an event) is cleared first.
inline void clear_stale_error() { (void)cudaGetLastError(); }

// Lanes-per-walker values compiled in.
constexpr int kMappings[] = {1, 2, 4, 8, 16, 32};

// Walker launch (one persistent grid, or one group for a single line).
cudaError_t launch_walk(int lattice, int S, bool det, bool idx16, dim3 grid, dim3 block,
                        size_t smem, cudaStream_t s, const WalkArgs& a);
cudaError_t walk_kernel_attrs(int lattice, int S, bool det, bool idx16, size_t smem,
                              int block_threads, int* blocks_per_sm, bool tbl = false);

cudaError_t launch_walk_square(int S, bool det, bool idx16, dim3 grid, dim3 block, size_t smem,
                               cudaStream_t s, const WalkArgs& a, int* bps);
cudaError_t launch_walk_triangular(int S, bool det, bool idx16, dim3 grid, dim3 block, size_t smem,
                                   cudaStream_t s, const WalkArgs& a, int* bps);
cudaError_t launch_walk_cubic(int S, bool det, bool idx16, dim3 grid, dim3 block, size_t smem,
                              cudaStream_t s, const WalkArgs& a, int* bps);
cudaError_t launch_walk_square_p2(int S, bool det, bool idx16, dim3 grid, dim3 block, size_t smem,
                                  cudaStream_t s, const WalkArgs& a, int* bps);
cudaError_t launch_walk_square_open(int S, bool det, bool idx16, dim3 grid, dim3 block, size_t smem,
                                    cudaStream_t s, const WalkArgs& a, int* bps);

cudaError_t launch_init(int lattice, bool idx16, const InitArgs& a, cudaStream_t s);
cudaError_t launch_assemble(const LineDesc* desc, const int64_t* lng, const hist_t* hist, int N,
                            int nlines, double u, double* out, cudaStream_t s);
cudaError_t launch_exp_table(double u, int q, uint64_t* out, cudaStream_t s);
cudaError_t launch_philox(size_t n, const uint32_t* ctr, const uint32_t* key, uint32_t* out,
                          cudaStream_t s);
cudaError_t launch_dmax(size_t n, const uint32_t* r, int det, const uint32_t* tab, int q,
                        float seg_per_log2, float inv_u, int64_t* out, cudaStream_t s);
cudaError_t launch_summary(const LineState* st, int nlines, int64_t budget, const int32_t* flags,
                           Summary* out, cudaStream_t s);
cudaError_t launch_set_deadline(uint64_t* deadline, uint64_t timeout_ns, cudaStream_t s);
cudaError_t launch_thermo(const LineDesc* desc, int nlines, const double* lng, int N, int NB,
                          int kstep, const double* T, int nT, const double* H, int nH, double* out,
                          cudaStream_t s);

}  // namespace wl
