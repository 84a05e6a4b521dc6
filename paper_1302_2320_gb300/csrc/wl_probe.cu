// wl_probe.cu -- wl_measure_peaks: the hardware rates the walker's roofline is
// stated against, measured on the device by the library's own microbenchmarks.
//
// The walk of a micromagnetic line (Eq. 3 and the text around it) is integer
// arithmetic and random memory access: per move attempt one Philox block, a few
// random reads of the up/down lists and of the packed spins, one read of ln g.
// Its roofline therefore has two kinds of ceilings, both measured here:
//   - random-access rates: 4-byte words read at random from shared memory (the
//     home of lists, spins and the ln g window up to the 64x64 lattice), and
//     32-byte sectors read at random from L2 (a buffer well inside L2) and from
//     HBM (a buffer far larger than L2; the home of the lists at 256x256);
//   - integer issue rates per instruction class: three-input logic/add (the
//     ALU pipe), 32-bit multiply-add, and the 32x32->64 products of Philox.
// Every kernel keeps many independent operations in flight per thread and
// fills every SM, so the figures are throughputs, not latencies.
#include <cstdint>
#include <cstdio>
#include <cstring>

#include "../../include/wl.h"
#include "wl_kernels.cuh"
#include "wl_runtime.cuh"

namespace {

constexpr int kStreams = 8;   // independent address streams / chains per thread

__device__ __forceinline__ uint32_t xorshift(uint32_t x)
{
    x ^= x << 13;
    x ^= x >> 17;
    x ^= x << 5;
    return x;
}

// Random 32-byte-aligned 16-byte reads (one sector each) from a buffer of
// nsec sectors (a power of two), through L2 only.
__global__ void random_sectors_kernel(const uint4* buf, uint32_t nsec_mask, int iters, uint32_t* out)
{
    uint32_t st[kStreams];
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll
    for (int s = 0; s < kStreams; ++s) st[s] = xorshift(tid * 2654435761u + 0x9E3779B9u * (s + 1)) | 1u;
    uint32_t acc = 0;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int s = 0; s < kStreams; ++s) {
            st[s] = xorshift(st[s]);
            const uint4 v = __ldcg(buf + 2 * (size_t)(st[s] & nsec_mask));
            acc ^= v.x ^ v.w;
        }
    }
    if (acc == 0x12345678u) out[tid] = acc;   // keeps the loads; practically never stores
}

// Random 4-byte reads from a 32 KB shared-memory table per block.
__global__ void random_smem_kernel(int iters, uint32_t* out)
{
    __shared__ uint32_t tab[8192];
    for (int x = threadIdx.x; x < 8192; x += blockDim.x) tab[x] = x * 2654435761u;
    __syncthreads();
    uint32_t st[kStreams];
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll
    for (int s = 0; s < kStreams; ++s) st[s] = xorshift(tid * 2246822519u + 0x85EBCA6Bu * (s + 1)) | 1u;
    uint32_t acc = 0;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int s = 0; s < kStreams; ++s) {
            st[s] = xorshift(st[s]);
            acc += tab[st[s] & 8191u];
        }
    }
    if (acc == 0x12345678u) out[tid] = acc;
}

// Integer issue: kStreams chains per thread; every round computes each chain's
// next value from its own and its neighbour's previous values (so nothing
// folds at compile time, and the kStreams operations of a round are
// independent), one operation of the class per chain step.  0: three-input
// logic (and-xor, nonlinear so that rounds cannot be folded), 1: three-input
// add, 2: 32-bit multiply-add, 3: a 32x32->64 product (high and low words)
// xor-ed with a neighbour, as in a Philox round.
template <int KIND>
__global__ void int_issue_kernel(int iters, uint32_t seed, uint32_t* out)
{
    uint32_t a[kStreams];
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll
    for (int s = 0; s < kStreams; ++s) a[s] = tid * (2u * s + 1u) + s + seed;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            uint32_t b[kStreams];
#pragma unroll
            for (int s = 0; s < kStreams; ++s) {
                const uint32_t x = a[s], y = a[(s + 1) % kStreams], k = 0x9E3779B9u * (r + 1);
                if (KIND == 0) b[s] = (x & y) ^ k;
                else if (KIND == 1) b[s] = x + y + k;
                else if (KIND == 2) b[s] = x * y + k;
                else b[s] = __umulhi(x, 0xD2511F53u) ^ (x * 0xD2511F53u) ^ y;
            }
#pragma unroll
            for (int s = 0; s < kStreams; ++s) a[s] = b[s];
        }
    }
    uint32_t acc = 0;
#pragma unroll
    for (int s = 0; s < kStreams; ++s) acc ^= a[s];
    if (acc == 0x12345678u) out[tid] = acc;
}

}  // namespace

extern "C" wl_status wl_measure_peaks(wl_peaks* out)
{
    if (!out) {
        wl::set_last_error("NULL argument");
        return WL_EINVAL;
    }
    memset(out, 0, sizeof *out);
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (!e) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    uint4* hbm = nullptr;
    uint32_t* sink = nullptr;
    const size_t hbm_bytes = (size_t)4 << 30, l2_bytes = (size_t)32 << 20;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (!e) e = cudaMalloc(&hbm, hbm_bytes);
    if (!e) e = cudaMalloc(&sink, (size_t)nsm * 8 * 256 * 4);
    if (!e) e = cudaMemset(hbm, 0x5A, hbm_bytes);
    if (!e) e = cudaEventCreate(&e0);
    if (!e) e = cudaEventCreate(&e1);
    const dim3 grid(nsm * 8), block(256);
    const double threads = (double)grid.x * block.x;
    auto timed = [&](auto launch, double ops, double* rate) {
        if (e) return;
        launch();                               // warm-up
        e = cudaEventRecord(e0);
        for (int r = 0; r < 3 && !e; ++r) launch();
        if (!e) e = cudaEventRecord(e1);
        if (!e) e = cudaEventSynchronize(e1);
        if (!e) e = cudaGetLastError();
        float ms = 0;
        if (!e) e = cudaEventElapsedTime(&ms, e0, e1);
        if (!e) *rate = 3.0 * ops / (ms * 1e-3);
    };
    const int it_mem = 256, it_smem = 512, it_int = 64;
    timed([&] { random_sectors_kernel<<<grid, block>>>(hbm, (uint32_t)(hbm_bytes / 32 - 1), it_mem, sink); },
          threads * it_mem * kStreams, &out->hbm_sectors_per_s);
    timed([&] { random_sectors_kernel<<<grid, block>>>(hbm, (uint32_t)(l2_bytes / 32 - 1), it_mem, sink); },
          threads * it_mem * kStreams, &out->l2_sectors_per_s);
    timed([&] { random_smem_kernel<<<grid, block>>>(it_smem, sink); },
          threads * it_smem * kStreams, &out->smem_words_per_s);
    const double int_ops = threads * it_int * 16 * kStreams;
    timed([&] { int_issue_kernel<0><<<grid, block>>>(it_int, 12345u, sink); }, int_ops, &out->lop3_ops_per_s);
    timed([&] { int_issue_kernel<1><<<grid, block>>>(it_int, 12345u, sink); }, int_ops, &out->iadd3_ops_per_s);
    timed([&] { int_issue_kernel<2><<<grid, block>>>(it_int, 12345u, sink); }, int_ops, &out->imad_ops_per_s);
    timed([&] { int_issue_kernel<3><<<grid, block>>>(it_int, 12345u, sink); }, int_ops, &out->mulwide_ops_per_s);
    out->sms = nsm;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(hbm);
    cudaFree(sink);
    if (e) {
        char buf[256];
        snprintf(buf, sizeof buf, "wl_measure_peaks: %s", cudaGetErrorString(e));
        wl::set_last_error(buf);
        return WL_ECUDA;
    }
    return WL_OK;
}
