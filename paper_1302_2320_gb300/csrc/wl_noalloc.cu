// wl_noalloc.cu -- wl_walk_noalloc: the persistent walker for callers that
// cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs while another framework
// owns the device's memory pool and forbids side allocations, code that must
// not synchronise the device (cudaMalloc/cudaFree can), or embedded hosts with
// a fixed memory plan decided up front.  They can still own and pass every
// input and output buffer.  What this entry point needs beyond those -- the
// exp threshold tables, the line descriptors, the work queue, the control words
// and the run summary -- lives in one file-scope __device__ array of fixed
// size, so nothing is allocated on any call.
//
// The paper has no counterpart: this is a deployment variant of the batched
// walker, not part of the method.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/wl.h"
#include "wl_kernels.cuh"
#include "wl_runtime.cuh"

using namespace wl;

namespace {

// Largest number of lines one call may walk (the full l <= N/2 surface of a
// lattice with N <= 8190 spins, e.g. the 64x64 square lattice's 2049 lines).
constexpr int kNoallocMaxLines = 4096;

// Scratch layout (byte offsets, each 256-aligned).
constexpr size_t kOffTable64 = 0;                                   // 4096 x u64
constexpr size_t kOffTable32 = kOffTable64 + kTableN * 8;           // 4096 x u32
constexpr size_t kOffDesc = kOffTable32 + kTableN * 4;              // lines x LineDesc
constexpr size_t kOffOrder = kOffDesc + kNoallocMaxLines * sizeof(LineDesc);
constexpr size_t kOffCtrl = kOffOrder + kNoallocMaxLines * 4;       // queue head, flags, deadline
constexpr size_t kOffSummary = kOffCtrl + 256;
constexpr size_t kScratchBytes = kOffSummary + 256;
static_assert(sizeof(Summary) <= 256, "summary slot");
static_assert(sizeof(LineDesc) == 16, "descriptor layout");

// Shared by every call on a device and kept between calls.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

wl_status nfail(wl_status s, const char* fmt, ...)
{
    char buf[256];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    wl::set_last_error(buf);
    return s;
}

// The device address of the scratch array on the current device; looked up
// once per device (the first call on a device does this set-up).
wl_status scratch_for_current_device(unsigned char** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return nfail(WL_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return nfail(WL_EINVAL, "device ordinal %d unsupported", dev);
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return nfail(WL_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        g_scratch_ptr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_scratch_ptr[dev]);
    return WL_OK;
}

// Host staging of one call (descriptors, work queue, exp tables, a copy of the
// caller's line states), kept out of the calling thread's stack: callers on
// small stacks (worker threads of another runtime, embedded hosts) stay safe.
// Calls serialise their staging on g_stage_mu.
std::mutex g_stage_mu;
LineDesc g_desc[kNoallocMaxLines];
int32_t g_order[kNoallocMaxLines];
uint64_t g_t64[kTableN];
uint32_t g_t32[kTableN];
LineState g_state[kNoallocMaxLines];

}  // namespace

extern "C" wl_status wl_walk_noalloc(wl_lattice lattice, int L, int ell_first, int nlines,
                                     uint32_t seed, int deterministic, double ln_f_min,
                                     double flatness, int64_t check_interval, int64_t move_budget,
                                     int mapping, int init, void* perm, uint32_t* spins,
                                     int64_t* lng, uint64_t* hist, int64_t* state,
                                     int64_t stream)
{
    // ---- arguments (host only; nothing is launched on a rejected call) ----
    int N = 0, z = 0;
    if (L < 3) return nfail(WL_EINVAL, "L must be >= 3");
    if (lattice == WL_SQUARE || lattice == WL_TRIANGULAR) N = L * L;
    else if (lattice == WL_SIMPLE_CUBIC && L <= 101) N = L * L * L;
    else return nfail(WL_EINVAL, "unsupported lattice %d / L %d", (int)lattice, L);
    if (N > (1 << 20)) return nfail(WL_EINVAL, "N > 2^20");
    z = lattice == WL_SQUARE ? 4 : 6;
    const int NB = N * z / 2;
    if (nlines < 1 || nlines > kNoallocMaxLines)
        return nfail(WL_EINVAL, "nlines %d outside [1, %d], the scratch limit", nlines, kNoallocMaxLines);
    if (ell_first < 0 || ell_first + nlines - 1 > N / 2)
        return nfail(WL_EINVAL, "lines [%d, %d] outside [0, N/2]", ell_first, ell_first + nlines - 1);
    if (!(ln_f_min >= 1e-10 && ln_f_min <= 0.5)) return nfail(WL_EINVAL, "ln_f_min out of [1e-10, 0.5]");
    if (!(flatness > 0.0 && flatness <= 1.0)) return nfail(WL_EINVAL, "flatness out of (0, 1]");
    const int flat_pm = (int)std::lround(flatness * 1000.0);
    if (flat_pm < 1) return nfail(WL_EINVAL, "flatness below 0.001");
    if (check_interval < 1 || check_interval > 0x7FFFFFFFll) return nfail(WL_EINVAL, "check_interval out of range");
    if (move_budget < 0) return nfail(WL_EINVAL, "move_budget < 0");
    if (mapping == 0) mapping = 8;
    if (!(mapping == 1 || mapping == 2 || mapping == 4 || mapping == 8 || mapping == 16 || mapping == 32))
        return nfail(WL_EINVAL, "mapping must be 0, 1, 2, 4, 8, 16 or 32");
    if (!perm || !spins || !lng || !hist || !state) return nfail(WL_EINVAL, "NULL buffer");
    if (((uintptr_t)perm | (uintptr_t)spins) & 15u) return nfail(WL_EINVAL, "perm and spins must be 16-byte aligned");
    if (((uintptr_t)lng | (uintptr_t)state | (uintptr_t)hist) & 7u)
        return nfail(WL_EINVAL, "lng, hist and state must be 8-byte aligned");
    const int q = wl::rt::table_shift(ln_f_min);
    if (q < 0) return nfail(WL_EINVAL, "ln_f_min out of range");
    const cudaStream_t s = (cudaStream_t)(intptr_t)stream;
    const bool idx16 = N <= 65536;
    const size_t isz = idx16 ? 2 : 4;
    const int pstride = (int)(((size_t)N * isz + 15) / 16 * 16 / isz);
    const int W = (int)((((size_t)(N + 31) / 32) * 4 + 15) / 16 * 4);

    unsigned char* scr = nullptr;
    wl_status st = scratch_for_current_device(&scr);
    if (st) return st;
    uint64_t* d_t64 = reinterpret_cast<uint64_t*>(scr + kOffTable64);
    uint32_t* d_t32 = reinterpret_cast<uint32_t*>(scr + kOffTable32);
    LineDesc* d_desc = reinterpret_cast<LineDesc*>(scr + kOffDesc);
    int32_t* d_order = reinterpret_cast<int32_t*>(scr + kOffOrder);
    int32_t* d_qnext = reinterpret_cast<int32_t*>(scr + kOffCtrl);
    int32_t* d_flags = reinterpret_cast<int32_t*>(scr + kOffCtrl + 16);
    uint64_t* d_deadline = reinterpret_cast<uint64_t*>(scr + kOffCtrl + 64);
    Summary* d_summary = reinterpret_cast<Summary*>(scr + kOffSummary);

#define NCU(call)                                                                              \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) return nfail(WL_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

    std::unique_lock<std::mutex> stage_lock(g_stage_mu);
    // ---- a continued walk must use the ln_f_min it was initialised with:
    // every running line has F = F0 >> 2 stage, every converged line F = 0 ----
    if (!init) {
        NCU(cudaMemcpyAsync(g_state, state, (size_t)nlines * sizeof(LineState), cudaMemcpyDeviceToHost, s));
        NCU(cudaStreamSynchronize(s));
        const int64_t F0 = std::llround(1.0 / ln_f_min);
        for (int i = 0; i < nlines; ++i) {
            const LineState& ls = g_state[i];
            const bool ok = ls.status == 1 ? ls.F == 0
                                           : (ls.stage >= 0 && ls.stage < 32 && ls.F == (F0 >> (2 * ls.stage)));
            if (!ok)
                return nfail(WL_EINVAL, "line %d: state (F %lld, stage %lld) was not initialised with ln_f_min %g",
                             ell_first + i, (long long)ls.F, (long long)ls.stage, ln_f_min);
        }
    }

    // ---- descriptors and work queue (static host staging -> scratch) ----
    int64_t off = 0;
    for (int i = 0; i < nlines; ++i) {
        const int l = ell_first + i;
        const int lm = std::min(l, N - l);
        const int64_t khi = std::min<int64_t>((int64_t)z * lm, NB);
        g_desc[i].bin_off = off;
        g_desc[i].ell = l;
        g_desc[i].nbins = (int)(khi / 2 + 1);
        off += g_desc[i].nbins;
        g_order[i] = i;
    }
    std::stable_sort(g_order, g_order + nlines,
                     [&](int a, int b) { return g_desc[a].nbins > g_desc[b].nbins; });
    NCU(cudaMemcpyAsync(d_desc, g_desc, nlines * sizeof(LineDesc), cudaMemcpyHostToDevice, s));
    NCU(cudaMemcpyAsync(d_order, g_order, nlines * 4, cudaMemcpyHostToDevice, s));
    // control words start at zero on every call
    NCU(cudaMemsetAsync(scr + kOffCtrl, 0, 256, s));

    // ---- exp threshold table: built on the device, checked against the host ----
    NCU(launch_exp_table(ln_f_min, q, d_t64, s));
    NCU(cudaMemcpyAsync(g_t64, d_t64, sizeof g_t64, cudaMemcpyDeviceToHost, s));
    NCU(cudaStreamSynchronize(s));
    if (deterministic) {
        for (int i = 0; i < kTableN; ++i)
            if (wl::rt::table_entry(ln_f_min, q, i) != g_t64[i])
                return nfail(WL_EMISMATCH, "exp table entry %d differs between device and host", i);
    }
    g_t32[0] = 0xFFFFFFFFu;
    for (int i = 1; i < kTableN; ++i) g_t32[i] = (uint32_t)g_t64[i];
    NCU(cudaMemcpyAsync(d_t32, g_t32, sizeof g_t32, cudaMemcpyHostToDevice, s));
    // pageable host -> device copies have taken the data once they return
    stage_lock.unlock();

    Geo g;
    g.type = (int)lattice;
    g.L = L;
    g.N = N;
    g.NB = NB;
    g.W = W;
    g.magic = (((uint64_t)1 << 40) + (uint64_t)L - 1) / (uint64_t)L;
    g.lshift = 0;
    while ((1 << (g.lshift + 1)) <= L) ++g.lshift;
    g.lmask = (uint32_t)L - 1u;
    const int klat = (lattice == WL_SQUARE && (L & (L - 1)) == 0) ? (int)kSquareP2 : (int)lattice;
    LineState* d_st = reinterpret_cast<LineState*>(state);

    if (init) {
        InitArgs ia;
        ia.g = g;
        ia.desc = d_desc;
        ia.st = d_st;
        ia.perm = perm;
        ia.spins = spins;
        ia.lng = lng;
        ia.hist = hist;
        ia.pstride = pstride;
        ia.nlines = nlines;
        ia.seed = seed;
        ia.F0 = std::llround(1.0 / ln_f_min);
        NCU(launch_init((int)lattice, idx16, ia, s));
    }

    // ---- launch shape: one warp per block, lists staged in shared memory
    // when a warp's walkers fit ----
    int dev = 0, nsm = 0, smem_optin = 0;
    NCU(cudaGetDevice(&dev));
    NCU(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    NCU(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const int S = mapping;
    const int groups = 32 / S;
    const size_t stg = (size_t)pstride * isz + (size_t)W * 4;
    const size_t cap = std::min<size_t>((size_t)smem_optin, 220 * 1024);
    const int stage = ((size_t)groups * (kWinBytes + stg) <= cap && stg <= 64 * 1024) ? 1 : 0;
    const size_t slot = kWinBytes + (stage ? stg : 0);
    const size_t smem = (size_t)groups * slot;
    int bps = 0;
    NCU(walk_kernel_attrs(klat, S, deterministic != 0, idx16, smem, 32, &bps));
    if (bps < 1) return nfail(WL_ECUDA, "walker cannot be resident");
    const int blocks = std::max(1, std::min((nlines + groups - 1) / groups, nsm * bps));

    WalkArgs a{};
    a.g = g;
    a.desc = d_desc;
    a.st = d_st;
    a.perm = perm;
    a.spins = spins;
    a.lng = lng;
    a.hist = hist;
    a.table = d_t32;
    a.order = d_order;
    a.qnext = d_qnext;
    a.nqueue = nlines;
    a.q = q;
    a.seg_per_log2 = (float)(std::log(2.0) / (std::ldexp(1.0, q) * ln_f_min));
    a.inv_u = (float)(1.0 / ln_f_min);
    a.seed = seed;
    a.flat_pm = flat_pm;
    a.stage_smem = stage;
    a.slot_bytes = (int)slot;
    a.pstride = pstride;
    a.C = check_interval;
    a.budget = move_budget;
    a.slice_moves = (int64_t)1 << 20;
    a.deadline_ns = d_deadline;
    a.abort_flag = nullptr;
    a.flags = d_flags;

    // ---- slices until every line converged or reached the budget ----
    Summary sm;
    for (;;) {
        NCU(cudaMemsetAsync(d_qnext, 0, 4, s));
        NCU(launch_walk(klat, S, deterministic != 0, idx16, dim3(blocks), dim3(32), smem, s, a));
        NCU(launch_summary(d_st, nlines, move_budget, d_flags, d_summary, s));
        NCU(cudaMemcpyAsync(&sm, d_summary, sizeof sm, cudaMemcpyDeviceToHost, s));
        NCU(cudaStreamSynchronize(s));
        if (sm.flags & 8) return nfail(WL_ECUDA, "walker state invariant broken");
        if (sm.overflow || (sm.flags & 4)) return nfail(WL_EOVERFLOW, "histogram bin overflow");
        if (sm.active == 0) break;
    }
#undef NCU
    return sm.converged == nlines ? WL_OK : nfail(WL_ENOTCONVERGED, "move budget reached");
}
