// wl_api.cu -- host runtime and C ABI (include/wl.h) of the micromagnetic-
// ensemble Wang-Landau library (arXiv:1302.2320).
//
// A handle owns one lattice's walkers: the line table (l = 0..N/2 by up-down
// symmetry), ragged per-line ln g / histogram arrays over the even k, packed
// spins and up/down index lists, all resident on the device across calls.
// wl_run drives the walk in slices: each slice is one persistent launch over a
// device work queue (lines ordered by estimated cost, most expensive first),
// followed by a summary kernel whose result is read back; the slice is
// captured once as a CUDA graph and replayed.  The alternative "plain" form
// issues one launch per line over a pool of streams.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/wl.h"
#include "wl_kernels.cuh"
#include "wl_runtime.cuh"

using namespace wl;
using namespace wl::rt;

namespace {

thread_local std::string g_err;

wl_status fail(wl_status s, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

#define CU(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(WL_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                        __FILE__, __LINE__);                                              \
    } while (0)

bool lattice_info(int type, int L, LatInfo* o)
{
    if (L < 3) return false;
    o->type = type;
    o->L = L;
    if (type == WL_SQUARE) {
        o->N = L * L;
        o->z = 4;
    } else if (type == WL_TRIANGULAR) {
        o->N = L * L;
        o->z = 6;
    } else if (type == WL_SIMPLE_CUBIC) {
        if (L > 101) return false;
        o->N = L * L * L;
        o->z = 6;
    } else if (type == WL_SQUARE_OPEN) {
        o->N = L * L;
        o->z = 4;
    } else {
        return false;
    }
    if (o->N > (1 << 20)) return false;
    o->NB = type == WL_SQUARE_OPEN ? 2 * L * (L - 1) : o->N * o->z / 2;
    o->kstep = type == WL_SQUARE_OPEN ? 1 : 2;
    return true;
}

// Bins of line l: k in [0, min(z*min(l, N-l), N_B)] (no more than z unhappy
// bonds per minority spin) with the lattice's spacing: every even k on the
// periodic lattices (even degrees), every k with open boundaries.
int line_nbins(const LatInfo& g, int ell)
{
    const int lm = std::min(ell, g.N - ell);
    const int64_t khi = std::min<int64_t>((int64_t)g.z * lm, g.NB);
    return (int)(khi / g.kstep + 1);
}

size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

Layout make_layout(const LatInfo& g)
{
    Layout lo;
    lo.nlines = g.N / 2 + 1;
    lo.idx16 = g.N <= 65536;
    const size_t isz = lo.idx16 ? 2 : 4;
    lo.pstride = (int)(align16((size_t)g.N * isz) / isz);
    lo.W = (int)(align16((size_t)((g.N + 31) / 32) * 4) / 4);
    lo.desc.resize(lo.nlines);
    int64_t off = 0;
    for (int l = 0; l < lo.nlines; ++l) {
        lo.desc[l].bin_off = off;
        lo.desc[l].ell = l;
        lo.desc[l].nbins = line_nbins(g, l);
        off += lo.desc[l].nbins;
    }
    lo.nbins_total = off;
    return lo;
}

size_t required_bytes(const LatInfo& g, const Layout& lo)
{
    const size_t isz = lo.idx16 ? 2 : 4;
    size_t b = 0;
    b += (size_t)lo.nlines * sizeof(LineDesc) + (size_t)lo.nlines * sizeof(LineState);
    b += (size_t)lo.nlines * lo.pstride * isz;
    b += (size_t)lo.nlines * lo.W * 4;
    b += (size_t)lo.nbins_total * (8 + 8 + 8);   // lng, hist, assembled output
    b += (size_t)lo.nlines * 3 * 4;               // queue, per-line queue heads, identity
    b += kTableN * (4 + 8) + 4096;
    return b;
}

// Host-side exp threshold table, an independent evaluation in long double used
// to verify the device-built table bit for bit before a deterministic run.
int host_table_q(double u) { return wl::rt::table_shift(u); }

void host_table(double u, int q, std::vector<uint64_t>& t)
{
    t.resize(kTableN);
    for (int i = 0; i < kTableN; ++i) t[i] = wl::rt::table_entry(u, q, i);
}

struct TuneKey {
    int type, L, det;
    bool operator<(const TuneKey& o) const
    {
        return std::tie(type, L, det) < std::tie(o.type, o.L, o.det);
    }
};
// Autotuner record per (lattice, L, mode): the rate each candidate lane count
// reached on a slice of real work, at the acceptance rate seen then.
struct TuneRec {
    double rate[3] = {-1.0, -1.0, -1.0};   // for kTuneS[0..2]
    double accept = -1.0;                  // acceptance rate when the candidates were timed
    int best = 0;                          // 0 until every candidate has a rate
};
constexpr int kTuneS[3] = {32, 16, 8};
std::mutex g_tune_mu;
std::map<TuneKey, TuneRec> g_tune_cache;

}  // namespace

namespace wl {
// Lets other translation units of the library report through wl_last_error().
void set_last_error(const char* msg) { g_err = msg; }
}  // namespace wl

namespace {

void free_all(wl_ctx* h)
{
    if (h->graph) cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
    void* ptrs[] = {h->d_desc, h->d_st, h->d_perm, h->d_spins, h->d_lng, h->d_hist, h->d_out,
                    h->d_table, h->d_table64, h->d_order, h->d_ident, h->d_qheads, h->d_flags,
                    h->d_deadline, h->d_summary};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (h->h_summary) cudaFreeHost(h->h_summary);
    if (h->h_abort) cudaFreeHost(h->h_abort);
    for (auto st : h->pool) cudaStreamDestroy(st);
    h->pool.clear();
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    if (h->ev_t0) cudaEventDestroy(h->ev_t0);
    if (h->ev_t1) cudaEventDestroy(h->ev_t1);
    if (h->s) cudaStreamDestroy(h->s);
    h->allocated = false;
}

wl_status allocate(wl_ctx* h)
{
    if (h->allocated) return WL_OK;
    const size_t need = required_bytes(h->g, h->lo);
    if (h->hbm_budget > 0 && need > (size_t)h->hbm_budget)
        return fail(WL_ENOMEM, "lattice needs %zu device bytes, budget is %lld", need,
                    (long long)h->hbm_budget);
    CU(cudaGetDevice(&h->device));
    CU(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device));
    int smem_optin = 0;
    CU(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device));
    h->max_smem = (size_t)smem_optin;
    CU(cudaStreamCreateWithFlags(&h->s, cudaStreamNonBlocking));
    CU(cudaEventCreate(&h->ev0));
    CU(cudaEventCreate(&h->ev1));
    CU(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
    CU(cudaEventCreate(&h->ev_t0));
    CU(cudaEventCreate(&h->ev_t1));
    const Layout& lo = h->lo;
    const size_t isz = lo.idx16 ? 2 : 4;
    auto alloc = [&](void** p, size_t bytes) -> cudaError_t { return cudaMalloc(p, bytes ? bytes : 16); };
    cudaError_t e = cudaSuccess;
    if (!e) e = alloc((void**)&h->d_desc, lo.nlines * sizeof(LineDesc));
    if (!e) e = alloc((void**)&h->d_st, lo.nlines * sizeof(LineState));
    if (!e) e = alloc(&h->d_perm, (size_t)lo.nlines * lo.pstride * isz);
    if (!e) e = alloc((void**)&h->d_spins, (size_t)lo.nlines * lo.W * 4);
    if (!e) e = alloc((void**)&h->d_lng, (size_t)lo.nbins_total * 8);
    if (!e) e = alloc((void**)&h->d_hist, (size_t)lo.nbins_total * sizeof(hist_t));
    if (!e) e = alloc((void**)&h->d_out, (size_t)lo.nbins_total * 8);
    if (!e) e = alloc((void**)&h->d_table, kTableN * 4);
    if (!e) e = alloc((void**)&h->d_table64, kTableN * 8);
    if (!e) e = alloc((void**)&h->d_order, lo.nlines * 4);
    if (!e) e = alloc((void**)&h->d_ident, lo.nlines * 4);
    if (!e) e = alloc((void**)&h->d_qheads, (lo.nlines + 1) * 4);
    if (!e) e = alloc((void**)&h->d_flags, 16);
    if (!e) e = alloc((void**)&h->d_deadline, 16);
    if (!e) e = alloc((void**)&h->d_summary, sizeof(Summary));
    if (!e) e = cudaHostAlloc((void**)&h->h_summary, sizeof(Summary), cudaHostAllocDefault);
    if (!e) e = cudaHostAlloc((void**)&h->h_abort, 16, cudaHostAllocMapped);
    if (e) {
        const char* msg = cudaGetErrorString(e);
        free_all(h);
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? WL_ENOMEM : WL_ECUDA, "allocation failed: %s", msg);
    }
    CU(cudaHostGetDevicePointer((void**)&h->d_abort, h->h_abort, 0));
    *h->h_abort = 0;
    CU(cudaMemcpyAsync(h->d_desc, lo.desc.data(), lo.nlines * sizeof(LineDesc),
                       cudaMemcpyHostToDevice, h->s));
    std::vector<int32_t> ident(lo.nlines);
    for (int l = 0; l < lo.nlines; ++l) ident[l] = l;
    CU(cudaMemcpyAsync(h->d_ident, ident.data(), lo.nlines * 4, cudaMemcpyHostToDevice, h->s));
    CU(cudaMemsetAsync(h->d_deadline, 0, 16, h->s));
    CU(cudaStreamSynchronize(h->s));
    h->allocated = true;
    return WL_OK;
}

Geo make_geo(const wl_ctx* h)
{
    Geo g;
    g.type = h->g.type;
    g.L = h->g.L;
    g.N = h->g.N;
    g.NB = h->g.NB;
    g.W = h->lo.W;
    g.magic = (((uint64_t)1 << 40) + (uint64_t)h->g.L - 1) / (uint64_t)h->g.L;
    g.lshift = 0;
    while ((1 << (g.lshift + 1)) <= h->g.L) ++g.lshift;
    g.lmask = (uint32_t)h->g.L - 1u;
    return g;
}

// The work queue: selected lines by estimated cost (bins^2), largest first.
wl_status upload_queue(wl_ctx* h)
{
    std::vector<int32_t> order;
    for (int l = h->ell_min; l <= h->ell_max; ++l)
        if (line_selected(h, l)) order.push_back(l);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return h->lo.desc[a].nbins > h->lo.desc[b].nbins;
    });
    h->nqueue = (int)order.size();
    CU(cudaMemcpyAsync(h->d_order, order.data(), order.size() * 4, cudaMemcpyHostToDevice, h->s));
    return WL_OK;
}

wl_status initialise(wl_ctx* h, double u, int flat_pm)
{
    const int q = host_table_q(u);
    if (q < 0) return fail(WL_EINVAL, "ln_f_min %g out of range", u);
    CU(launch_exp_table(u, q, h->d_table64, h->s));
    h->table64.assign(kTableN, 0);
    CU(cudaMemcpyAsync(h->table64.data(), h->d_table64, kTableN * 8, cudaMemcpyDeviceToHost, h->s));
    CU(cudaStreamSynchronize(h->s));
    std::vector<uint64_t> ref;
    host_table(u, q, ref);
    if (h->det) {
        for (int i = 0; i < kTableN; ++i)
            if (ref[i] != h->table64[i])
                return fail(WL_EMISMATCH, "exp table entry %d: device %llu host %llu", i,
                            (unsigned long long)h->table64[i], (unsigned long long)ref[i]);
    }
    std::vector<uint32_t> t32(kTableN);
    t32[0] = 0xFFFFFFFFu;   // entry 0 (2^32) is implicit in the kernel
    for (int i = 1; i < kTableN; ++i) t32[i] = (uint32_t)h->table64[i];
    CU(cudaMemcpyAsync(h->d_table, t32.data(), kTableN * 4, cudaMemcpyHostToDevice, h->s));
    wl_status st = upload_queue(h);
    if (st) return st;
    CU(cudaMemsetAsync(h->d_flags, 0, 16, h->s));
    CU(cudaMemsetAsync(h->d_st, 0, h->lo.nlines * sizeof(LineState), h->s));
    // lines outside [ell_min, ell_max], or not in a selected set, are marked
    // converged with t = 0 so that no launch touches them
    InitArgs a;
    a.g = make_geo(h);
    a.desc = h->d_desc + h->ell_min;
    a.st = h->d_st + h->ell_min;
    a.perm = (uint8_t*)h->d_perm + (size_t)h->ell_min * h->lo.pstride * (h->lo.idx16 ? 2 : 4);
    a.spins = h->d_spins + (size_t)h->ell_min * h->lo.W;
    a.lng = h->d_lng;
    a.hist = h->d_hist;
    a.pstride = h->lo.pstride;
    a.nlines = h->ell_max - h->ell_min + 1;
    a.seed = h->seed;
    a.F0 = std::llround(1.0 / u);
    CU(cudaEventRecord(h->ev0, h->s));
    CU(launch_init(h->g.type == WL_SQUARE_OPEN ? (int)kSquareOpen : h->g.type, h->lo.idx16, a, h->s));
    CU(cudaEventRecord(h->ev1, h->s));
    {
        std::vector<LineState> out(h->lo.nlines);
        for (auto& s : out) {
            memset(&s, 0, sizeof s);
            s.status = 1;
        }
        // runs of lines that are not walked
        for (int l = 0; l < h->lo.nlines;) {
            if (line_selected(h, l)) {
                ++l;
                continue;
            }
            int e = l;
            while (e < h->lo.nlines && !line_selected(h, e)) ++e;
            CU(cudaMemcpyAsync(h->d_st + l, out.data(), (size_t)(e - l) * sizeof(LineState),
                               cudaMemcpyHostToDevice, h->s));
            l = e;
        }
    }
    CU(cudaStreamSynchronize(h->s));
    float ms = 0;
    CU(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
    h->init_ms = ms;
    h->u = u;
    h->flat_pm = flat_pm;
    h->q = q;
    h->initialized = true;
    h->assembled = false;
    return WL_OK;
}

WalkArgs base_args(wl_ctx* h)
{
    WalkArgs a{};
    a.g = make_geo(h);
    a.desc = h->d_desc;
    a.st = h->d_st;
    a.perm = h->d_perm;
    a.spins = h->d_spins;
    a.lng = h->d_lng;
    a.hist = h->d_hist;
    a.table = h->d_table;
    a.order = h->d_order;
    a.qnext = h->d_qheads + h->lo.nlines;
    a.nqueue = h->nqueue;
    a.q = h->q;
    a.seg_per_log2 = (float)(std::log(2.0) / (std::ldexp(1.0, h->q) * h->u));
    a.inv_u = (float)(1.0 / h->u);
    a.seed = h->seed;
    a.flat_pm = h->flat_pm;
    a.pstride = h->lo.pstride;
    a.same_f_resets = h->same_f_resets;
    a.C = h->C;
    a.C_per_bin = h->C_per_bin;
    a.budget = h->budget;
    a.slice_moves = h->slice_moves;
    a.deadline_ns = h->d_deadline;
    a.slice_end_ns = h->slice_ms > 0 ? h->d_deadline + 1 : nullptr;
    a.abort_flag = h->d_abort;
    a.flags = h->d_flags;
    return a;
}

int kernel_lattice(const wl_ctx* h);

// Tail shape: when no more lines are running than there are SMs, each gets a
// block of its own with a conflict filter table (exact when it has N entries).
bool tail_shape(wl_ctx* h, int S, int active, Shape* sh)
{
    if (!h->tail || S != 32 || active < 1 || active > h->num_sms) return false;
    const size_t isz = h->lo.idx16 ? 2 : 4;
    const size_t stg = (size_t)h->lo.pstride * isz + (size_t)h->lo.W * 4;
    const size_t cap = std::min<size_t>(h->max_smem, 220 * 1024);
    int H = 32;
    while (H < h->g.N && H < 32768) H <<= 1;
    size_t tbl = (size_t)H * 4;
    int stage = (kWinBytes + tbl + stg <= cap && stg <= 64 * 1024) ? 1 : 0;
    while (kWinBytes + tbl + (stage ? stg : 0) > cap && H > 32) {
        H >>= 1;
        tbl = (size_t)H * 4;
    }
    const size_t slot = kWinBytes + tbl + (stage ? stg : 0);
    if (slot > cap) return false;
    int bps = 0;
    if (walk_kernel_attrs(kernel_lattice(h), 32, h->det != 0, h->lo.idx16, slot, 32, &bps, true) != cudaSuccess ||
        bps < 1)
        return false;
    sh->grid = dim3(std::min(active, h->num_sms));
    sh->block = dim3(32);
    sh->smem = slot;
    sh->stage = stage;
    sh->slot = (int)slot;
    sh->tbl_mask = H - 1;
    return true;
}

wl_status persistent_shape(wl_ctx* h, int S, int* blocks_per_sm_out, Shape* sh, int active = -1)
{
    if (active >= 0 && !blocks_per_sm_out && tail_shape(h, S, active, sh)) return WL_OK;
    const size_t isz = h->lo.idx16 ? 2 : 4;
    const size_t stg = (size_t)h->lo.pstride * isz + (size_t)h->lo.W * 4;
    const size_t cap = std::min<size_t>(h->max_smem, 220 * 1024);
    const int groups_per_warp = 32 / S;
    int stage = 0, max_warps = 0;
    size_t slot = kWinBytes;
    const size_t warps_staged = cap / ((size_t)groups_per_warp * (kWinBytes + stg));
    if (warps_staged >= 1 && stg <= 64 * 1024) {
        stage = 1;
        slot = kWinBytes + stg;
        max_warps = (int)std::min<size_t>(8, warps_staged);
    } else {
        max_warps = (int)std::min<size_t>(8, cap / ((size_t)groups_per_warp * kWinBytes));
    }
    if (max_warps < 1) return fail(WL_ECUDA, "no walker shape fits shared memory (S=%d)", S);
    // The smallest block that still holds every queued line in one wave spreads
    // the walkers over the most SMs; otherwise take the largest capacity.
    int best_w = 0, best_bps = 0;
    long best_cap = -1;
    for (int w = 1; w <= max_warps; ++w) {
        const int threads = w * 32;
        const size_t smem = (size_t)(threads / S) * slot;
        int bps = 0;
        CU(walk_kernel_attrs(kernel_lattice(h), S, h->det != 0, h->lo.idx16, smem, threads, &bps));
        if (bps < 1) continue;
        const long capy = (long)h->num_sms * bps * (threads / S);
        if (capy >= h->nqueue) {
            best_w = w;
            best_bps = bps;
            best_cap = capy;
            break;
        }
        if (capy > best_cap) {
            best_w = w;
            best_bps = bps;
            best_cap = capy;
        }
    }
    if (best_w == 0) return fail(WL_ECUDA, "walker kernel cannot be resident (S=%d)", S);
    const int threads = best_w * 32;
    const size_t smem = (size_t)(threads / S) * slot;
    const int groups_per_block = threads / S;
    const int need_blocks = (h->nqueue + groups_per_block - 1) / groups_per_block;
    const int blocks = std::max(1, std::min(need_blocks, h->num_sms * best_bps));
    sh->grid = dim3(blocks);
    sh->block = dim3(threads);
    sh->smem = smem;
    sh->stage = stage;
    sh->slot = (int)slot;
    if (blocks_per_sm_out) *blocks_per_sm_out = best_bps;
    return WL_OK;
}

// One slice of the persistent form on stream h->s (capturable).
wl_status enqueue_slice(wl_ctx* h, int S, const Shape& sh)
{
    WalkArgs a = base_args(h);
    a.stage_smem = sh.stage;
    a.slot_bytes = sh.slot;
    a.tbl_mask = sh.tbl_mask;
    CU(cudaMemsetAsync(a.qnext, 0, 4, h->s));
    if (h->slice_ms > 0) CU(launch_set_deadline(h->d_deadline + 1, (uint64_t)h->slice_ms * 1000000ull, h->s));
    CU(launch_walk(kernel_lattice(h), S, h->det != 0, h->lo.idx16, sh.grid, sh.block, sh.smem, h->s, a));
    CU(launch_summary(h->d_st, h->lo.nlines, h->budget, h->d_flags, h->d_summary, h->s));
    CU(cudaMemcpyAsync(h->h_summary, h->d_summary, sizeof(Summary), cudaMemcpyDeviceToHost, h->s));
    return WL_OK;
}

wl_status run_slice(wl_ctx* h, int S, const Shape& sh, bool use_graph)
{
    if (!use_graph) {
        wl_status st = enqueue_slice(h, S, sh);
        if (st) return st;
        h->launches += 2;
        return WL_OK;
    }
    WalkArgs now = base_args(h);
    now.stage_smem = sh.stage;
    now.slot_bytes = sh.slot;
    now.tbl_mask = sh.tbl_mask;
    const bool same = h->graph && h->graph_S == S && h->graph_stage == sh.stage &&
                      h->graph_grid == sh.grid.x && h->graph_block == sh.block.x &&
                      memcmp(&h->graph_args, &now, sizeof now) == 0;
    if (!same) {
        if (h->graph) cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
        cudaGraph_t g;
        CU(cudaStreamBeginCapture(h->s, cudaStreamCaptureModeThreadLocal));
        wl_status st = enqueue_slice(h, S, sh);
        cudaError_t e = cudaStreamEndCapture(h->s, &g);
        if (st) return st;
        if (e != cudaSuccess) return fail(WL_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&h->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return fail(WL_ECUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
        h->graph_S = S;
        h->graph_stage = sh.stage;
        h->graph_grid = sh.grid.x;
        h->graph_block = sh.block.x;
        memcpy(&h->graph_args, &now, sizeof now);
    }
    CU(cudaGraphLaunch(h->graph, h->s));
    h->launches += 2;
    return WL_OK;
}

// Device-side stop conditions recorded during a launch.
wl_status check_flags(wl_ctx* h, const Summary& sm)
{
    if (sm.flags & 8) return fail(WL_ECUDA, "walker state invariant broken (k' outside its bins)");
    if (sm.overflow || (sm.flags & 4)) return fail(WL_EOVERFLOW, "a histogram bin exceeded 2^63-1 within one stage");
    if (sm.flags & 3) {
        CU(cudaMemsetAsync(h->d_flags, 0, 16, h->s));
        *h->h_abort = 0;
        if (sm.flags & 2) return fail(WL_EABORTED, "aborted");
        return fail(WL_ETIMEOUT, "device deadline reached");
    }
    return WL_OK;
}

// Walker specialisation: the square lattice with L a power of two takes the
// shift-and-mask geometry.
int kernel_lattice(const wl_ctx* h)
{
    if (h->g.type == WL_SQUARE && (h->g.L & (h->g.L - 1)) == 0) return kSquareP2;
    if (h->g.type == WL_SQUARE_OPEN) return kSquareOpen;
    return h->g.type;
}

// 32 lanes per walker: on the 64x64 lattice a batch commits ~26 moves and this
// mapping was fastest for every lattice measured.
int pick_mapping_default(const wl_ctx*)
{
    return 32;
}

// Persistent form: slices until every selected line converged or hit the
// budget, or the run is stopped.
//
// Lane count: fixed by the "mapping" option, or (mapping = 0) tuned online
// over real slices: each candidate (32, 16, 8 lanes per walker) walks one
// slice, timed with CUDA events, then the fastest is used; the candidates are
// timed again when the acceptance rate has moved by more than 0.15 since (the
// best count depends on it).  With no more running lines than SMs the tail
// shape (32 lanes, one walker per block) is used whatever the tuning says,
// unless a lane count other than 32 was forced.  Every count walks the same
// chain, so the choice never changes results.
wl_status run_persistent(wl_ctx* h, std::chrono::steady_clock::time_point t_start)
{
    const TuneKey key{h->g.type, h->g.L, h->det};
    int64_t prev_moves = -1, prev_accepts = 0;
    double last_accept = -1.0;
    int tried = -1;                       // candidate timed by the current slice
    for (;;) {
        int curS = h->mapping;
        tried = -1;
        const int active = prev_moves < 0 ? h->nqueue : h->h_summary->active;
        const bool tail = h->tail && (h->mapping == 0 || h->mapping == 32) && active <= h->num_sms;
        if (tail) {
            curS = 32;
        } else if (curS == 0) {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            TuneRec& tr = g_tune_cache[key];
            if (tr.best && last_accept >= 0.0 && tr.accept >= 0.0 && std::fabs(last_accept - tr.accept) > 0.15)
                tr = TuneRec();           // the walk has changed character: time the candidates again
            for (int c = 0; c < 3 && tried < 0; ++c)
                if (tr.rate[c] < 0.0) tried = c;
            curS = tried >= 0 ? kTuneS[tried] : tr.best;
        }
        Shape sh;
        wl_status st = persistent_shape(h, curS, nullptr, &sh, tail ? active : -1);
        if (st) return st;
        if (prev_moves < 0) {
            // moves before this run, for the tuning rates
            CU(launch_summary(h->d_st, h->lo.nlines, h->budget, h->d_flags, h->d_summary, h->s));
            CU(cudaMemcpyAsync(h->h_summary, h->d_summary, sizeof(Summary), cudaMemcpyDeviceToHost, h->s));
            CU(cudaStreamSynchronize(h->s));
            prev_moves = h->h_summary->moves;
            prev_accepts = h->h_summary->accepts;
        }
        CU(cudaEventRecord(h->ev_t0, h->s));
        st = run_slice(h, curS, sh, true);
        if (st) return st;
        CU(cudaEventRecord(h->ev_t1, h->s));
        CU(cudaStreamSynchronize(h->s));
        const Summary sm = *h->h_summary;
        h->last_mapping = curS;
        const int64_t dm = sm.moves - prev_moves;
        if (dm > 0) last_accept = (double)(sm.accepts - prev_accepts) / (double)dm;
        if (tried >= 0 && dm > 0) {
            float ms = 0;
            CU(cudaEventElapsedTime(&ms, h->ev_t0, h->ev_t1));
            std::lock_guard<std::mutex> lk(g_tune_mu);
            TuneRec& tr = g_tune_cache[key];
            tr.rate[tried] = (double)dm / std::max(1e-6, (double)ms);
            if (tr.accept < 0.0) tr.accept = last_accept;
            bool all = true;
            int bi = 0;
            for (int c = 0; c < 3; ++c) {
                all &= tr.rate[c] >= 0.0;
                if (tr.rate[c] > tr.rate[bi]) bi = c;
            }
            if (all) tr.best = kTuneS[bi];
        }
        prev_moves = sm.moves;
        prev_accepts = sm.accepts;
        st = check_flags(h, sm);
        if (st) return st;
        if (sm.active == 0) break;
        const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
        if ((sm.flags & 1) || (h->timeout_ms > 0 && el * 1000.0 > (double)h->timeout_ms)) {
            CU(cudaMemsetAsync(h->d_flags, 0, 16, h->s));
            return fail(WL_ETIMEOUT, "timeout after %.1f ms", el * 1000.0);
        }
        if (*h->h_abort) {
            *h->h_abort = 0;
            return fail(WL_EABORTED, "aborted");
        }
    }
    return WL_OK;
}

// Plain form: one launch per line (one walker group per launch) issued
// round-robin over a pool of streams; each launch runs its line to the budget
// or to convergence.
wl_status run_plain(wl_ctx* h)
{
    int S = h->mapping ? h->mapping : pick_mapping_default(h);
    h->last_mapping = S;
    const int npool = 128;      // the device runs at most 128 kernels at once
    while ((int)h->pool.size() < npool) {
        cudaStream_t st;
        CU(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        h->pool.push_back(st);
    }
    const size_t isz = h->lo.idx16 ? 2 : 4;
    const size_t stg = (size_t)h->lo.pstride * isz + (size_t)h->lo.W * 4;
    const int stage = (kWinBytes + stg <= std::min<size_t>(h->max_smem, 220 * 1024) &&
                       stg <= 64 * 1024) ? 1 : 0;
    const size_t slot = kWinBytes + (stage ? stg : 0);
    const size_t smem = slot;
    CU(cudaMemsetAsync(h->d_qheads, 0, h->lo.nlines * 4, h->s));
    CU(cudaEventRecord(h->ev_join, h->s));
    for (auto st : h->pool) CU(cudaStreamWaitEvent(st, h->ev_join, 0));
    WalkArgs a = base_args(h);
    a.stage_smem = stage;
    a.slot_bytes = (int)slot;
    a.nqueue = 1;
    std::vector<LineState> st_host(h->lo.nlines);
    for (;;) {
        // one launch per unfinished line, each running one slice of that line
        CU(cudaMemcpyAsync(st_host.data(), h->d_st, st_host.size() * sizeof(LineState),
                           cudaMemcpyDeviceToHost, h->s));
        CU(cudaMemsetAsync(h->d_qheads, 0, h->lo.nlines * 4, h->s));
        CU(cudaStreamSynchronize(h->s));
        CU(cudaEventRecord(h->ev_join, h->s));
        for (auto st : h->pool) CU(cudaStreamWaitEvent(st, h->ev_join, 0));
        int issued = 0;
        for (int l = h->ell_min; l <= h->ell_max; ++l) {
            if (!line_selected(h, l) || st_host[l].status != 0 || st_host[l].t >= h->budget) continue;
            a.order = h->d_ident + l;
            a.qnext = h->d_qheads + l;
            cudaStream_t st = h->pool[issued % npool];
            CU(launch_walk(kernel_lattice(h), S, h->det != 0, h->lo.idx16, dim3(1), dim3(S), smem, st, a));
            ++issued;
        }
        for (auto st : h->pool) {
            CU(cudaEventRecord(h->ev_join, st));
            CU(cudaStreamWaitEvent(h->s, h->ev_join, 0));
        }
        h->launches += issued + 1;
        CU(launch_summary(h->d_st, h->lo.nlines, h->budget, h->d_flags, h->d_summary, h->s));
        CU(cudaMemcpyAsync(h->h_summary, h->d_summary, sizeof(Summary), cudaMemcpyDeviceToHost, h->s));
        CU(cudaStreamSynchronize(h->s));
        const Summary sm = *h->h_summary;
        wl_status fs = check_flags(h, sm);
        if (fs) return fs;
        if (sm.active == 0 || issued == 0) break;
    }
    return WL_OK;
}

bool valid_handle(wl_handle h) { return h != nullptr; }

}  // namespace

namespace wl {
namespace rt {

wl_status prepare(wl_ctx* h, double ln_f_min, double flatness, cudaStream_t after)
{
    if (!(ln_f_min >= 1e-10 && ln_f_min <= 0.5)) return fail(WL_EINVAL, "ln_f_min must be in [1e-10, 0.5]");
    if (!(flatness > 0.0 && flatness <= 1.0)) return fail(WL_EINVAL, "flatness must be in (0, 1]");
    if (h->ell_min > h->ell_max) return fail(WL_EINVAL, "ell_min > ell_max");
    const int flat_pm = (int)std::lround(flatness * 1000.0);
    if (flat_pm < 1) return fail(WL_EINVAL, "flatness below 0.001");
    wl_status st = allocate(h);
    if (st) return st;
    if (after) {
        CU(cudaEventRecord(h->ev_join, after));
        CU(cudaStreamWaitEvent(h->s, h->ev_join, 0));
    }
    if (!h->initialized) {
        st = initialise(h, ln_f_min, flat_pm);
        if (st) return st;
        h->launches += 2;
    } else if (ln_f_min != h->u || flat_pm != h->flat_pm) {
        return fail(WL_EINVAL, "a continued run must use the same ln_f_min and flatness");
    }
    h->assembled = false;
    return WL_OK;
}

wl_status choose_shape(wl_ctx* h, int* S, Shape* sh)
{
    int m = h->mapping;
    if (m == 0) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find({h->g.type, h->g.L, h->det});
        m = it != g_tune_cache.end() && it->second.best ? it->second.best : pick_mapping_default(h);
    }
    *S = m;
    h->last_mapping = m;
    return persistent_shape(h, m, nullptr, sh);
}

wl_status launch_slice_async(wl_ctx* h, int S, const Shape& sh) { return run_slice(h, S, sh, true); }

wl_status summary_status(wl_ctx* h, const Summary& sm) { return check_flags(h, sm); }

size_t handle_bytes(const wl_ctx* h) { return required_bytes(h->g, h->lo); }

wl_status assemble_copy_async(wl_ctx* h, double* dst, size_t cap, size_t* n_out)
{
    if (!h->initialized) return fail(WL_ESTATE, "no run to assemble");
    const LineDesc& a = h->lo.desc[h->ell_min];
    const LineDesc& b = h->lo.desc[h->ell_max];
    const size_t n = (size_t)(b.bin_off + b.nbins - a.bin_off);
    if (n_out) *n_out = n;
    if (!dst || cap < n) return fail(WL_EINVAL, "output capacity %zu < %zu bins", cap, n);
    CU(launch_assemble(h->d_desc + h->ell_min, h->d_lng, h->d_hist, h->g.N,
                       h->ell_max - h->ell_min + 1, h->u, h->d_out, h->s));
    CU(cudaMemcpyAsync(dst, h->d_out + a.bin_off, n * 8, cudaMemcpyDeviceToHost, h->s));
    h->assembled = true;
    return WL_OK;
}

int table_shift(double u)
{
    const double need = 32.0 * std::log(2.0);
    for (int q = 0; q < 40; ++q)
        if (4095.0 * std::ldexp(1.0, q) * u >= need) return q;
    return -1;
}

uint64_t table_entry(double u, int q, int i)
{
    volatile double x = (double)((uint64_t)i << q) * u;
    const long double v = std::ldexp(std::exp(-(long double)x), 32) + 0.5L;
    return (uint64_t)std::floor(v);
}

}  // namespace rt
}  // namespace wl

extern "C" {

const char* wl_last_error(void) { return g_err.c_str(); }

size_t wl_required_bytes(wl_lattice lattice, int L)
{
    LatInfo g;
    if (!lattice_info((int)lattice, L, &g)) return 0;
    Layout lo = make_layout(g);
    return required_bytes(g, lo);
}

wl_status wl_create(wl_lattice lattice, int L, wl_handle* out)
{
    if (!out) return fail(WL_EINVAL, "out is NULL");
    *out = nullptr;
    LatInfo g;
    if (!lattice_info((int)lattice, L, &g))
        return fail(WL_EINVAL, "unsupported lattice %d with L=%d (L >= 3, N <= 2^20)", (int)lattice, L);
    wl_ctx* h = new (std::nothrow) wl_ctx();
    if (!h) return fail(WL_ENOMEM, "host allocation failed");
    h->g = g;
    h->lo = make_layout(g);
    h->ell_min = 0;
    h->ell_max = h->lo.nlines - 1;
    *out = h;
    g_err.clear();
    return WL_OK;
}

wl_status wl_destroy(wl_handle h)
{
    if (!valid_handle(h)) return fail(WL_EINVAL, "NULL handle");
    free_all(h);
    delete h;
    return WL_OK;
}

wl_status wl_set_option(wl_handle h, const char* key, int64_t v)
{
    if (!valid_handle(h) || !key) return fail(WL_EINVAL, "NULL handle or key");
    const std::string k(key);
    const bool semantic = (k == "seed" || k == "deterministic" || k == "check_interval" || k == "check_per_bin" ||
                           k == "ell_min" || k == "ell_max" || k == "same_f_resets");
    if (semantic && h->initialized)
        return fail(WL_ESTATE, "option '%s' changes the walk; call wl_reset first", key);
    if (k == "seed") {
        if (v < 0 || v > 0xFFFFFFFFll) return fail(WL_EINVAL, "seed must fit 32 bits");
        h->seed = (uint32_t)v;
    } else if (k == "deterministic") {
        h->det = v ? 1 : 0;
    } else if (k == "check_interval") {
        if (v < 1 || v > 0x7FFFFFFFll) return fail(WL_EINVAL, "check_interval must be in [1, 2^31-1]");
        h->C = v;
    } else if (k == "check_per_bin") {
        if (v < 0 || v > (1ll << 24)) return fail(WL_EINVAL, "check_per_bin must be in [0, 2^24]");
        h->C_per_bin = v;
    } else if (k == "move_budget") {
        if (v < 0) return fail(WL_EINVAL, "move_budget must be >= 0");
        h->budget = v;
    } else if (k == "mapping") {
        if (!(v == 0 || v == 1 || v == 2 || v == 4 || v == 8 || v == 16 || v == 32))
            return fail(WL_EINVAL, "mapping must be 0, 1, 2, 4, 8, 16 or 32");
        h->mapping = (int)v;
    } else if (k == "form") {
        if (v != 0 && v != 1) return fail(WL_EINVAL, "form must be 0 or 1");
        h->form = (int)v;
    } else if (k == "stream") {
        h->user_stream = (cudaStream_t)(intptr_t)v;
        h->has_user_stream = true;
    } else if (k == "slice_moves") {
        if (v < 1) return fail(WL_EINVAL, "slice_moves must be >= 1");
        h->slice_moves = v;
    } else if (k == "slice_ms") {
        if (v < 0) return fail(WL_EINVAL, "slice_ms must be >= 0");
        h->slice_ms = v;
    } else if (k == "timeout_ms") {
        if (v < 0) return fail(WL_EINVAL, "timeout_ms must be >= 0");
        h->timeout_ms = v;
    } else if (k == "hbm_budget") {
        if (v < 0) return fail(WL_EINVAL, "hbm_budget must be >= 0");
        h->hbm_budget = v;
    } else if (k == "same_f_resets") {
        if (v < 0 || v > 1000000) return fail(WL_EINVAL, "same_f_resets must be in [0, 10^6]");
        h->same_f_resets = (int)v;
    } else if (k == "tail") {
        if (v != 0 && v != 1) return fail(WL_EINVAL, "tail must be 0 or 1");
        h->tail = (int)v;
    } else if (k == "ell_min" || k == "ell_max") {
        if (v < 0 || v >= h->lo.nlines) return fail(WL_EINVAL, "%s must be in [0, %d]", key, h->lo.nlines - 1);
        (k == "ell_min" ? h->ell_min : h->ell_max) = (int)v;
        h->sel.clear();
    } else {
        return fail(WL_EINVAL, "unknown option '%s'", key);
    }
    return WL_OK;
}

wl_status wl_get_option(wl_handle h, const char* key, int64_t* v)
{
    if (!valid_handle(h) || !key || !v) return fail(WL_EINVAL, "NULL argument");
    const std::string k(key);
    if (k == "seed") *v = h->seed;
    else if (k == "deterministic") *v = h->det;
    else if (k == "check_interval") *v = h->C;
    else if (k == "check_per_bin") *v = h->C_per_bin;
    else if (k == "move_budget") *v = h->budget;
    else if (k == "mapping") *v = h->mapping;
    else if (k == "form") *v = h->form;
    else if (k == "stream") *v = (int64_t)(intptr_t)h->user_stream;
    else if (k == "slice_moves") *v = h->slice_moves;
    else if (k == "timeout_ms") *v = h->timeout_ms;
    else if (k == "slice_ms") *v = h->slice_ms;
    else if (k == "tuned_mapping") {
        // the lane count the tuner settled on for this lattice and mode (0: not yet)
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find({h->g.type, h->g.L, h->det});
        *v = it != g_tune_cache.end() ? it->second.best : 0;
    }
    else if (k == "hbm_budget") *v = h->hbm_budget;
    else if (k == "ell_min") *v = h->ell_min;
    else if (k == "same_f_resets") *v = h->same_f_resets;
    else if (k == "tail") *v = h->tail;
    else if (k == "ell_max") *v = h->ell_max;
    else if (k == "N") *v = h->g.N;
    else if (k == "NB") *v = h->g.NB;
    else if (k == "z") *v = h->g.z;
    else if (k == "k_step") *v = h->g.kstep;
    else if (k == "lines") *v = h->lo.nlines;
    else if (k == "bins") *v = h->lo.nbins_total;
    else if (k == "device_bytes") *v = (int64_t)required_bytes(h->g, h->lo);
    else return fail(WL_EINVAL, "unknown option '%s'", key);
    return WL_OK;
}

wl_status wl_reset(wl_handle h)
{
    if (!valid_handle(h)) return fail(WL_EINVAL, "NULL handle");
    if (h->ell_min > h->ell_max) return fail(WL_EINVAL, "ell_min > ell_max");
    h->initialized = false;
    h->assembled = false;
    return WL_OK;
}

wl_status wl_select_lines(wl_handle h, const int32_t* ells, int n)
{
    if (!valid_handle(h)) return fail(WL_EINVAL, "NULL handle");
    if (h->initialized) return fail(WL_ESTATE, "the line set changes the walk; call wl_reset first");
    if (n < 0 || (n > 0 && !ells)) return fail(WL_EINVAL, "bad line list");
    if (n == 0) {
        h->sel.clear();
        h->ell_min = 0;
        h->ell_max = h->lo.nlines - 1;
        return WL_OK;
    }
    std::vector<uint8_t> sel(h->lo.nlines, 0);
    int lo = h->lo.nlines, hi = -1;
    for (int x = 0; x < n; ++x) {
        const int l = ells[x];
        if (l < 0 || l >= h->lo.nlines) return fail(WL_EINVAL, "line %d outside [0, %d]", l, h->lo.nlines - 1);
        sel[l] = 1;
        lo = std::min(lo, l);
        hi = std::max(hi, l);
    }
    h->sel.swap(sel);
    h->ell_min = lo;
    h->ell_max = hi;
    return WL_OK;
}

wl_status wl_abort(wl_handle h)
{
    if (!valid_handle(h)) return fail(WL_EINVAL, "NULL handle");
    if (h->h_abort) *(volatile int32_t*)h->h_abort = 1;
    return WL_OK;
}

wl_status wl_run(wl_handle h, double ln_f_min, double flatness)
{
    if (!valid_handle(h)) return fail(WL_EINVAL, "NULL handle");
    const auto t_start = std::chrono::steady_clock::now();
    h->launches = 0;
    wl_status st = wl::rt::prepare(h, ln_f_min, flatness, h->has_user_stream ? h->user_stream : nullptr);
    if (st) return st;
    CU(launch_set_deadline(h->d_deadline, (uint64_t)h->timeout_ms * 1000000ull, h->s));
    CU(cudaEventRecord(h->ev0, h->s));
    st = h->form == 0 ? run_persistent(h, t_start) : run_plain(h);
    cudaError_t e = cudaEventRecord(h->ev1, h->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->s);
    if (e == cudaSuccess) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, h->ev0, h->ev1) == cudaSuccess) h->walk_ms = ms;
    }
    if (h->has_user_stream) {
        cudaEventRecord(h->ev_join, h->s);
        cudaStreamWaitEvent(h->user_stream, h->ev_join, 0);
    }
    if (st) return st;
    if (e != cudaSuccess) return fail(WL_ECUDA, "run failed: %s", cudaGetErrorString(e));
    const Summary sm = *h->h_summary;
    int selected = 0;
    for (int l = h->ell_min; l <= h->ell_max; ++l) selected += line_selected(h, l);
    const int outside = h->lo.nlines - selected;
    if (sm.converged - outside < selected) return fail(WL_ENOTCONVERGED, "move budget reached before convergence");
    g_err.clear();
    return WL_OK;
}

wl_status wl_assemble(wl_handle h)
{
    if (!valid_handle(h)) return fail(WL_EINVAL, "NULL handle");
    if (!h->initialized) return fail(WL_ESTATE, "no run to assemble");
    if (h->has_user_stream) {
        CU(cudaEventRecord(h->ev_join, h->user_stream));
        CU(cudaStreamWaitEvent(h->s, h->ev_join, 0));
    }
    CU(cudaEventRecord(h->ev0, h->s));
    CU(launch_assemble(h->d_desc + h->ell_min, h->d_lng, h->d_hist, h->g.N,
                       h->ell_max - h->ell_min + 1, h->u, h->d_out, h->s));
    CU(cudaEventRecord(h->ev1, h->s));
    if (h->has_user_stream) {
        CU(cudaEventRecord(h->ev_join, h->s));
        CU(cudaStreamWaitEvent(h->user_stream, h->ev_join, 0));
    }
    CU(cudaEventSynchronize(h->ev1));
    float ms = 0;
    CU(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
    h->assemble_ms = ms;
    h->assembled = true;
    return WL_OK;
}

wl_status wl_get_lng(wl_handle h, int ell, double* out, size_t cap, int* k_lo, int* k_step,
                     size_t* n_out)
{
    if (!valid_handle(h)) return fail(WL_EINVAL, "NULL handle");
    if (ell < 0 || ell > h->g.N) return fail(WL_EINVAL, "ell out of range");
    if (!h->assembled) return fail(WL_ESTATE, "call wl_assemble first");
    const int li = std::min(ell, h->g.N - ell);
    if (!line_selected(h, li)) return fail(WL_EINVAL, "line %d was not walked", ell);
    const LineDesc& d = h->lo.desc[li];
    if (n_out) *n_out = (size_t)d.nbins;
    if (k_lo) *k_lo = 0;
    if (k_step) *k_step = h->g.kstep;
    if (!out || cap < (size_t)d.nbins) return fail(WL_EINVAL, "output capacity %zu < %d bins", cap, d.nbins);
    CU(cudaMemcpyAsync(out, h->d_out + d.bin_off, (size_t)d.nbins * 8, cudaMemcpyDeviceToHost, h->s));
    CU(cudaStreamSynchronize(h->s));
    return WL_OK;
}

wl_status wl_get_surface(wl_handle h, double* out, size_t cap, int64_t* offsets, size_t offsets_cap,
                         size_t* n_out)
{
    if (!valid_handle(h)) return fail(WL_EINVAL, "NULL handle");
    if (!h->assembled) return fail(WL_ESTATE, "call wl_assemble first");
    const LineDesc& a = h->lo.desc[h->ell_min];
    const LineDesc& b = h->lo.desc[h->ell_max];
    const int64_t n = b.bin_off + b.nbins - a.bin_off;
    const int lines = h->ell_max - h->ell_min + 1;
    if (n_out) *n_out = (size_t)n;
    if (!out || cap < (size_t)n) return fail(WL_EINVAL, "output capacity %zu < %lld bins", cap, (long long)n);
    if (offsets) {
        if (offsets_cap < (size_t)lines + 1) return fail(WL_EINVAL, "offsets capacity too small");
        for (int l = 0; l < lines; ++l) offsets[l] = h->lo.desc[h->ell_min + l].bin_off - a.bin_off;
        offsets[lines] = n;
    }
    CU(cudaMemcpyAsync(out, h->d_out + a.bin_off, (size_t)n * 8, cudaMemcpyDeviceToHost, h->s));
    CU(cudaStreamSynchronize(h->s));
    return WL_OK;
}

wl_status wl_get_stats(wl_handle h, wl_stats* out)
{
    if (!valid_handle(h) || !out) return fail(WL_EINVAL, "NULL argument");
    memset(out, 0, sizeof *out);
    for (int l = h->ell_min; l <= h->ell_max; ++l) out->lines += line_selected(h, l);
    out->mapping = h->last_mapping;
    out->form = h->form;
    out->launches = h->launches;
    out->walk_ms = h->walk_ms;
    out->init_ms = h->init_ms;
    out->assemble_ms = h->assemble_ms;
    if (!h->initialized) return WL_OK;
    std::vector<LineState> st(h->lo.nlines);
    CU(cudaMemcpyAsync(st.data(), h->d_st, st.size() * sizeof(LineState), cudaMemcpyDeviceToHost, h->s));
    CU(cudaStreamSynchronize(h->s));
    out->min_stage = INT32_MAX;
    for (int l = h->ell_min; l <= h->ell_max; ++l) {
        if (!line_selected(h, l)) continue;
        const LineState& s = st[l];
        out->moves += s.t;
        out->accepts += s.accepts;
        out->checks += s.checks;
        out->batches += s.batches;
        out->lines_converged += s.status == 1;
        out->min_stage = std::min<int32_t>(out->min_stage, (int32_t)s.stage);
        out->max_stage = std::max<int32_t>(out->max_stage, (int32_t)s.stage);
    }
    return WL_OK;
}

wl_status wl_get_line_state(wl_handle h, int ell, int64_t* scal, int32_t* perm, uint8_t* spins,
                            int64_t* lng, int64_t* hist, uint8_t* visited)
{
    if (!valid_handle(h)) return fail(WL_EINVAL, "NULL handle");
    if (!h->initialized) return fail(WL_ESTATE, "no walker state yet");
    if (ell < 0 || ell >= h->lo.nlines) return fail(WL_EINVAL, "ell must be in [0, N/2]");
    const LineDesc& d = h->lo.desc[ell];
    const int N = h->g.N;
    if (scal) {
        LineState s;
        CU(cudaMemcpyAsync(&s, h->d_st + ell, sizeof s, cudaMemcpyDeviceToHost, h->s));
        CU(cudaStreamSynchronize(h->s));
        const int64_t v[8] = {s.k, s.t, s.F, s.stage, s.accepts, s.t_stage, s.status, s.checks};
        memcpy(scal, v, sizeof v);
    }
    if (perm) {
        const size_t isz = h->lo.idx16 ? 2 : 4;
        std::vector<uint8_t> raw((size_t)N * isz);
        CU(cudaMemcpyAsync(raw.data(), (uint8_t*)h->d_perm + (size_t)ell * h->lo.pstride * isz,
                           raw.size(), cudaMemcpyDeviceToHost, h->s));
        CU(cudaStreamSynchronize(h->s));
        for (int i = 0; i < N; ++i)
            perm[i] = isz == 2 ? (int32_t)((uint16_t*)raw.data())[i] : (int32_t)((uint32_t*)raw.data())[i];
    }
    if (spins) {
        std::vector<uint32_t> w(h->lo.W);
        CU(cudaMemcpyAsync(w.data(), h->d_spins + (size_t)ell * h->lo.W, w.size() * 4,
                           cudaMemcpyDeviceToHost, h->s));
        CU(cudaStreamSynchronize(h->s));
        for (int i = 0; i < N; ++i) spins[i] = (uint8_t)((w[i >> 5] >> (i & 31)) & 1u);
    }
    if (lng) {
        CU(cudaMemcpyAsync(lng, h->d_lng + d.bin_off, (size_t)d.nbins * 8, cudaMemcpyDeviceToHost, h->s));
        CU(cudaStreamSynchronize(h->s));
    }
    if (hist || visited) {
        std::vector<hist_t> hw(d.nbins);
        CU(cudaMemcpyAsync(hw.data(), h->d_hist + d.bin_off, (size_t)d.nbins * sizeof(hist_t),
                           cudaMemcpyDeviceToHost, h->s));
        CU(cudaStreamSynchronize(h->s));
        for (int b = 0; b < d.nbins; ++b) {
            if (hist) hist[b] = (int64_t)(hw[b] & ~kVisited);
            if (visited) visited[b] = (hw[b] & kVisited) ? 1 : 0;
        }
    }
    return WL_OK;
}

wl_status wl_thermo(wl_handle h, const double* T, int nT, const double* H, int nH, double* out)
{
    if (!valid_handle(h) || !T || !H || !out || nT < 1 || nH < 1) return fail(WL_EINVAL, "bad arguments");
    if (!h->assembled) return fail(WL_ESTATE, "call wl_assemble first");
    if (h->ell_min != 0 || h->ell_max != h->lo.nlines - 1 || !h->sel.empty())
        return fail(WL_ESTATE, "thermodynamics needs every line l = 0..N/2");
    for (int a = 0; a < nT; ++a)
        if (!(T[a] > 0.0)) return fail(WL_EINVAL, "temperatures must be > 0");
    const size_t nd = (size_t)nT + (size_t)nH + 6 * (size_t)nT * (size_t)nH;
    double* d = nullptr;
    CU(cudaMallocAsync(&d, nd * sizeof(double), h->s));
    cudaError_t e = cudaMemcpyAsync(d, T, nT * sizeof(double), cudaMemcpyHostToDevice, h->s);
    if (!e) e = cudaMemcpyAsync(d + nT, H, nH * sizeof(double), cudaMemcpyHostToDevice, h->s);
    if (!e) e = launch_thermo(h->d_desc, h->lo.nlines, h->d_out, h->g.N, h->g.NB, h->g.kstep, d, nT,
                              d + nT, nH, d + nT + nH, h->s);
    if (!e) e = cudaMemcpyAsync(out, d + nT + nH, 6 * (size_t)nT * nH * sizeof(double),
                                cudaMemcpyDeviceToHost, h->s);
    cudaFreeAsync(d, h->s);
    if (!e) e = cudaStreamSynchronize(h->s);
    if (e) return fail(WL_ECUDA, "wl_thermo: %s", cudaGetErrorString(e));
    return WL_OK;
}

wl_status wl_get_exp_table(wl_handle h, uint64_t* table, int* q)
{
    if (!valid_handle(h)) return fail(WL_EINVAL, "NULL handle");
    if (!h->initialized || h->table64.empty()) return fail(WL_ESTATE, "no table before the first run");
    if (table) memcpy(table, h->table64.data(), kTableN * 8);
    if (q) *q = h->q;
    return WL_OK;
}

wl_status wl_accept_threshold(double ln_f_min, int deterministic, size_t n, const uint32_t* r,
                              int64_t* out)
{
    if (!(ln_f_min >= 1e-10 && ln_f_min <= 0.5)) return fail(WL_EINVAL, "ln_f_min must be in [1e-10, 0.5]");
    if (n == 0) return WL_OK;
    if (!r || !out) return fail(WL_EINVAL, "NULL argument");
    const int q = host_table_q(ln_f_min);
    uint64_t* d64 = nullptr;
    uint32_t *d32 = nullptr, *dr = nullptr;
    int64_t* dout = nullptr;
    std::vector<uint64_t> t64(kTableN), ref;
    std::vector<uint32_t> t32(kTableN);
    host_table(ln_f_min, q, ref);
    cudaError_t e = cudaMalloc(&d64, kTableN * 8);
    if (!e) e = cudaMalloc(&d32, kTableN * 4);
    if (!e) e = cudaMalloc(&dr, n * 4);
    if (!e) e = cudaMalloc(&dout, n * 8);
    if (!e) e = launch_exp_table(ln_f_min, q, d64, 0);
    if (!e) e = cudaMemcpy(t64.data(), d64, kTableN * 8, cudaMemcpyDeviceToHost);
    bool same = true;
    if (!e) {
        for (int i = 0; i < kTableN; ++i) same &= t64[i] == ref[i];
        t32[0] = 0xFFFFFFFFu;
        for (int i = 1; i < kTableN; ++i) t32[i] = (uint32_t)t64[i];
        e = cudaMemcpy(d32, t32.data(), kTableN * 4, cudaMemcpyHostToDevice);
    }
    if (!e) e = cudaMemcpy(dr, r, n * 4, cudaMemcpyHostToDevice);
    if (!e)
        e = launch_dmax(n, dr, deterministic ? 1 : 0, d32, q,
                        (float)(std::log(2.0) / (std::ldexp(1.0, q) * ln_f_min)),
                        (float)(1.0 / ln_f_min), dout, 0);
    if (!e) e = cudaMemcpy(out, dout, n * 8, cudaMemcpyDeviceToHost);
    cudaFree(d64);
    cudaFree(d32);
    cudaFree(dr);
    cudaFree(dout);
    if (e) return fail(WL_ECUDA, "wl_accept_threshold: %s", cudaGetErrorString(e));
    if (deterministic && !same) return fail(WL_EMISMATCH, "device exp table differs from the host table");
    return WL_OK;
}

wl_status wl_philox(size_t n, const uint32_t* ctr, const uint32_t* key, uint32_t* out)
{
    if (n == 0) return WL_OK;
    if (!ctr || !key || !out) return fail(WL_EINVAL, "NULL argument");
    uint32_t *dc = nullptr, *dk = nullptr, *dout = nullptr;
    cudaError_t e = cudaMalloc(&dc, n * 16);
    if (!e) e = cudaMalloc(&dk, n * 8);
    if (!e) e = cudaMalloc(&dout, n * 16);
    if (!e) e = cudaMemcpy(dc, ctr, n * 16, cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(dk, key, n * 8, cudaMemcpyHostToDevice);
    if (!e) e = launch_philox(n, dc, dk, dout, 0);
    if (!e) e = cudaMemcpy(out, dout, n * 16, cudaMemcpyDeviceToHost);
    cudaFree(dc);
    cudaFree(dk);
    cudaFree(dout);
    if (e) return fail(WL_ECUDA, "wl_philox: %s", cudaGetErrorString(e));
    return WL_OK;
}

}  // extern "C"
