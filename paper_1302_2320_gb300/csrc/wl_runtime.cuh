// wl_runtime.cuh -- internal to libwl.so: the handle and the runtime helpers
// shared by the C ABI (wl_api.cu) and the serving loop (wl_server.cu).
#pragma once

#include <cstdint>
#include <vector>

#include "../../include/wl.h"
#include "wl_kernels.cuh"

namespace wl {
namespace rt {

struct LatInfo {
    int type, L, N, NB, z;
    int kstep;      // spacing of the reachable k (2 periodic, 1 open boundaries)
};

struct Layout {
    int nlines;
    int pstride;     // list entries per line
    int W;           // spin words per line (multiple of 4)
    bool idx16;
    int64_t nbins_total;
    std::vector<LineDesc> desc;
};

// Launch shape of the persistent form for S lanes per walker.
struct Shape {
    dim3 grid, block;
    size_t smem;
    int stage;
    int slot;
    int tbl_mask = 0;   // tail shape: one walker per block with a conflict filter table
};

}  // namespace rt
}  // namespace wl

struct wl_ctx {
    wl::rt::LatInfo g{};
    wl::rt::Layout lo;
    // options
    uint32_t seed = 1;
    int det = 1;
    int64_t C = 1000;
    int64_t C_per_bin = 0;   // option "check_per_bin"
    int64_t budget = (int64_t)1 << 62;
    int mapping = 0;
    int form = 0;
    cudaStream_t user_stream = nullptr;
    bool has_user_stream = false;
    int64_t slice_moves = (int64_t)1 << 20;
    int64_t slice_ms = 0;    // option "slice_ms": a slice also ends after this much device time
    int64_t timeout_ms = 0;
    int64_t hbm_budget = 0;
    int ell_min = 0, ell_max = 0;
    std::vector<uint8_t> sel;   // lines chosen by wl_select_lines (empty: every line in [ell_min, ell_max])
    int same_f_resets = 0;
    int tail = 1;            // option "tail": few active lines get the one-walker-per-SM shape
    // state
    bool allocated = false, initialized = false, assembled = false;
    double u = 0.0;
    int flat_pm = 0;
    int q = 0;
    int last_mapping = 0;
    int64_t launches = 0;
    double walk_ms = 0, init_ms = 0, assemble_ms = 0;
    int64_t init_moves = 0;
    // device
    int device = 0, num_sms = 0;
    size_t max_smem = 0;
    cudaStream_t s = nullptr;
    std::vector<cudaStream_t> pool;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev_join = nullptr;
    cudaEvent_t ev_t0 = nullptr, ev_t1 = nullptr;   // one slice, for the lane-count tuner
    wl::LineDesc* d_desc = nullptr;
    wl::LineState* d_st = nullptr;
    void* d_perm = nullptr;
    uint32_t* d_spins = nullptr;
    int64_t* d_lng = nullptr;
    wl::hist_t* d_hist = nullptr;
    double* d_out = nullptr;
    uint32_t* d_table = nullptr;
    uint64_t* d_table64 = nullptr;
    int32_t* d_order = nullptr;
    int32_t* d_ident = nullptr;
    int32_t* d_qheads = nullptr;
    int32_t* d_flags = nullptr;
    uint64_t* d_deadline = nullptr;
    wl::Summary* d_summary = nullptr;
    wl::Summary* h_summary = nullptr;         // pinned
    int32_t* h_abort = nullptr;           // pinned, mapped
    int32_t* d_abort = nullptr;
    std::vector<uint64_t> table64;        // device-built table, copied back
    int nqueue = 0;
    // captured slice graph
    cudaGraphExec_t graph = nullptr;
    int graph_S = -1, graph_stage = -1;
    unsigned graph_grid = 0, graph_block = 0;
    wl::WalkArgs graph_args{};          // arguments baked into the captured graph
};

namespace wl {
void set_last_error(const char* msg);   // the message wl_last_error() returns

// Line l is walked: inside [ell_min, ell_max] and, if a set was selected, in it.
inline bool line_selected(const wl_ctx* h, int l)
{
    return l >= h->ell_min && l <= h->ell_max && (h->sel.empty() || h->sel[l]);
}

namespace rt {

// Validate (ln_f_min, flatness), allocate, make the handle's stream wait for
// `after` (may be null), and initialise the walkers on the first call after
// wl_create / wl_reset (the first part of wl_run).
wl_status prepare(wl_ctx* h, double ln_f_min, double flatness, cudaStream_t after);
// Lanes per walker (option, autotune cache or default) and the launch shape.
wl_status choose_shape(wl_ctx* h, int* S, Shape* sh);
// Enqueue one slice (captured graph) on the handle's stream; asynchronous.
// The slice's summary lands in h->h_summary when the stream reaches it.
wl_status launch_slice_async(wl_ctx* h, int S, const Shape& sh);
// Status implied by a slice summary (errors, stop requests).
wl_status summary_status(wl_ctx* h, const Summary& sm);
// Device bytes held by a handle of this lattice.
size_t handle_bytes(const wl_ctx* h);
// Enqueue the assembly of every walked line (Eq. 4) and the copy of the
// surface into host memory `dst` (pinned for an asynchronous copy) on the
// handle's stream; returns without waiting.  n_out = bins copied.
wl_status assemble_copy_async(wl_ctx* h, double* dst, size_t cap, size_t* n_out);
// The exp threshold table as built on the host, to check the device-built one:
// q, the smallest shift with 4095 * 2^q * u >= 32 ln 2 (-1 if none below 40),
// and entry i, round(2^32 exp(-(i 2^q) u)) evaluated in long double.
int table_shift(double u);
uint64_t table_entry(double u, int q, int i);

}  // namespace rt
}  // namespace wl
