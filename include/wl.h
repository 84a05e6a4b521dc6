/*
 * wl.h -- C ABI of the GB300 micromagnetic-ensemble Wang-Landau library
 * (method of B. D. Stosic, "Parallelizing Wang-Landau algorithm in the field:
 * the micromagnetic ensemble", arXiv:1302.2320).
 *
 * The problem (Eq. 1, Eq. 2): for the nearest-neighbour Ising model on a
 * lattice with N spins and N_B bonds, estimate the degeneracies g_kl, where k
 * in [0, N_B] counts antiparallel ("unhappy") bonds and l in [0, N] counts up
 * spins.  The method runs one independent one-dimensional Wang-Landau walk on
 * k per micromagnetic line l (spin-exchange moves that keep l fixed,
 * acceptance min(1, g(k|l)/g(k'|l)) of Eq. 3, ln g += ln f and h += 1 at the
 * current state, an 80%/80% histogram flatness test, ln f -> ln f / 4 until
 * ln f < ln f_min) and assembles g_kl = C(N,l) * normalised g(k|l) (Eq. 4).
 * Lines l and N-l are equal by up-down symmetry; only l <= N/2 is walked.
 *
 * Conventions for every entry point:
 *   - Handles are opaque and owned by the library; all device memory and all
 *     walker state belong to the handle and live across calls.
 *   - Output buffers are HOST memory owned by the caller.
 *   - No call aborts the process or traps the GPU.  A CUDA failure returns
 *     WL_ECUDA; the message is available from wl_last_error() (thread-local).
 *   - Calls on one handle must not overlap; distinct handles are independent.
 *   - ln g is held on the device as an int64 count of u = ln f_min (ln f is
 *     F*u with F an integer, F0 = round(1/u), F >>= 2 per stage; a line
 *     converges when F reaches 0); the assembled output is FP64.
 */
#ifndef WL_H
#define WL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wl_ctx* wl_handle;

typedef enum {
    WL_OK = 0,
    WL_EINVAL = 1,         /* bad argument or option value                       */
    WL_ENOMEM = 2,         /* allocation failed or exceeds the "hbm_budget" option */
    WL_ECUDA = 3,          /* a CUDA call failed (message in wl_last_error)      */
    WL_ETIMEOUT = 4,       /* "timeout_ms" elapsed; state is consistent, resumable */
    WL_EABORTED = 5,       /* wl_abort() was called; state consistent, resumable */
    WL_ENOTCONVERGED = 6,  /* "move_budget" reached before every line converged  */
    WL_EMISMATCH = 7,      /* device exp table differs from the host-built table */
    WL_ESTATE = 8,         /* call not valid in the handle's current state       */
    WL_EOVERFLOW = 9       /* a histogram bin would exceed 2^63-1 within a stage */
} wl_status;

/* Lattices.  Square: site i = y*L + x, neighbours (x+-1, y), (x, y+-1), periodic.
 * Triangular: rhombic LxL torus, the square's neighbours plus (x+1, y-1) and
 * (x-1, y+1).  Simple cubic: i = (z*L + y)*L + x, +-1 along each axis,
 * periodic.  Square with open boundaries (Fig. 2): the square lattice without
 * the wrap-around bonds, N_B = 2L(L-1).  L >= 3 (no double bonds); N <= 2^20.
 * On the periodic lattices k is always even (bins k = 0, 2, 4, ...); with open
 * boundaries every k occurs (bins k = 0, 1, 2, ...). */
typedef enum { WL_SQUARE = 0, WL_TRIANGULAR = 1, WL_SIMPLE_CUBIC = 2, WL_SQUARE_OPEN = 3 } wl_lattice;

/* Aggregate counters of a handle (totals over lines l <= N/2). */
typedef struct {
    int64_t moves;            /* move attempts made, summed over lines          */
    int64_t accepts;          /* accepted exchange proposals                    */
    int64_t checks;           /* flatness checks made                           */
    int64_t batches;          /* speculative batches evaluated (moves per batch = moves / batches) */
    int32_t lines;            /* lines walked (l = 0..N/2)                      */
    int32_t lines_converged;  /* lines with ln f < ln f_min                     */
    int32_t min_stage;        /* fewest completed stages over lines             */
    int32_t max_stage;        /* most completed stages over lines               */
    int32_t mapping;          /* lanes per walker used by the last wl_run       */
    int32_t form;             /* 0 persistent batched, 1 one launch per line    */
    int64_t launches;         /* kernels launched by the last wl_run            */
    double walk_ms;           /* device time of the last wl_run (CUDA events)   */
    double init_ms;           /* device time of walker initialisation           */
    double assemble_ms;       /* device time of the last wl_assemble            */
} wl_stats;

/* Create a handle for an L x L (square, triangular, open square) or L^3
 * (cubic) lattice (Eq. 1, "arbitrary lattice").  Computes the line table (bins
 * of the k in [0, min(z*min(l, N-l), N_B)], Eq. 2's k range per line);
 * device memory is allocated at the first wl_run.  *out receives the handle.
 * Errors: WL_EINVAL (bad lattice or L). */
wl_status wl_create(wl_lattice lattice, int L, wl_handle* out);

/* Device bytes a handle for (lattice, L) will hold once run, or 0 on bad
 * arguments: the ragged ln g / histogram arrays over each line's bins (Eq. 2's
 * k range per l) plus walker state.  Used to admit jobs against a memory
 * budget; the paper has no counterpart. */
size_t wl_required_bytes(wl_lattice lattice, int L);

/* Set an integer option before (or between) runs.  The options are the free
 * parameters of the walk of the method section (around Eq. 3 and Eq. 4, and
 * the Wang-Landau recap it builds on: how often flatness is checked, the random
 * stream, the move cap) and of how the library maps it onto the GPU.  Keys:
 *   "seed"           Philox key word 1 of every walker (default 1)
 *   "deterministic"  1: integer acceptance against the exp threshold table, the
 *                    chain bit-identical to the same walk taken one move at a
 *                    time (the CPU oracle's); 0: FP32 (d <= -ln U / u) (default 1)
 *   "check_interval" C: flatness is tested whenever t is a multiple of C (default 1000)
 *   "check_per_bin"  c > 0: a line with n bins tests flatness every max(C, c*n)
 *                    moves instead, so lines with more bins get longer stages
 *                    and find their rarest states before ln f shrinks (default 0)
 *   "move_budget"    per-line cap on the move counter t (default 2^62)
 *   "mapping"        lanes per walker S in {1,2,4,8,16,32}; 0 = tuned online: each
 *                    of 32, 16, 8 walks one slice (timed with CUDA events), the
 *                    fastest is kept, and they are timed again when the
 *                    acceptance rate drifts by more than 0.15 (default 0).
 *                    Every S walks the same chain.
 *   "form"           0: one persistent launch over all lines with a device
 *                    work queue; 1: one launch per line (default 0)
 *   "stream"         cudaStream_t (as an integer) for every launch (default: own stream)
 *   "slice_moves"    moves per line per persistent launch (default 2^20)
 *   "slice_ms"       if > 0, a persistent launch also ends after this many
 *                    milliseconds of device time, so that no line waits for a
 *                    slower one at the end of a slice (default 0)
 *   "tail"           1: with no more running lines than SMs, each line gets an
 *                    SM of its own (32 lanes per walker, unless another lane
 *                    count is forced); 0: keep the throughput shape (default 1)
 *   "timeout_ms"     wall-clock limit of one wl_run, 0 = none (default 0)
 *   "hbm_budget"     refuse to allocate more than this many bytes (default 0 = none)
 *   "ell_min", "ell_max"  walk only lines in [ell_min, ell_max] (defaults 0, N/2)
 *   "same_f_resets"  R: within the first R flatness checks of each stage, a
 *                    histogram that is not flat is reset and ln g normalised
 *                    while ln f is kept -- the extra reset the paper remarks
 *                    after Eq. 4 speeds the walk; its trigger is not given
 *                    there, this is one choice (default 0: off)
 * Setting "seed", "deterministic", "check_interval", "check_per_bin", "same_f_resets" or the
 * line range after a run requires wl_reset().  Errors: WL_EINVAL (unknown key or bad value), WL_ESTATE. */
wl_status wl_set_option(wl_handle h, const char* key, int64_t value);
/* Read an option back; also the read-only keys "N", "NB", "z", "k_step",
 * "lines", "bins", "device_bytes" and "tuned_mapping" (the lane count the tuner
 * settled on for this lattice and mode, 0 while it is still timing candidates). */
wl_status wl_get_option(wl_handle h, const char* key, int64_t* value);

/* The walk of the method section, on every selected line: spin-exchange
 * proposals that keep l fixed, acceptance min(1, g(k)/g(k')) (Eq. 3),
 * ln g(k) += ln f and h(k) += 1 at the current k, the flatness test of the
 * Wang-Landau recap every check_interval moves, and on a flat histogram the
 * stage step of Eq. 4 (h reset, ln g normalised, ln f -> ln f / 4).
 * Run the walks until every selected line has ln f < ln_f_min (returns WL_OK),
 * the move budget is reached (WL_ENOTCONVERGED), the timeout elapses
 * (WL_ETIMEOUT) or wl_abort() is called (WL_EABORTED).  ln_f_min in
 * [1e-10, 0.5]; flatness in (0, 1] is the fraction x of the x/x flatness test
 * (0.8 = "80% of visited k at or above 80% of the mean"), resolved to 1/1000.
 * The first run after wl_create or wl_reset initialises every walker (l up
 * spins at random, up/down index lists, ln g = 0, h = 0, ln f = 1); later runs
 * continue from the saved state and must pass the same ln_f_min and flatness.
 * Blocks the calling thread until the run stops. */
wl_status wl_run(wl_handle h, double ln_f_min, double flatness);

/* Walk only the lines ells[0..n) (each in [0, N/2], in any order; n = 0
 * restores every line).  Lines are independent walks (the paper's central
 * point: each micromagnetic line is its own one-dimensional Wang-Landau walk),
 * so a surface can be split across devices or hosts by lines and gathered
 * afterwards; a line walked here is bit-identical to the same line walked
 * with every other line.  Sets ell_min/ell_max to the set's extremes (setting
 * either option afterwards drops the set).  Before the first run or after
 * wl_reset (else WL_ESTATE).  wl_get_lng answers for walked lines only;
 * wl_get_surface covers [ell_min, ell_max], where lines outside the set hold
 * -inf (no bin visited).  Errors: WL_EINVAL, WL_ESTATE. */
wl_status wl_select_lines(wl_handle h, const int32_t* ells, int n);

/* Request that a wl_run in progress on another thread stop at its next
 * flatness check.  Safe to call from any thread.  No paper counterpart. */
wl_status wl_abort(wl_handle h);

/* Discard walker state (keeps allocations); the next wl_run re-initialises
 * (the initial state of the method section).  Errors: WL_EINVAL. */
wl_status wl_reset(wl_handle h);

/* Assemble ln g_kl = ln C(N,l) + ln g(k|l) - ln sum_k' g(k'|l) (Eq. 4 applied
 * once, FP64) for every walked line on the device.  Unvisited k get -inf. */
wl_status wl_assemble(wl_handle h);

/* The result of Eq. 4 for one line: ln g_kl, the line's density of states
 * normalised to C(N, l) (Eq. 2's g_kl; lines l and N-l equal by up-down
 * symmetry).  Copy line ell (0..N; ell > N/2 is served by its mirror N-ell) of the last
 * wl_assemble into out[0..n), n = number of bins, bin b holding k = k_lo +
 * b*k_step (k_lo = 0; k_step = 2 periodic, 1 open boundaries).  If cap < n nothing is copied, *n_out is
 * set and WL_EINVAL is returned.  Errors: WL_ESTATE before wl_assemble. */
wl_status wl_get_lng(wl_handle h, int ell, double* out, size_t cap,
                     int* k_lo, int* k_step, size_t* n_out);

/* The whole assembled surface ln g_kl of Eq. 2 / Eq. 4.  Copy every walked
 * line's assembled ln g (l = ell_min..ell_max, ragged, in
 * order of l) into out; offsets (length lines+1, may be NULL) receives the
 * start of each line.  *n_out = total bins.  cap too small: WL_EINVAL. */
wl_status wl_get_surface(wl_handle h, double* out, size_t cap, int64_t* offsets,
                         size_t offsets_cap, size_t* n_out);

/* Counters and timings of the handle (wl_stats above) into *out: moves,
 * accepted proposals (Eq. 3), flatness checks and stages (Eq. 4) of the walk;
 * the timings have no paper counterpart.  Errors: WL_EINVAL, WL_ECUDA. */
wl_status wl_get_stats(wl_handle h, wl_stats* out);

/* Thermodynamics from the assembled surface (the partition function of Eq. 2
 * with the energy of Eq. 1, J = k_B = 1): for every temperature T[a] > 0 and
 * field H[c], per spin, out[(a*nH + c)*6 + 0..5] = ln Z / N, <E>/N,
 * C/N = (<E^2> - <E>^2) / (N T^2), <M>/N, <|M|>/N, chi/N = (<M^2> - <M>^2)/(N T),
 * with M = 2l - N (l up spins; lines l > N/2 are their mirrors).  Host arrays.
 * Needs wl_assemble over every line l = 0..N/2 (else WL_ESTATE).  FP64. */
wl_status wl_thermo(wl_handle h, const double* T, int nT, const double* H, int nH, double* out);

/* The walker of one line as the method section defines it (current k, the
 * up/down lists the exchange move draws from, ln g, histogram, ln f).
 * Full state of one line walker, in plain layouts: scal[8] = {k, t, F (ln f
 * in units of u), stage, accepts, t at stage start, status (0 running,
 * 1 converged, 2 overflow), flatness checks}; perm[N] = up-spin list in
 * entries [0, l) followed by the down-spin list; spins[N] = 0/1 per site;
 * lng, hist, visited: one entry per bin (k = b * k_step).  Any pointer may be NULL. */
wl_status wl_get_line_state(wl_handle h, int ell, int64_t* scal, int32_t* perm,
                            uint8_t* spins, int64_t* lng, int64_t* hist, uint8_t* visited);

/* The deterministic form of Eq. 3's acceptance: the device-built exp
 * threshold table of the last run (4096 entries:
 * round(2^32 exp(-(i 2^q) u)), q the smallest shift with 4095*2^q*u >=
 * 32 ln 2) and its q.  Errors: WL_ESTATE before the first wl_run. */
wl_status wl_get_exp_table(wl_handle h, uint64_t* table, int* q);

/* The random numbers of the walk (the paper does not name a generator; this
 * library uses Philox4x32-10 keyed by (l, seed), counter = move number).
 * Run the library's device Philox4x32-10 on n counters: out[4i..4i+3] =
 * Philox(ctr[4i..4i+3], key[2i..2i+1]).  Host arrays.  For verification.
 * Errors: WL_EINVAL, WL_ECUDA. */
wl_status wl_philox(size_t n, const uint32_t* ctr, const uint32_t* key, uint32_t* out);

/* The walker's form of Eq. 3 for n random words r[i] (the third Philox word of
 * a move attempt): out[i] = dmax, the largest ln g increase d (in units of
 * u = ln_f_min) that the word accepts; a move with d <= dmax is accepted, every
 * d <= 0 included.  Deterministic rule: accept iff r < T(d), T the linear
 * interpolation of the exp threshold table (wl_get_exp_table); production
 * rule: accept iff (r/2^8 + 1/2) 2^-24 < exp(-u d) (FP32).  Host arrays.  For
 * verification.  Errors: WL_EINVAL, WL_EMISMATCH (device table differs from
 * the host-built table, deterministic only), WL_ECUDA. */
wl_status wl_accept_threshold(double ln_f_min, int deterministic, size_t n, const uint32_t* r,
                              int64_t* out);

/* Hardware rates the walk's roofline is stated against, measured by the
 * library's own microbenchmarks on the current device (all SMs busy, many
 * independent operations in flight per thread): random 4-byte reads from
 * shared memory, random 32-byte sectors from L2 (32 MB buffer) and from HBM
 * (4 GB buffer), and lane operations per second of three integer classes.
 * The walk of Eq. 3 is random access plus integer arithmetic (one Philox
 * block, list and spin reads, one ln g read per move attempt); the paper has
 * no counterpart.  Allocates 4 GB of device memory for the duration of the
 * call.  Errors: WL_EINVAL, WL_ECUDA. */
typedef struct {
    double smem_words_per_s;     /* random 4-byte shared-memory reads          */
    double l2_sectors_per_s;     /* random 32-byte sectors, L2-resident buffer */
    double hbm_sectors_per_s;    /* random 32-byte sectors, 4 GB buffer        */
    double lop3_ops_per_s;       /* three-input xor                            */
    double iadd3_ops_per_s;      /* three-input add                            */
    double imad_ops_per_s;       /* 32-bit multiply-add                        */
    double mulwide_ops_per_s;    /* 32x32->64 products (hi and lo) with an xor */
    int32_t sms;                 /* streaming multiprocessors of the device    */
} wl_peaks;

wl_status wl_measure_peaks(wl_peaks* out);

/* Free the handle's device memory and the handle; h is invalid afterwards.
 * No paper counterpart.  Errors: WL_EINVAL (NULL handle). */
wl_status wl_destroy(wl_handle h);

/* ---- Serving: density-of-states requests with continuous batching ----
 * No paper counterpart: a deployment of the method (each request is the
 * method's full walk of one lattice, wl_run + wl_assemble).
 * A server owns a scheduler thread on the device current at creation.
 * Requests (one lattice each, walked as wl_run would, to ln_f_min or to
 * move_budget) are admitted in arrival order while their device footprint
 * (wl_required_bytes) fits hbm_budget (0 = no limit) and fewer than max_active
 * are running; every admitted request keeps its walker state on the device and
 * has one slice in flight on its own stream, so the walks of all admitted
 * requests overlap on the GPU.  A finished request's assembled surface (l =
 * 0..N/2, as wl_get_surface) is kept in host memory until released.  In
 * deterministic mode each result is bit-identical to the same request run
 * alone through wl_run/wl_assemble. */
typedef struct wl_server_ctx* wl_server;

typedef struct {
    int32_t state;         /* 0 queued, 1 running, 2 done, 3 failed             */
    int32_t status;        /* wl_status of a finished request                   */
    int32_t lattice, L;
    int64_t moves;         /* move attempts so far (updated after each slice)   */
    int64_t bins;          /* bins of the stored result, once done              */
    int64_t device_bytes;  /* device memory held while admitted                 */
    double submit_s, start_s, finish_s;   /* seconds since wl_server_create; -1 if not yet */
} wl_request_info;

wl_status wl_server_create(int64_t hbm_budget, int max_active, wl_server* out);
/* Queue a request; *id identifies it.  WL_ENOMEM if it alone exceeds the budget. */
wl_status wl_server_submit(wl_server s, wl_lattice lattice, int L, uint32_t seed, double ln_f_min,
                           double flatness, int64_t check_interval, int64_t move_budget,
                           int64_t* id);
wl_status wl_server_info(wl_server s, int64_t id, wl_request_info* info);
/* Block until the request finished (its status) or timeout_s elapsed
 * (WL_ETIMEOUT; timeout_s < 0 waits forever). */
wl_status wl_server_wait(wl_server s, int64_t id, double timeout_s);
/* Copy a finished request's surface; *n_out = bins (set even if cap is too small). */
wl_status wl_server_result(wl_server s, int64_t id, double* out, size_t cap, size_t* n_out);
/* Forget a finished request and its stored surface. */
wl_status wl_server_release(wl_server s, int64_t id);
/* Stop the scheduler; running requests are dropped. */
wl_status wl_server_destroy(wl_server s);

/* The batched walker for callers that cannot allocate device memory.  The
 * paper has no counterpart; this is a deployment variant.  Some callers cannot
 * call cudaMalloc -- while another framework owns the device's memory pool,
 * where an allocation (or the synchronisation cudaMalloc/cudaFree may imply)
 * is not allowed, or under a memory plan fixed up front -- but can own every
 * input and output buffer.  This call allocates no device memory: its scratch
 * (exp tables, line descriptors, work queue, control words, run summary) is
 * one fixed ~129 KB __device__ array inside the library, held by every GPU
 * that loads it until the process exits; its host staging uses fixed static
 * arrays, not the caller's stack.
 *
 * Walks lines ell_first .. ell_first+nlines-1 (all <= N/2; nlines <= 4096, the
 * scratch limit -- larger requests return WL_EINVAL before any launch) of the
 * periodic lattice, exactly as wl_run does with the same options (seed,
 * deterministic, check_interval, move_budget, mapping; 0 = 8 lanes per walker),
 * on `stream` (a cudaStream_t as an integer, 0 = default stream), in slices of
 * 2^20 moves per line, and returns when every line converged (WL_OK) or
 * reached move_budget (WL_ENOTCONVERGED).  move_budget bounds the call: there
 * is no timeout, and move_budget = 0 makes no move and returns
 * WL_ENOTCONVERGED.  init != 0 first initialises every line (as the first
 * wl_run does); init == 0 continues the state held in the buffers and must
 * repeat the initialising call's lattice, L, lines, seed, deterministic,
 * ln_f_min, flatness and check_interval (ln_f_min is checked against the
 * states' ln f; the others cannot be checked).  Caller-owned DEVICE buffers:
 *   perm   nlines x P list entries, P = N rounded up so a line spans a multiple
 *          of 16 bytes; uint16 entries if N <= 65536, else uint32; 16-byte aligned
 *   spins  nlines x W uint32 words, W = ceil(N/32) rounded up to a multiple of 4
 *   lng    int64, hist uint64 (count, bit 63 = bin ever visited): the lines'
 *          bins back to back, line l holding min(z*min(l, N-l), N_B)/2 + 1 bins
 *          (k = 0, 2, ...)
 *   state  nlines x 9 int64: k, t, F, stage, accepts, t at stage start,
 *          status, checks, batches
 * The call blocks the calling thread until its stream has finished the walk
 * (it synchronises the stream after every slice and reads a summary into host
 * memory), so it cannot be captured into a CUDA graph.  The first call on a
 * device looks up the scratch address (cudaGetSymbolAddress), so that first
 * call must not run while any stream of the process is capturing.  Every call
 * shares the scratch and resets its control words; calls whose work overlaps on
 * the GPU (from several threads or streams) race on it and must be serialised
 * by the caller.  Errors as for wl_run; the message is in wl_last_error(). */
wl_status wl_walk_noalloc(wl_lattice lattice, int L, int ell_first, int nlines, uint32_t seed,
                          int deterministic, double ln_f_min, double flatness,
                          int64_t check_interval, int64_t move_budget, int mapping, int init,
                          void* perm, uint32_t* spins, int64_t* lng, uint64_t* hist,
                          int64_t* state, int64_t stream);

/* Message of the last failed call on this thread ("" if none).  No paper
 * counterpart. */
const char* wl_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* WL_H */
