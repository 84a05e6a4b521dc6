// wl_server.cu -- a serving loop for density-of-states requests with continuous
// batching (include/wl.h, wl_server_*).
//
// Each request is one lattice to walk to ln f_min (every line l <= N/2, as
// wl_run).  Three parts cooperate:
//   - the scheduler thread admits queued requests (oldest first; a later one
//     that fits passes a head that waits for memory) while their device
//     footprint fits the memory budget and fewer than max_active run, keeps one
//     slice of every running request in flight on the request's own stream --
//     so the walks of all running requests overlap on the GPU -- and, when a
//     request's lines have all converged (or reached its move budget), enqueues
//     its assembly and the copy of its surface into pinned host memory on the
//     same stream.  It only launches work and polls events: it never waits for
//     the device, allocates or frees, so no admission or retirement stalls the
//     other requests' slices;
//   - a helper thread prepares admitted requests (walker initialisation, and
//     the first allocation of a handle) and frees evicted handles;
//   - handles are pooled by lattice: a finished request's handle (its device
//     arrays, stream and pinned result buffer) serves the next request of the
//     same lattice, so after warm-up nothing is allocated or freed while
//     requests come and go.  Idle handles count against the budget and are
//     evicted when a new lattice needs the room.
// Walker state stays on the device for the whole life of a request.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/wl.h"
#include "wl_runtime.cuh"

namespace {

using Clock = std::chrono::steady_clock;

// A handle with what a request needs around it, kept between requests.
struct Pooled {
    wl_ctx* h = nullptr;
    int lattice = 0, L = 0;
    size_t bytes = 0;              // device bytes (wl_required_bytes)
    double* pinned = nullptr;      // assembled surface, pinned host memory
    size_t pinned_n = 0;
    cudaEvent_t ev = nullptr;      // completion of the last slice / of the surface copy
};

struct Request {
    int64_t id = 0;
    wl_lattice lattice = WL_SQUARE;
    int L = 0;
    uint32_t seed = 1;
    double u = 1e-6, flatness = 0.8;
    int64_t C = 1000, move_budget = (int64_t)1 << 62;
    size_t bytes = 0;
    int state = 0;                 // 0 queued, 1 running, 2 done, 3 failed
    wl_status status = WL_OK;
    Clock::time_point t_submit, t_start, t_finish;
    int64_t moves = 0;
    Pooled* p = nullptr;
    int S = 32;
    wl::rt::Shape shape{};
    int phase = 0;                 // scheduler: 0 walking, 1 assembling and copying out
    bool in_flight = false;        // scheduler thread only
    std::string error;             // message of a failed request
    std::vector<double> result;
};

}  // namespace

struct wl_server_ctx {
    std::mutex mu;
    std::condition_variable cv_done, cv_work, cv_helper;
    std::deque<Request*> pending;                   // queued, arrival order
    std::deque<Request*> to_start, started;         // scheduler -> helper -> scheduler
    std::deque<Pooled*> to_free;                    // evicted handles, freed by the helper
    std::vector<Pooled*> idle;                      // pooled handles not in use
    std::vector<Request*> active;                   // scheduler thread only
    std::unordered_map<int64_t, std::unique_ptr<Request>> reqs;
    int64_t budget = 0;
    int max_active = 0;
    int admitted = 0;              // starting + running requests
    size_t in_use = 0;             // device bytes of every pooled handle (busy, idle or being freed)
    int64_t next_id = 1;
    int device = 0;
    bool stop = false, helper_stop = false;
    Clock::time_point t0;
    std::thread th, helper;
};

namespace {

double secs(const wl_server_ctx* s, Clock::time_point t)
{
    return std::chrono::duration<double>(t - s->t0).count();
}

void free_pooled(Pooled* p)
{
    if (p->ev) cudaEventDestroy(p->ev);
    if (p->pinned) cudaFreeHost(p->pinned);
    if (p->h) wl_destroy(p->h);
    delete p;
}

// Helper thread: a request's walker set-up (handle and pinned buffer on first
// use, options, initialisation, launch shape).
wl_status start_request(Request* r)
{
    Pooled* p = r->p;
    wl_status st = WL_OK;
    if (!p->h) {
        if ((st = wl_create(r->lattice, r->L, &p->h))) return st;
        int64_t bins = 0;
        wl_get_option(p->h, "bins", &bins);
        p->pinned_n = (size_t)bins;
        if (cudaHostAlloc((void**)&p->pinned, p->pinned_n * sizeof(double), cudaHostAllocDefault) != cudaSuccess ||
            cudaEventCreateWithFlags(&p->ev, cudaEventDisableTiming) != cudaSuccess) {
            wl::set_last_error("pinned buffer or event creation failed");
            return WL_ECUDA;
        }
    }
    if ((st = wl_reset(p->h))) return st;
    // slices end by device time (50 ms), so a request's lines never wait for
    // its slowest line at a slice end
    const std::pair<const char*, int64_t> opts[] = {
        {"seed", r->seed}, {"check_interval", r->C}, {"move_budget", r->move_budget},
        {"slice_moves", (int64_t)1 << 40}, {"slice_ms", 50}};
    for (const auto& o : opts)
        if ((st = wl_set_option(p->h, o.first, o.second))) return st;
    if ((st = wl::rt::prepare(p->h, r->u, r->flatness, nullptr))) return st;
    return wl::rt::choose_shape(p->h, &r->S, &r->shape);
}

void helper_loop(wl_server_ctx* s)
{
    cudaSetDevice(s->device);
    for (;;) {
        Request* r = nullptr;
        Pooled* f = nullptr;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_helper.wait(lk, [&] { return s->helper_stop || !s->to_start.empty() || !s->to_free.empty(); });
            if (!s->to_free.empty()) {
                f = s->to_free.front();
                s->to_free.pop_front();
            } else if (!s->to_start.empty() && !s->helper_stop) {
                r = s->to_start.front();
                s->to_start.pop_front();
            } else {
                return;                            // stop requested, nothing left
            }
        }
        if (f) {
            const size_t b = f->bytes;
            free_pooled(f);
            std::lock_guard<std::mutex> lk(s->mu);
            s->in_use -= b;
            s->cv_work.notify_all();
            continue;
        }
        const wl_status st = start_request(r);
        std::lock_guard<std::mutex> lk(s->mu);
        r->status = st;
        if (st) r->error = wl_last_error();
        s->started.push_back(r);
        s->cv_work.notify_all();
    }
}

// Scheduler, under s->mu: a handle for request r -- an idle one of the same
// lattice, or a new one when the budget allows after `reserved` bytes kept for
// earlier requests that are waiting.  For the oldest waiting request (reserved
// == 0) idle handles of other lattices are evicted to make room.  nullptr: r
// waits.
Pooled* take_handle(wl_server_ctx* s, Request* r, size_t reserved)
{
    for (size_t x = 0; x < s->idle.size(); ++x) {
        Pooled* p = s->idle[x];
        if (p->lattice == (int)r->lattice && p->L == r->L) {
            s->idle.erase(s->idle.begin() + (long)x);
            return p;
        }
    }
    if (s->budget > 0 && s->in_use + reserved + r->bytes > (size_t)s->budget) {
        if (reserved == 0) {
            size_t freeing = 0, idle_bytes = 0;
            for (Pooled* p : s->to_free) freeing += p->bytes;
            for (Pooled* p : s->idle) idle_bytes += p->bytes;
            if (s->in_use - freeing - idle_bytes + r->bytes <= (size_t)s->budget) {
                while (!s->idle.empty() && s->in_use - freeing + r->bytes > (size_t)s->budget) {
                    Pooled* p = s->idle.front();
                    s->idle.erase(s->idle.begin());
                    freeing += p->bytes;
                    s->to_free.push_back(p);
                }
                s->cv_helper.notify_all();
            }
        }
        return nullptr;              // admitted once running requests or the helper free memory
    }
    Pooled* p = new Pooled();
    p->lattice = (int)r->lattice;
    p->L = r->L;
    p->bytes = r->bytes;
    s->in_use += r->bytes;
    return p;
}

void finish(wl_server_ctx* s, Request* r, wl_status st, bool reuse)
{
    std::lock_guard<std::mutex> lk(s->mu);
    if (st && st != WL_ENOTCONVERGED && r->error.empty()) r->error = wl_last_error();
    r->status = st;
    r->state = (st == WL_OK || st == WL_ENOTCONVERGED) ? 2 : 3;
    r->t_finish = Clock::now();
    if (r->p) {
        if (reuse) s->idle.push_back(r->p);
        else {
            s->to_free.push_back(r->p);
            s->cv_helper.notify_all();
        }
        r->p = nullptr;
    }
    s->admitted -= 1;
    s->cv_done.notify_all();
}

void scheduler(wl_server_ctx* s)
{
    cudaSetDevice(s->device);
    for (;;) {
        bool progressed = false;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->stop) break;
            // admit: oldest first; a later request may pass a waiting one only
            // with memory the waiting ones do not need
            size_t reserved = 0;
            for (auto it = s->pending.begin(); it != s->pending.end() && s->admitted < s->max_active;) {
                Request* r = *it;
                Pooled* p = take_handle(s, r, reserved);
                if (!p) {
                    reserved += r->bytes;
                    ++it;
                    continue;
                }
                r->p = p;
                it = s->pending.erase(it);
                s->admitted += 1;
                s->to_start.push_back(r);
                s->cv_helper.notify_all();
                progressed = true;
            }
            // requests the helper has prepared
            while (!s->started.empty()) {
                Request* r = s->started.front();
                s->started.pop_front();
                progressed = true;
                if (r->status) {
                    lk.unlock();
                    finish(s, r, r->status, false);
                    lk.lock();
                    continue;
                }
                r->state = 1;
                r->t_start = Clock::now();
                r->phase = 0;
                s->active.push_back(r);
            }
            if (s->active.empty() && !progressed) {
                s->cv_work.wait_for(lk, std::chrono::milliseconds(5));
                continue;
            }
        }
        // one slice of every walking request in flight at once
        for (Request* r : s->active) {
            if (r->in_flight || r->phase != 0) continue;
            wl_status st = wl::rt::launch_slice_async(r->p->h, r->S, r->shape);
            if (!st && cudaEventRecord(r->p->ev, r->p->h->s) != cudaSuccess) {
                wl::set_last_error("cudaEventRecord failed");
                st = WL_ECUDA;
            }
            if (st) {
                r->status = st;
                r->error = wl_last_error();
                r->phase = 2;                      // failed: retire below
                continue;
            }
            r->in_flight = true;
        }
        // completed slices and surface copies
        for (size_t x = 0; x < s->active.size();) {
            Request* r = s->active[x];
            if (r->phase == 2) {                    // failed to launch
                s->active.erase(s->active.begin() + (long)x);
                finish(s, r, r->status, false);
                progressed = true;
                continue;
            }
            if (!r->in_flight) {
                ++x;
                continue;
            }
            const cudaError_t q = cudaEventQuery(r->p->ev);
            if (q == cudaErrorNotReady) {
                (void)cudaGetLastError();          // not an error: still running
                ++x;
                continue;
            }
            r->in_flight = false;
            progressed = true;
            if (q != cudaSuccess) {
                wl::set_last_error(cudaGetErrorString(q));
                r->error = wl_last_error();
                s->active.erase(s->active.begin() + (long)x);
                finish(s, r, WL_ECUDA, false);
                continue;
            }
            if (r->phase == 1) {                    // the surface is in pinned memory
                {
                    std::lock_guard<std::mutex> lk(s->mu);
                    r->result.assign(r->p->pinned, r->p->pinned + r->result.size());
                }
                s->active.erase(s->active.begin() + (long)x);
                finish(s, r, r->status, true);
                continue;
            }
            const wl::Summary sm = *r->p->h->h_summary;
            {
                std::lock_guard<std::mutex> lk(s->mu);
                r->moves = sm.moves;
            }
            wl_status st = wl::rt::summary_status(r->p->h, sm);
            if (st) {
                r->error = wl_last_error();
                s->active.erase(s->active.begin() + (long)x);
                finish(s, r, st, false);
                continue;
            }
            if (sm.active != 0) {
                ++x;
                continue;
            }
            // every line converged or at its budget: assemble and copy out, asynchronously
            r->status = sm.converged < r->p->h->lo.nlines ? WL_ENOTCONVERGED : WL_OK;
            size_t n = 0;
            st = wl::rt::assemble_copy_async(r->p->h, r->p->pinned, r->p->pinned_n, &n);
            if (!st && cudaEventRecord(r->p->ev, r->p->h->s) != cudaSuccess) {
                wl::set_last_error("cudaEventRecord failed");
                st = WL_ECUDA;
            }
            if (st) {
                r->error = wl_last_error();
                s->active.erase(s->active.begin() + (long)x);
                finish(s, r, st, false);
                continue;
            }
            {
                std::lock_guard<std::mutex> lk(s->mu);
                r->result.resize(n);               // filled when the copy has landed
            }
            r->phase = 1;
            r->in_flight = true;
            ++x;
        }
        if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    // shutting down: wait for what is on the device, drop whatever is still admitted
    for (Request* r : s->active) {
        if (r->in_flight) cudaEventSynchronize(r->p->ev);
        finish(s, r, WL_EABORTED, false);
    }
    s->active.clear();
    std::lock_guard<std::mutex> lk(s->mu);
    s->cv_done.notify_all();
}

Request* find(wl_server s, int64_t id)
{
    auto it = s->reqs.find(id);
    return it == s->reqs.end() ? nullptr : it->second.get();
}

}  // namespace

extern "C" {

wl_status wl_server_create(int64_t hbm_budget, int max_active, wl_server* out)
{
    if (!out || hbm_budget < 0 || max_active < 1) {
        wl::set_last_error("wl_server_create: bad arguments");
        return WL_EINVAL;
    }
    wl_server s = new (std::nothrow) wl_server_ctx();
    if (!s) return WL_ENOMEM;
    s->budget = hbm_budget;
    s->max_active = max_active;
    s->t0 = Clock::now();
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        wl::set_last_error("wl_server_create: no CUDA device");
        return WL_ECUDA;
    }
    s->helper = std::thread(helper_loop, s);
    s->th = std::thread(scheduler, s);
    *out = s;
    return WL_OK;
}

wl_status wl_server_submit(wl_server s, wl_lattice lattice, int L, uint32_t seed, double ln_f_min,
                           double flatness, int64_t check_interval, int64_t move_budget, int64_t* id)
{
    if (!s || !id) return WL_EINVAL;
    const size_t bytes = wl_required_bytes(lattice, L);
    if (!bytes || !(ln_f_min >= 1e-10 && ln_f_min <= 0.5) || !(flatness > 0 && flatness <= 1) ||
        check_interval < 1 || check_interval > 0x7FFFFFFFll || move_budget < 0) {
        wl::set_last_error("wl_server_submit: bad request");
        return WL_EINVAL;
    }
    if (s->budget > 0 && bytes > (size_t)s->budget) {
        wl::set_last_error("wl_server_submit: request larger than the memory budget");
        return WL_ENOMEM;
    }
    auto r = std::make_unique<Request>();
    r->lattice = lattice;
    r->L = L;
    r->seed = seed;
    r->u = ln_f_min;
    r->flatness = flatness;
    r->C = check_interval;
    r->move_budget = move_budget;
    r->bytes = bytes;
    r->t_submit = Clock::now();
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return WL_ESTATE;
    r->id = s->next_id++;
    *id = r->id;
    s->pending.push_back(r.get());
    s->reqs.emplace(r->id, std::move(r));
    s->cv_work.notify_all();
    return WL_OK;
}

wl_status wl_server_info(wl_server s, int64_t id, wl_request_info* info)
{
    if (!s || !info) return WL_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    Request* r = find(s, id);
    if (!r) return WL_EINVAL;
    info->state = r->state;
    info->status = r->status;
    info->lattice = (int32_t)r->lattice;
    info->L = r->L;
    info->moves = r->moves;
    info->bins = (int64_t)r->result.size();
    info->device_bytes = (int64_t)r->bytes;
    info->submit_s = secs(s, r->t_submit);
    info->start_s = r->state >= 1 ? secs(s, r->t_start) : -1.0;
    info->finish_s = r->state >= 2 ? secs(s, r->t_finish) : -1.0;
    return WL_OK;
}

wl_status wl_server_wait(wl_server s, int64_t id, double timeout_s)
{
    if (!s) return WL_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    Request* r = find(s, id);
    if (!r) return WL_EINVAL;
    const auto pred = [&] { return r->state >= 2; };
    if (timeout_s < 0) s->cv_done.wait(lk, pred);
    else if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), pred)) return WL_ETIMEOUT;
    if (r->status != WL_OK) wl::set_last_error(r->error.c_str());
    return r->status;
}

wl_status wl_server_result(wl_server s, int64_t id, double* out, size_t cap, size_t* n_out)
{
    if (!s) return WL_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    Request* r = find(s, id);
    if (!r || r->state != 2) return r ? WL_ESTATE : WL_EINVAL;
    if (n_out) *n_out = r->result.size();
    if (!out || cap < r->result.size()) return WL_EINVAL;
    memcpy(out, r->result.data(), r->result.size() * sizeof(double));
    return WL_OK;
}

wl_status wl_server_release(wl_server s, int64_t id)
{
    if (!s) return WL_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    Request* r = find(s, id);
    if (!r) return WL_EINVAL;
    if (r->state < 2) return WL_ESTATE;
    s->reqs.erase(id);
    return WL_OK;
}

wl_status wl_server_destroy(wl_server s)
{
    if (!s) return WL_EINVAL;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv_work.notify_all();
    }
    s->th.join();
    {
        // queued, starting and started requests are dropped; pooled handles freed
        std::lock_guard<std::mutex> lk(s->mu);
        for (Request* r : s->pending) {
            r->status = WL_EABORTED;
            r->state = 3;
        }
        s->pending.clear();
        for (Pooled* p : s->idle) s->to_free.push_back(p);
        s->idle.clear();
        s->helper_stop = true;
        s->cv_helper.notify_all();
    }
    s->helper.join();
    for (Request* r : s->started) {
        if (r->p) free_pooled(r->p);
        r->p = nullptr;
    }
    for (Request* r : s->to_start) {
        if (r->p) free_pooled(r->p);
        r->p = nullptr;
    }
    for (Pooled* p : s->to_free) free_pooled(p);
    delete s;
    return WL_OK;
}

}  // extern "C"
