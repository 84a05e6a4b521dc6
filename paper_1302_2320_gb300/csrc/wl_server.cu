// wl_server.cu -- a serving loop for density-of-states requests with continuous
// batching (include/wl.h, wl_server_*).
//
// Each request is one lattice to walk to ln f_min (every line l <= N/2, as
// wl_run).  A scheduler thread admits queued requests in arrival order while
// their device footprint fits the memory budget (and a cap on concurrent
// requests), keeps one slice of every admitted request in flight on the
// request's own stream -- so the walks of all admitted requests overlap on the
// GPU -- and, when a request's lines have all converged (or reached its move
// budget), assembles its surface, copies it to host memory, frees the device
// state and admits the next request.  Walker state stays on the device for the
// whole life of a request.
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
    wl_ctx* h = nullptr;
    int S = 32;
    wl::rt::Shape shape{};
    cudaEvent_t ev = nullptr;
    bool in_flight = false;          // scheduler thread only
    bool failed = false;             // scheduler thread only
    std::string error;               // message of a failed request
    std::vector<double> result;
};

}  // namespace

struct wl_server_ctx {
    std::mutex mu;
    std::condition_variable cv_done, cv_work;
    std::deque<Request*> pending;
    std::vector<Request*> active;                   // scheduler thread only
    std::unordered_map<int64_t, std::unique_ptr<Request>> reqs;
    int64_t budget = 0;
    int max_active = 0;
    size_t in_use = 0;
    int64_t next_id = 1;
    int device = 0;
    bool stop = false;
    Clock::time_point t0;
    std::thread th;
};

namespace {

double secs(const wl_server_ctx* s, Clock::time_point t)
{
    return std::chrono::duration<double>(t - s->t0).count();
}

// Runs on the scheduler thread: walker set-up for an admitted request.
wl_status start_request(Request* r)
{
    wl_status st = wl_create(r->lattice, r->L, &r->h);
    if (st) return st;
    const std::pair<const char*, int64_t> opts[] = {
        {"seed", r->seed}, {"check_interval", r->C}, {"move_budget", r->move_budget},
        {"slice_moves", (int64_t)1 << 18}};
    for (const auto& o : opts)
        if ((st = wl_set_option(r->h, o.first, o.second))) return st;
    if ((st = wl::rt::prepare(r->h, r->u, r->flatness, nullptr))) return st;
    if ((st = wl::rt::choose_shape(r->h, &r->S, &r->shape))) return st;
    if (cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming) != cudaSuccess) {
        wl::set_last_error("cudaEventCreate failed");
        return WL_ECUDA;
    }
    return WL_OK;
}

// Runs on the scheduler thread: assemble, copy the surface out, free the device.
wl_status finish_request(Request* r, wl_status st)
{
    if (st == WL_OK || st == WL_ENOTCONVERGED) {
        wl_status a = wl_assemble(r->h);
        size_t n = 0;
        if (!a) a = wl_get_surface(r->h, nullptr, 0, nullptr, 0, &n) == WL_EINVAL ? WL_OK : WL_ECUDA;
        if (!a) {
            r->result.resize(n);
            a = wl_get_surface(r->h, r->result.data(), n, nullptr, 0, &n);
        }
        if (a) st = a;
    }
    if (r->ev) cudaEventDestroy(r->ev);
    r->ev = nullptr;
    if (r->h) wl_destroy(r->h);
    r->h = nullptr;
    return st;
}

void scheduler(wl_server_ctx* s)
{
    cudaSetDevice(s->device);
    for (;;) {
        // admit queued requests, oldest first, while memory and slots allow
        for (;;) {
            Request* r = nullptr;
            {
                std::unique_lock<std::mutex> lk(s->mu);
                if (s->stop) break;
                if (s->pending.empty() || (int)s->active.size() >= s->max_active) break;
                Request* f = s->pending.front();
                if (s->budget > 0 && s->in_use + f->bytes > (size_t)s->budget) break;
                s->pending.pop_front();
                s->in_use += f->bytes;
                r = f;
            }
            wl_status st = start_request(r);
            std::string msg = st ? wl_last_error() : "";
            if (st) st = finish_request(r, st);
            std::lock_guard<std::mutex> lk(s->mu);
            if (st) {
                r->error = msg;
                r->status = st;
                r->state = 3;
                r->t_finish = Clock::now();
                s->in_use -= r->bytes;
                s->cv_done.notify_all();
            } else {
                r->state = 1;
                r->t_start = Clock::now();
                s->active.push_back(r);
            }
        }
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->stop) break;
            if (s->active.empty()) {
                s->cv_work.wait_for(lk, std::chrono::milliseconds(5));
                continue;
            }
        }
        // one slice of every admitted request in flight at once
        for (Request* r : s->active) {
            if (r->in_flight) continue;
            wl_status st = wl::rt::launch_slice_async(r->h, r->S, r->shape);
            if (!st) {
                const cudaError_t e = cudaEventRecord(r->ev, r->h->s);
                if (e != cudaSuccess) {
                    wl::set_last_error(cudaGetErrorString(e));
                    st = WL_ECUDA;
                }
            }
            if (st) {
                r->status = st;
                r->error = wl_last_error();
                r->failed = true;
                continue;
            }
            r->in_flight = true;
        }
        // retire finished slices
        bool progressed = false;
        for (size_t x = 0; x < s->active.size();) {
            Request* r = s->active[x];
            bool done = r->failed;
            wl_status st = r->status;
            if (!done && r->in_flight) {
                const cudaError_t q = cudaEventQuery(r->ev);
                if (q == cudaSuccess) {
                    r->in_flight = false;
                    progressed = true;
                    const wl::Summary sm = *r->h->h_summary;
                    {
                        std::lock_guard<std::mutex> lk(s->mu);
                        r->moves = sm.moves;
                    }
                    st = wl::rt::summary_status(r->h, sm);
                    if (st) r->error = wl_last_error();
                    if (st || sm.active == 0) {
                        done = true;
                        if (!st && sm.converged < r->h->lo.nlines) st = WL_ENOTCONVERGED;
                    }
                } else if (q == cudaErrorNotReady) {
                    (void)cudaGetLastError();      // not an error: the slice is still running
                } else {
                    done = true;
                    st = WL_ECUDA;
                    wl::set_last_error(cudaGetErrorString(q));
                    r->error = wl_last_error();
                }
            }
            if (!done) {
                ++x;
                continue;
            }
            if (r->in_flight) cudaEventSynchronize(r->ev);
            std::string msg = r->error;
            if (st && st != WL_ENOTCONVERGED && msg.empty()) msg = wl_last_error();
            st = finish_request(r, st);
            if (st && st != WL_ENOTCONVERGED && msg.empty()) msg = wl_last_error();
            std::lock_guard<std::mutex> lk(s->mu);
            r->error = msg;
            r->status = st;
            r->state = (st == WL_OK || st == WL_ENOTCONVERGED) ? 2 : 3;
            r->t_finish = Clock::now();
            s->in_use -= r->bytes;
            s->active.erase(s->active.begin() + (long)x);
            s->cv_done.notify_all();
            progressed = true;
        }
        if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    // shutting down: drop whatever is still admitted
    for (Request* r : s->active) {
        if (r->in_flight && r->ev) cudaEventSynchronize(r->ev);
        finish_request(r, WL_EABORTED);
        std::lock_guard<std::mutex> lk(s->mu);
        r->status = WL_EABORTED;
        r->state = 3;
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
    delete s;
    return WL_OK;
}

}  // extern "C"
