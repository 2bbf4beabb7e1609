// serve.cu - the request loop: continuous batching of independent solves.
//
// Requests are admitted by device-memory footprint and slot count, set up by
// worker threads (hierarchy built, or taken from a cache of idle hierarchies
// of the same grid and options; RHS uploaded), and then iterate together:
// every step of the stepper thread is one outer iteration of all admitted
// requests as one batch (one launch per level operation).  Requests that
// become ready while others iterate join at the next step; converged ones
// retire at once, freeing their slot and memory for the queue.  Each request
// uses the same kernels and the same stop rule as mg_solve, so its result is
// bitwise the lone solve's.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <list>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "engine.h"

using namespace mgs;

namespace {

double now_s() {
    using clk = std::chrono::steady_clock;
    return std::chrono::duration<double>(clk::now().time_since_epoch()).count();
}

enum { RQ_QUEUED = 0, RQ_SETUP, RQ_READY, RQ_ACTIVE, RQ_DONE };

struct Request {
    uint64_t ticket = 0;
    mg_grid_desc grid{};
    mg_opts opts{};
    double tol = 0.0;
    std::vector<double> f;          // RHS (host copy taken at submit)
    mg_report rep{};
    mg_status status = MG_OK;
    int state = RQ_QUEUED;
    double t_submit = 0.0;
    mg_handle* h = nullptr;
    double* d_f = nullptr;
    double* d_x = nullptr;
    size_t bytes = 0;               // reserved footprint
    size_t x_bytes = 0;             // the part of it held by d_x until the poll
    cudaEvent_t ready = nullptr;    // recorded after the epilogue wrote d_x
    SolveState S;
    std::string key;
    std::string err;                // why the request failed (mg_last_error of its poll)
};

std::string key_of(const mg_grid_desc& g, const mg_opts& o) {
    char buf[512];
    std::snprintf(buf, sizeof(buf), "%d %d %d %.17g %.17g %.17g %.17g %d %.17g %.17g %.17g %d | %d %d %d %d %d %d %d %d %d %d %d",
                  g.nr, g.nth, g.nph, g.r_in, g.r_out, g.th0, g.th1, g.mapping, g.flattening, g.e2, g.stretch, g.cut,
                  o.precision, o.smoother, o.nu1, o.nu2, o.max_levels, o.coarsen, o.coarse_max, o.max_iters,
                  o.stencil, o.metric, o.plane_cycles);
    return buf;
}

}  // namespace

struct mg_server {
    mg_serve_opts o{};
    int device = 0;
    cudaStream_t stream = nullptr;  // every batched step, prologue and epilogue runs here
    cudaStream_t io = nullptr;      // result copies of mg_serve_poll
    std::mutex mu, io_mu;
    std::condition_variable cv_setup, cv_step, cv_done;
    std::deque<Request*> pending;
    std::vector<Request*> ready;
    std::unordered_map<uint64_t, Request*> all;
    size_t bytes_reserved = 0;
    int slots_in_use = 0;
    uint64_t next_ticket = 1;
    bool stop = false;
    // idle hierarchies, most recent first
    std::list<std::pair<std::string, mg_handle*>> cache;
    size_t cache_used = 0;
    // statistics
    long long steps = 0, retired = 0, cache_hits = 0, plan_rebuilds = 0;
    double t_start = 0, t_plan = 0, t_step = 0, t_retire = 0;
    std::vector<std::thread> workers;
    std::thread stepper;
    // evicted hierarchies wait here for their last use (an event on the
    // server stream) and are freed by the reaper thread, off the stepping path
    std::deque<std::pair<mg_handle*, cudaEvent_t>> reap;
    std::condition_variable cv_reap;
    bool reap_stop = false;
    std::thread reaper;
    mg_status fault = MG_OK;        // a CUDA error stops the server
    std::string fault_msg;
};

namespace {

size_t handle_bytes(const mg_handle* h) { return h->bytes; }

// Take an idle hierarchy of the same grid and options, or build one (on the
// calling worker's stream).
mg_status acquire_handle(mg_server* sv, Request* r, cudaStream_t ws) {
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        for (auto it = sv->cache.begin(); it != sv->cache.end(); ++it)
            if (it->first == r->key) {
                r->h = it->second;
                sv->cache_used -= handle_bytes(r->h);
                sv->cache.erase(it);
                sv->cache_hits += 1;
                return MG_OK;
            }
    }
    return mg_setup(&r->grid, &r->opts, ws, &r->h);
}

void release_handle(mg_server* sv, Request* r) {
    if (!r->h) return;
    std::vector<mg_handle*> evict;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->cache.emplace_front(r->key, r->h);
        sv->cache_used += handle_bytes(r->h);
        while (sv->cache_used > sv->o.cache_bytes && !sv->cache.empty()) {
            evict.push_back(sv->cache.back().second);
            sv->cache_used -= handle_bytes(sv->cache.back().second);
            sv->cache.pop_back();
        }
    }
    r->h = nullptr;
    if (evict.empty()) return;
    // last used on the server stream: freed by the reaper once that work is done
    cudaEvent_t e = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess || cudaEventRecord(e, sv->stream) != cudaSuccess) {
        cudaGetLastError();
        if (e) cudaEventDestroy(e);
        for (mg_handle* h : evict) destroy_handle_after(h, sv->stream);
        return;
    }
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        for (size_t i = 0; i < evict.size(); ++i) {
            cudaEvent_t ei = e;
            if (i > 0 && (cudaEventCreateWithFlags(&ei, cudaEventDisableTiming) != cudaSuccess ||
                          cudaEventRecord(ei, sv->stream) != cudaSuccess)) {
                cudaGetLastError();
                ei = nullptr;
            }
            sv->reap.emplace_back(evict[i], ei);
        }
    }
    sv->cv_reap.notify_one();
}

void reaper_loop(mg_server* sv) {
    cudaSetDevice(sv->device);
    for (;;) {
        std::pair<mg_handle*, cudaEvent_t> item;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            sv->cv_reap.wait(lk, [&] { return sv->reap_stop || !sv->reap.empty(); });
            if (sv->reap.empty()) break;   // stopping and drained
            item = sv->reap.front();
            sv->reap.pop_front();
        }
        if (item.second) {
            cudaEventSynchronize(item.second);
            cudaEventDestroy(item.second);
            destroy_handle_after(item.first, nullptr);
        } else {
            destroy_handle_after(item.first, sv->stream);
        }
    }
}

void worker_loop(mg_server* sv) {
    cudaSetDevice(sv->device);
    cudaStream_t ws = nullptr;
    if (cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking) != cudaSuccess) ws = nullptr;
    for (;;) {
        Request* r = nullptr;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            sv->cv_setup.wait(lk, [&] {
                if (sv->stop) return true;
                if (sv->pending.empty() || sv->slots_in_use >= sv->o.max_slots) return false;
                const size_t need = sv->pending.front()->bytes;
                return sv->bytes_reserved + need <= sv->o.max_bytes || sv->slots_in_use == 0;
            });
            if (sv->stop) break;
            r = sv->pending.front();
            sv->pending.pop_front();
            sv->slots_in_use += 1;
            sv->bytes_reserved += r->bytes;
            r->state = RQ_SETUP;
        }
        mg_status st = ws ? acquire_handle(sv, r, ws) : MG_ECUDA;
        const size_t n = r->f.size();
        cudaStream_t hs = nullptr;
        if (st == MG_OK) {
            hs = r->h->stream;
            cudaMemPool_t pool = lib_pool(sv->device);
            if (cudaMallocFromPoolAsync((void**)&r->d_f, sizeof(double) * n, pool, hs) != cudaSuccess ||
                cudaMallocFromPoolAsync((void**)&r->d_x, sizeof(double) * n, pool, hs) != cudaSuccess) {
                cudaGetLastError();
                st = MG_ENOMEM;
            }
        }
        if (st == MG_OK &&
            (cudaMemcpyAsync(r->d_f, r->f.data(), sizeof(double) * n, cudaMemcpyHostToDevice, hs) != cudaSuccess ||
             cudaMemsetAsync(r->d_x, 0, sizeof(double) * n, hs) != cudaSuccess ||
             cudaStreamSynchronize(hs) != cudaSuccess)) {
            st = MG_ECUDA;
        }
        if (st != MG_OK) {   // give back what was taken, then report the failure
            r->err = std::string("set-up: ") + mg_last_error();
            if (st == MG_ECUDA) r->err += std::string(" / ") + cudaGetErrorString(cudaGetLastError());
            if (hs) {
                if (r->d_f) cudaFreeAsync(r->d_f, hs);
                if (r->d_x) cudaFreeAsync(r->d_x, hs);
                cudaStreamSynchronize(hs);
            }
            r->d_f = r->d_x = nullptr;
            if (r->h) release_handle(sv, r);
        }
        std::lock_guard<std::mutex> lk(sv->mu);
        if (st != MG_OK) {
            r->status = st;
            r->rep.status = st;
            r->state = RQ_DONE;
            sv->slots_in_use -= 1;
            sv->bytes_reserved -= r->bytes;
            sv->cv_done.notify_all();
            sv->cv_setup.notify_all();
            continue;
        }
        r->state = RQ_READY;
        sv->ready.push_back(r);
        sv->cv_step.notify_one();
    }
    if (ws) {
        cudaStreamSynchronize(ws);
        cudaStreamDestroy(ws);
    }
}

// Finished requests: their epilogues (gauge, copy into the request's x) are
// queued on the server stream behind an event, and the requests are marked
// done at once; the poll that collects a result waits for its event and
// copies x out.  Slots, hierarchies and the right side are released here;
// the 8 bytes per cell of x stay reserved until the poll.
void retire(mg_server* sv, const std::vector<Request*>& done, Plan** finish_plan) {
    if (done.empty()) return;
    std::vector<mg_handle*> hs;
    std::vector<double*> xs;
    for (Request* r : done) {
        hs.push_back(r->h);
        xs.push_back(r->d_x);
    }
    mg_status st = *finish_plan ? plan_reset(*finish_plan, hs.data(), (int)hs.size(), false)
                                : plan_create(hs.data(), (int)hs.size(), finish_plan, sv->stream, false);
    if (st == MG_OK) st = plan_finish(*finish_plan, xs.data());
    const double t = now_s();
    for (Request* r : done) {
        SolveState& q = r->S;
        q.R.iters = q.it;
        q.R.seconds = t - r->t_submit;   // latency, submit to result
        q.R.model_bytes = model_bytes_per_iteration(r->h) * q.it;
        if (st == MG_OK && (cudaEventCreateWithFlags(&r->ready, cudaEventDisableTiming) != cudaSuccess ||
                            cudaEventRecord(r->ready, sv->stream) != cudaSuccess)) {
            st = MG_ECUDA;
            r->err = std::string("epilogue event: ") + cudaGetErrorString(cudaGetLastError());
        } else if (st != MG_OK && r->err.empty()) {
            r->err = std::string("epilogue: ") + mg_last_error();
        }
        q.R.status = st != MG_OK ? st : q.st;
        r->rep = q.R;
        r->status = (mg_status)q.R.status;
        cudaFreeAsync(r->d_f, sv->stream);
        r->d_f = nullptr;
        release_handle(sv, r);
    }
    std::lock_guard<std::mutex> lk(sv->mu);
    for (Request* r : done) {
        r->state = RQ_DONE;
        sv->slots_in_use -= 1;
        sv->bytes_reserved -= r->bytes - r->x_bytes;
        sv->retired += 1;
    }
    sv->cv_done.notify_all();
    sv->cv_setup.notify_all();
}

void stepper_loop(mg_server* sv) {
    cudaSetDevice(sv->device);
    Plan* start_plan = nullptr;
    Plan* step_plan = nullptr;
    Plan* finish_plan = nullptr;
    std::vector<Request*> active;
    bool changed = true;
    int steps_since_reset = 0;
    int graph_after = 2;   // steps of an unchanged batch before it is captured as a graph
    if (const char* v = std::getenv("MG_SERVE_GRAPH_AFTER")) graph_after = std::atoi(v);
    auto fail = [&](mg_status st) {
        const std::string why = mg_last_error();
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->fault = st;
        sv->fault_msg = why;
        sv->stop = true;
        sv->cv_setup.notify_all();
        sv->cv_done.notify_all();
    };
    for (;;) {
        std::vector<Request*> fresh;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            sv->cv_step.wait(lk, [&] { return sv->stop || !sv->ready.empty() || !active.empty(); });
            if (sv->stop) break;
            fresh.swap(sv->ready);
        }
        double t0 = now_s();
        if (!fresh.empty()) {   // prologue for the newcomers, then they join
            std::vector<mg_handle*> hs;
            std::vector<const double*> fs;
            std::vector<double*> xs;
            std::vector<double> tols;
            for (Request* r : fresh) {
                hs.push_back(r->h);
                fs.push_back(r->d_f);
                xs.push_back(r->d_x);
                tols.push_back(r->tol);
            }
            std::vector<SolveState> S(fresh.size());
            mg_status st = start_plan ? plan_reset(start_plan, hs.data(), (int)hs.size(), false)
                                      : plan_create(hs.data(), (int)hs.size(), &start_plan, sv->stream, false);
            if (st == MG_OK) st = plan_start(start_plan, fs.data(), xs.data(), tols.data(), S.data());
            if (st != MG_OK) {
                fail(st);
                break;
            }
            for (size_t i = 0; i < fresh.size(); ++i) {
                fresh[i]->S = S[i];
                fresh[i]->state = RQ_ACTIVE;
                active.push_back(fresh[i]);
            }
            changed = true;
        }
        double t1 = now_s();
        if (active.empty()) continue;
        if (changed) {
            std::vector<mg_handle*> hs;
            for (Request* r : active) hs.push_back(r->h);
            const mg_status st = step_plan ? plan_reset(step_plan, hs.data(), (int)hs.size())
                                           : plan_create(hs.data(), (int)hs.size(), &step_plan, sv->stream);
            if (st != MG_OK) {
                fail(st);
                break;
            }
            changed = false;
            steps_since_reset = 0;
            std::lock_guard<std::mutex> lk(sv->mu);
            sv->plan_rebuilds += 1;
        }
        double t2 = now_s();
        std::vector<SolveState> S(active.size());
        for (size_t i = 0; i < active.size(); ++i) S[i] = active[i]->S;
        const int nact = plan_check(step_plan, S.data());
        std::vector<Request*> done, still;
        for (size_t i = 0; i < active.size(); ++i) {
            active[i]->S = S[i];
            (S[i].done ? done : still).push_back(active[i]);
        }
        if (nact > 0) {
            const mg_status st = plan_iterate(step_plan, S.data(), steps_since_reset >= graph_after);
            if (st != MG_OK) {
                fail(st);
                break;
            }
            for (size_t i = 0; i < active.size(); ++i)
                if (!S[i].done) active[i]->S = S[i];
            steps_since_reset += 1;
            std::lock_guard<std::mutex> lk(sv->mu);
            sv->steps += 1;
        }
        double t3 = now_s();
        if (!done.empty()) {
            retire(sv, done, &finish_plan);
            active.swap(still);
            changed = true;
        }
        double t4 = now_s();
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            sv->t_start += t1 - t0;
            sv->t_plan += t2 - t1;
            sv->t_step += t3 - t2;
            sv->t_retire += t4 - t3;
        }
    }
    plan_destroy(start_plan);
    plan_destroy(step_plan);
    plan_destroy(finish_plan);
}

}  // namespace

extern "C" {

mg_status mg_serve_default_opts(mg_serve_opts* o) {
    if (!o) return MG_EINVAL;
    std::memset(o, 0, sizeof(*o));
    o->max_bytes = 0;
    o->max_slots = 64;
    o->setup_threads = 4;
    o->cache_bytes = 0;
    o->device = -1;
    return MG_OK;
}

mg_status mg_serve_create(const mg_serve_opts* opts, mg_server** out) {
    if (!out) return MG_EINVAL;
    *out = nullptr;
    mg_serve_opts o;
    if (opts) o = *opts;
    else mg_serve_default_opts(&o);
    if (o.max_slots < 1 || o.setup_threads < 1 || o.setup_threads > 64) {
        set_error("serve: max_slots >= 1 and 1 <= setup_threads <= 64");
        return MG_EINVAL;
    }
    mg_server* sv = new (std::nothrow) mg_server();
    if (!sv) return MG_ENOMEM;
    if (o.device < 0) cudaGetDevice(&o.device);
    sv->device = o.device;
    if (cudaSetDevice(o.device) != cudaSuccess) {
        delete sv;
        set_error("serve: cannot select the device");
        return MG_ECUDA;
    }
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    if (o.max_bytes == 0) o.max_bytes = (size_t)(0.8 * (double)free_b);
    if (o.cache_bytes == 0) o.cache_bytes = o.max_bytes / 4;
    sv->o = o;
    if (cudaStreamCreateWithFlags(&sv->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&sv->io, cudaStreamNonBlocking) != cudaSuccess) {
        if (sv->stream) cudaStreamDestroy(sv->stream);
        delete sv;
        set_error("serve: stream creation failed");
        return MG_ECUDA;
    }
    for (int t = 0; t < o.setup_threads; ++t) sv->workers.emplace_back(worker_loop, sv);
    sv->stepper = std::thread(stepper_loop, sv);
    sv->reaper = std::thread(reaper_loop, sv);
    *out = sv;
    return MG_OK;
}

mg_status mg_serve_submit(mg_server* sv, const mg_grid_desc* grid, const mg_opts* opts, const double* f_host,
                          double tol, uint64_t* ticket) {
    if (!sv || !grid || !f_host || !ticket || !(tol >= 0) || !std::isfinite(tol)) return MG_EINVAL;
    mg_opts o;
    if (opts) o = *opts;
    else mg_default_opts(&o);
    const size_t fp = mg_footprint_bytes(grid, &o);
    if (fp == 0) {
        set_error("serve: invalid grid or options");
        return MG_EINVAL;
    }
    Request* r = new (std::nothrow) Request();
    if (!r) return MG_ENOMEM;
    r->grid = *grid;
    r->opts = o;
    // hierarchies of the serve loop never time schedules (timings taken while
    // other requests run on the GPU would measure the load, not the
    // schedule): they take the one tuned earlier in the process for their
    // shape, else the default (results are the same bits either way)
    r->opts.autotune = 2;
    r->tol = tol;
    const size_t n = (size_t)grid->nr * grid->nth * grid->nph;
    r->f.assign(f_host, f_host + n);
    r->bytes = fp + 2 * sizeof(double) * n;
    r->x_bytes = sizeof(double) * n;
    r->key = key_of(*grid, o);
    r->t_submit = now_s();
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->fault != MG_OK) {
        delete r;
        return sv->fault;
    }
    r->ticket = sv->next_ticket++;
    sv->all[r->ticket] = r;
    sv->pending.push_back(r);
    *ticket = r->ticket;
    sv->cv_setup.notify_one();
    return MG_OK;
}

mg_status mg_serve_poll(mg_server* sv, uint64_t ticket, double* x_host, mg_report* rep) {
    if (!sv) return MG_EINVAL;
    Request* r = nullptr;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        auto it = sv->all.find(ticket);
        if (it == sv->all.end()) {
            set_error("serve: unknown ticket");
            return MG_EINVAL;
        }
        r = it->second;
        if (r->state != RQ_DONE) {
            if (sv->fault != MG_OK) set_error("serve: stopped: " + sv->fault_msg);
            return sv->fault != MG_OK ? sv->fault : MG_EAGAIN;
        }
        sv->all.erase(it);
    }
    mg_status st = r->status;
    {
        std::lock_guard<std::mutex> lk(sv->io_mu);
        if (r->ready) {
            const cudaError_t e = cudaEventSynchronize(r->ready);
            if (e != cudaSuccess) {
                st = MG_ECUDA;
                r->err = std::string("result event: ") + cudaGetErrorString(e);
            }
        }
        if (r->d_x) {
            if (x_host && st != MG_ECUDA &&
                (cudaMemcpyAsync(x_host, r->d_x, r->x_bytes, cudaMemcpyDeviceToHost, sv->io) != cudaSuccess ||
                 cudaStreamSynchronize(sv->io) != cudaSuccess))
                st = MG_ECUDA;
            cudaFreeAsync(r->d_x, sv->io);
        }
        if (r->ready) cudaEventDestroy(r->ready);
    }
    if (rep) {
        *rep = r->rep;
        rep->status = st;
    }
    if (st != MG_OK && st != MG_ENOCONV) set_error("serve: " + r->err);
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (r->d_x) sv->bytes_reserved -= r->x_bytes;
    }
    delete r;
    return st;
}

mg_status mg_serve_stats(mg_server* sv, mg_serve_stats_t* out) {
    if (!sv || !out) return MG_EINVAL;
    std::lock_guard<std::mutex> lk(sv->mu);
    out->queued = (long long)sv->pending.size();
    out->active = sv->slots_in_use;
    out->steps = sv->steps;
    out->retired = sv->retired;
    out->cache_hits = sv->cache_hits;
    out->bytes_reserved = sv->bytes_reserved;
    out->cached_hierarchies = (long long)sv->cache.size();
    out->t_start = sv->t_start;
    out->t_plan = sv->t_plan;
    out->t_step = sv->t_step;
    out->t_retire = sv->t_retire;
    out->plan_rebuilds = sv->plan_rebuilds;
    return MG_OK;
}

void mg_serve_destroy(mg_server* sv) {
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv_setup.notify_all();
    sv->cv_step.notify_all();
    for (auto& t : sv->workers) t.join();
    if (sv->stepper.joinable()) sv->stepper.join();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->reap_stop = true;
    }
    sv->cv_reap.notify_all();
    if (sv->reaper.joinable()) sv->reaper.join();   // frees what it still holds, then stops
    cudaDeviceSynchronize();
    for (auto& kv : sv->all) {
        Request* r = kv.second;
        if (r->d_f) cudaFree(r->d_f);
        if (r->d_x) cudaFree(r->d_x);
        if (r->ready) cudaEventDestroy(r->ready);
        if (r->h) mg_destroy(r->h);
        delete r;
    }
    for (auto& kv : sv->cache) mg_destroy(kv.second);
    if (sv->stream) cudaStreamDestroy(sv->stream);
    if (sv->io) cudaStreamDestroy(sv->io);
    delete sv;
}

}  // extern "C"
