// Continuous-batching request server: transient solves of different sizes
// and step counts are admitted by device-memory budget, kept resident, and
// advanced together. Every scheduler tick picks the residents with the least
// remaining work (cells x steps) until about 64 M cells are in the tick
// (shortest remaining work first, with no resident passed over more than 8
// ticks in a row) and moves each by up to `quantum` steps (all of its steps
// when fewer than two quanta are left), all of them together in one batched
// launch (the batched sweep; measured faster than stepping the large ones
// alone, which serialises them). A tick is launched without waiting: the host
// builds the next one while it runs, then waits for it and hands its finished
// requests to read-back. Requests that arrive while others run join at the
// next tick. Four more threads move inputs to the device and results back, each
// on its own stream, while the ticks run; a finished request's memory is
// released as soon as its result is on the host.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/wfa.h"

namespace wfa {
void set_error(const char* fmt, ...);
int grid_rebind_stream(wfa_grid g, cudaStream_t st);
int grid_move_stream(wfa_grid g, cudaStream_t st);
int batch_launch(wfa_grid* gs, const long long* steps, int count, int slot, bool wait);
int batch_wait(cudaStream_t st, int slot);
}

namespace {

using clk = std::chrono::steady_clock;

constexpr double TICK_CELLS = 64.0 * 1024 * 1024;   // cells advanced per tick, at least
constexpr int MAX_SKIP = 8;                          // ticks a resident may be passed over
constexpr int PREP_THREADS = 4;                      // set-up / read-back threads (host copies run in parallel)

struct Req {
    long long ticket = 0;
    wfa_request spec{};   // T0_host / k_host are read when the request is set up
    wfa_grid g = nullptr;
    long long remaining = 0;
    int skipped = 0;   // ticks in a row this resident was not advanced
    size_t bytes = 0;
    int state = 0;   // 0 queued, 1 resident, 2 done, -1 failed
    std::string err;
    clk::time_point t_submit, t_done;
};

// Device bytes a request holds while resident (two field buffers with their
// halo, per-cell k, the dense staging buffer).
size_t device_bytes(const wfa_request& r) {
    const long long halo = 8;
    const long long es = r.storage == WFA_BF16 ? 2 : 4;
    const long long align = 128 / es;
    const long long px = ((r.nx + 2 * halo + align - 1) / align) * align;
    const long long padded = px * (r.ny + 2 * halo) * (r.nz + 2 * halo);
    const long long dense = (long long)r.nx * r.ny * r.nz;
    size_t b = (size_t)(2 * padded * es + dense * 4 + 64 * 1024);
    if (r.k_host) b += (size_t)padded * 4;
    return b;
}

}  // namespace

// One tick: the residents it advances, by how many steps, and those it
// finishes. Ticks are launched without waiting, so the host builds the next
// tick (selection, descriptors, graph) while this one runs on the GPU.
struct Tick {
    bool live = false;   // launched, not yet waited for
    int slot = 0;        // batch context (two alternate)
    std::vector<Req*> work, finished;
    double upd = 0.0;    // cell updates
    clk::time_point t0;
};

struct wfa_server_s {
    size_t budget = 0;
    int max_resident = 1024;
    long long quantum = 64;
    int device = 0;
    cudaStream_t stream = nullptr;   // ticks
    cudaStream_t prep[PREP_THREADS] = {};   // set-up and read-back, beside the ticks

    std::mutex mu;
    std::condition_variable cv_work, cv_done, cv_prep;
    std::deque<Req*> pending;        // submitted, not admitted
    std::deque<Req*> to_setup;       // admitted, inputs not yet on the device
    std::vector<Req*> ready;         // on the device, joining at the next tick
    std::vector<Req*> resident;      // advanced by the ticks
    std::deque<Req*> to_retire;      // finished, result not yet on the host
    std::unordered_map<long long, Req*> all;
    long long next_ticket = 1;
    int in_setup = 0;                // taken from to_setup, not yet ready
    bool stop = false, sched_done = false;
    std::thread th, prep_th[PREP_THREADS];

    // stats
    long long submitted = 0, admitted = 0, completed = 0, rejected = 0, ticks = 0;
    double cell_updates = 0.0, busy_s = 0.0;
    size_t used = 0, peak_used = 0;
    std::vector<double> latencies;

    clk::time_point busy_end{};     // when the last waited tick ended

    void run();
    void settle(Tick& t, int rc, const std::string& why);
    void prep_loop(int w);
    int setup(Req* r, cudaStream_t st);
    int setup_grid(Req* r, cudaStream_t st);
    void finish(Req* r, bool ok, const std::string& why);
};

int wfa_server_s::setup(Req* r, cudaStream_t st) {
    nvtxRangePushA("wfa_server_setup");
    const int rc = setup_grid(r, st);
    nvtxRangePop();
    return rc;
}

int wfa_server_s::setup_grid(Req* r, cudaStream_t st) {
    const wfa_request& s = r->spec;
    int rc = wfa_create_grid(s.nx, s.ny, s.nz, s.hx, s.hy, s.hz, s.storage, st, &r->g);
    if (rc) return rc;
    for (int f = 0; f < 6 && !rc; ++f) rc = wfa_set_bc(r->g, f, s.bc_kind[f], s.bc_value[f]);
    if (!rc) rc = wfa_set_coeffs(r->g, s.k_host, s.k_uniform, s.ux, s.uy, s.uz);
    if (!rc) rc = wfa_set_field(r->g, s.T0_host);
    double dt = s.dt;
    if (!rc && !(dt > 0)) {
        double lim = 0;
        rc = wfa_stability_dt(r->g, &lim);
        dt = std::isfinite(lim) ? 0.9 * lim : 1.0;
    }
    if (!rc) rc = wfa_set_dt(r->g, dt);
    return rc;
}

void wfa_server_s::finish(Req* r, bool ok, const std::string& why) {
    if (r->g) {
        wfa_destroy_grid(r->g);
        r->g = nullptr;
    }
    std::lock_guard<std::mutex> lk(mu);
    r->state = ok ? 2 : -1;
    r->err = why;
    r->t_done = clk::now();
    used -= r->bytes;
    if (ok) {
        ++completed;
        latencies.push_back(std::chrono::duration<double>(r->t_done - r->t_submit).count());
    }
    cv_done.notify_all();
    cv_work.notify_all();   // memory freed: more requests may be admitted
}

// A set-up / read-back thread (one of PREP_THREADS): inputs of admitted
// requests go to the device and results of finished ones come back, on the
// thread's own stream, while the scheduler's ticks run, so the GPU does not
// wait for host transfers.
void wfa_server_s::prep_loop(int w) {
    cudaSetDevice(device);
    for (;;) {
        Req* r = nullptr;
        bool retire = false;
        {
            std::unique_lock<std::mutex> lk(mu);
            cv_prep.wait(lk, [&] { return sched_done || !to_setup.empty() || !to_retire.empty(); });
            if (!to_retire.empty()) {   // finishing first: it frees memory and completes a request
                r = to_retire.front();
                to_retire.pop_front();
                retire = true;
            } else if (!to_setup.empty()) {
                r = to_setup.front();
                to_setup.pop_front();
                ++in_setup;
            } else {
                return;   // the scheduler has stopped and nothing is left to do
            }
        }
        if (retire) {
            // its last tick has been waited for: nothing of it is pending on the tick stream
            int rc = r->err.empty() ? wfa::grid_move_stream(r->g, prep[w]) : WFA_ERR_STATE;
            if (!rc) rc = wfa_read_field(r->g, r->spec.out_host);
            finish(r, rc == 0, rc ? (r->err.empty() ? std::string(wfa_last_error()) : r->err) : std::string());
            continue;
        }
        int rc = setup(r, prep[w]);
        if (!rc) rc = wfa::grid_rebind_stream(r->g, stream);
        if (rc) finish(r, false, wfa_last_error());
        std::lock_guard<std::mutex> lk(mu);
        if (!rc) ready.push_back(r);
        --in_setup;
        cv_work.notify_all();
    }
}

// Waits for a launched tick; its finished requests go to read-back. On
// failure every request of the tick fails and leaves the resident set
// (the caller has waited for any later tick that still used them).
void wfa_server_s::settle(Tick& t, int rc, const std::string& why) {
    const auto t1 = clk::now();
    std::lock_guard<std::mutex> lk(mu);
    ++ticks;
    busy_s += std::chrono::duration<double>(t1 - std::max(t.t0, busy_end)).count();
    busy_end = t1;
    if (!rc) {
        cell_updates += t.upd;
    } else {
        for (Req* r : t.work) {
            if (r->err.empty()) r->err = why.empty() ? "tick failed" : why;
            auto it = std::find(resident.begin(), resident.end(), r);
            if (it != resident.end()) {
                resident.erase(it);
                t.finished.push_back(r);
            }
        }
    }
    for (Req* r : t.finished) to_retire.push_back(r);
    t.live = false;
    t.work.clear();
    t.finished.clear();
    cv_prep.notify_all();
}

void wfa_server_s::run() {
    cudaSetDevice(device);
    std::vector<wfa_grid> gs;
    std::vector<long long> steps;
    Tick ticks_[2];
    int cur = 0;   // ticks_[cur] is the next to launch, ticks_[1 - cur] may be in flight
    auto wait_tick = [&](Tick& t) {
        const int rc = wfa::batch_wait(stream, t.slot);
        settle(t, rc, rc ? std::string(wfa_last_error()) : std::string());
        return rc;
    };
    for (;;) {
        Tick& prev = ticks_[1 - cur];
        std::vector<Req*> work;
        {
            std::unique_lock<std::mutex> lk(mu);
            if (!prev.live)
                cv_work.wait(lk, [&] {
                    return stop || !pending.empty() || !resident.empty() || !ready.empty();
                });
            // admission: first come, first served, while memory and slots allow
            // (a slot is held from admission on: queued for set-up, in set-up,
            // ready or resident)
            while (!pending.empty() &&
                   (int)(resident.size() + ready.size() + to_setup.size()) + in_setup < max_resident) {
                Req* r = pending.front();
                if (used + r->bytes > budget) break;
                pending.pop_front();
                used += r->bytes;
                peak_used = std::max(peak_used, used);
                r->state = 1;
                ++admitted;
                to_setup.push_back(r);
                cv_prep.notify_all();
            }
            for (Req* r : ready) resident.push_back(r);
            ready.clear();
            if (resident.empty()) {
                if (prev.live) {   // finish the tick in flight first: it frees memory and slots
                    lk.unlock();
                    wait_tick(prev);
                    continue;
                }
                if (stop && pending.empty() && to_setup.empty() && in_setup == 0) {
                    sched_done = true;
                    cv_prep.notify_all();
                    break;
                }
                // nothing to advance yet: wait for set-up (or new requests)
                cv_work.wait_for(lk, std::chrono::milliseconds(2));
                continue;
            }
            work = resident;
        }
        // this tick: the residents with the least remaining work first, up to
        // about TICK_CELLS cells (enough to fill the GPU), plus any resident
        // passed over MAX_SKIP ticks in a row; one that is nearly done gets
        // all its remaining steps (remaining work already counts the tick in
        // flight)
        auto cells = [](const Req* r) { return (double)r->spec.nx * r->spec.ny * r->spec.nz; };
        std::stable_sort(work.begin(), work.end(),
                         [&](const Req* a, const Req* b) { return cells(a) * a->remaining < cells(b) * b->remaining; });
        Tick& t = ticks_[cur];
        t.work.clear();
        t.finished.clear();
        t.upd = 0.0;
        double sel_cells = 0.0;
        for (Req* r : work) {
            if (sel_cells < TICK_CELLS || r->skipped >= MAX_SKIP) {
                t.work.push_back(r);
                sel_cells += cells(r);
                r->skipped = 0;
            } else {
                ++r->skipped;
            }
        }
        gs.clear();
        steps.clear();
        std::vector<long long> q_of(t.work.size());
        for (size_t i = 0; i < t.work.size(); ++i) {
            Req* r = t.work[i];
            const long long q = r->remaining <= 2 * quantum ? r->remaining : quantum;
            q_of[i] = q;
            t.upd += (double)q * cells(r);
            gs.push_back(r->g);
            steps.push_back(q);
        }
        t.t0 = clk::now();
        t.slot = cur;
        nvtxRangePushA("wfa_server_tick");
        const int rc = wfa::batch_launch(gs.data(), steps.data(), (int)gs.size(), t.slot, false);
        nvtxRangePop();
        const std::string why = rc ? std::string(wfa_last_error()) : std::string();
        {
            std::lock_guard<std::mutex> lk(mu);
            for (size_t i = 0; i < t.work.size(); ++i) {
                Req* r = t.work[i];
                if (!rc && (r->remaining -= q_of[i]) <= 0) {
                    resident.erase(std::find(resident.begin(), resident.end(), r));
                    t.finished.push_back(r);
                }
            }
        }
        t.live = !rc;
        // the previous tick has run meanwhile: retire what it finished
        int rc_prev = prev.live ? wait_tick(prev) : 0;
        if (rc_prev && t.live) {   // its requests may be in this tick too: fail both
            wfa::batch_wait(stream, t.slot);
            settle(t, rc_prev, "an earlier tick failed");
        }
        if (rc) {   // nothing of this tick runs: its requests fail
            t.live = true;
            t.t0 = clk::now();
            settle(t, rc, why);
        }
        cur = 1 - cur;
    }
}

extern "C" {

int wfa_server_create(size_t hbm_budget_bytes, int max_resident, long long quantum, wfa_server* out) {
    if (!out || hbm_budget_bytes == 0 || max_resident < 0 || quantum < 0) {
        wfa::set_error("wfa_server_create: bad arguments");
        return WFA_ERR_ARG;
    }
    wfa_server_s* s = new wfa_server_s();
    s->budget = hbm_budget_bytes;
    s->max_resident = max_resident ? max_resident : 1024;
    s->quantum = quantum ? quantum : 64;
    cudaGetDevice(&s->device);
    cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    for (int w = 0; w < PREP_THREADS && e == cudaSuccess; ++w)
        e = cudaStreamCreateWithFlags(&s->prep[w], cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        wfa::set_error("cudaStreamCreate failed: %s", cudaGetErrorString(e));
        if (s->stream) cudaStreamDestroy(s->stream);
        for (cudaStream_t p : s->prep)
            if (p) cudaStreamDestroy(p);
        delete s;
        return WFA_ERR_CUDA;
    }
    s->th = std::thread([s] { s->run(); });
    for (int w = 0; w < PREP_THREADS; ++w) s->prep_th[w] = std::thread([s, w] { s->prep_loop(w); });
    *out = s;
    return WFA_OK;
}

int wfa_server_submit(wfa_server s, const wfa_request* r, long long* ticket) {
    if (!s || !r || !ticket || !r->T0_host || !r->out_host || r->steps < 0 || r->nx < 2 || r->ny < 2 ||
        r->nz < 2) {
        wfa::set_error("wfa_server_submit: bad arguments");
        return WFA_ERR_ARG;
    }
    Req* q = new Req();
    q->spec = *r;
    q->bytes = device_bytes(*r);
    q->remaining = r->steps;
    q->t_submit = clk::now();
    std::lock_guard<std::mutex> lk(s->mu);
    if (q->bytes > s->budget) {
        ++s->rejected;
        delete q;
        wfa::set_error("request needs %zu bytes, above the server budget %zu", device_bytes(*r), s->budget);
        return WFA_ERR_BUDGET;
    }
    q->ticket = s->next_ticket++;
    s->all[q->ticket] = q;
    s->pending.push_back(q);
    ++s->submitted;
    *ticket = q->ticket;
    s->cv_work.notify_one();
    return WFA_OK;
}

int wfa_server_poll(wfa_server s, long long ticket, int* done) {
    if (!s || !done) return WFA_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) {
        wfa::set_error("unknown ticket %lld", ticket);
        return WFA_ERR_ARG;
    }
    const Req* r = it->second;
    *done = r->state == 2 ? 1 : (r->state < 0 ? -1 : 0);
    if (r->state < 0) wfa::set_error("%s", r->err.c_str());
    return WFA_OK;
}

int wfa_server_latency(wfa_server s, long long ticket, double* seconds) {
    if (!s || !seconds) return WFA_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) {
        wfa::set_error("unknown ticket %lld", ticket);
        return WFA_ERR_ARG;
    }
    const Req* r = it->second;
    if (r->state != 2) {
        wfa::set_error("ticket %lld is not done", ticket);
        return WFA_ERR_STATE;
    }
    *seconds = std::chrono::duration<double>(r->t_done - r->t_submit).count();
    return WFA_OK;
}

int wfa_server_wait(wfa_server s, long long ticket, double timeout_s) {
    if (!s) return WFA_ERR_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) {
        wfa::set_error("unknown ticket %lld", ticket);
        return WFA_ERR_ARG;
    }
    Req* r = it->second;
    const auto deadline = clk::now() + std::chrono::duration_cast<clk::duration>(
                                           std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 1e9));
    if (!s->cv_done.wait_until(lk, deadline, [&] { return r->state == 2 || r->state < 0; })) {
        wfa::set_error("ticket %lld not done within %.3f s", ticket, timeout_s);
        return WFA_ERR_TIMEOUT;
    }
    if (r->state < 0) {
        wfa::set_error("%s", r->err.c_str());
        return WFA_ERR_STATE;
    }
    return WFA_OK;
}

int wfa_server_stats_get(wfa_server s, wfa_server_stats* st) {
    if (!s || !st) return WFA_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    memset(st, 0, sizeof *st);
    st->submitted = s->submitted;
    st->admitted = s->admitted;
    st->completed = s->completed;
    st->rejected = s->rejected;
    st->ticks = s->ticks;
    st->cell_updates = s->cell_updates;
    st->busy_seconds = s->busy_s;
    st->resident_bytes = s->used;
    st->peak_resident_bytes = s->peak_used;
    if (!s->latencies.empty()) {
        std::vector<double> v = s->latencies;
        std::sort(v.begin(), v.end());
        auto pct = [&](double p) {
            const double pos = p * (v.size() - 1);
            const size_t lo = (size_t)pos;
            const size_t hi = std::min(lo + 1, v.size() - 1);
            return v[lo] + (pos - lo) * (v[hi] - v[lo]);
        };
        st->p50_latency_s = pct(0.50);
        st->p99_latency_s = pct(0.99);
        double sum = 0;
        for (double x : v) sum += x;
        st->mean_latency_s = sum / v.size();
    }
    return WFA_OK;
}

int wfa_server_destroy(wfa_server s) {
    if (!s) return WFA_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv_work.notify_all();
    }
    if (s->th.joinable()) s->th.join();   // resident work finished; results queued for read-back
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->cv_prep.notify_all();
    }
    for (std::thread& t : s->prep_th)
        if (t.joinable()) t.join();
    for (auto& kv : s->all) delete kv.second;
    cudaStreamDestroy(s->stream);
    for (cudaStream_t p : s->prep) cudaStreamDestroy(p);
    delete s;
    return WFA_OK;
}

}  // extern "C"
