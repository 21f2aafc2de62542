// server.cu -- continuous-batching localization server.
//
// One worker thread owns an Engine (engine.cuh) and a CUDA stream.  Clients
// submit requests (a map handle, a scan that is copied, ranges, options) and
// poll tickets.  The worker runs the engine's device loop until a search
// finishes or fails or a request arrives or is cancelled (a flag in mapped
// host memory the loop polls every iteration); then it reports finished
// searches and admits queued requests into free
// search slots as long as the device-memory budget allows -- the shared
// frontier pool is charged once, each admitted search its scan, rotation
// tables and frontier arrays -- so requests that arrive while others run join
// the next iteration and their work shares the same launches.  Finished
// searches release their memory and slot at once.  Because a search's
// trajectory depends only on its own batches, every result is the one
// bbs_localize returns for the same request alone.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "engine.cuh"

namespace bbs {

namespace {

double now_ms()
{
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Request {
    uint64_t ticket = 0;
    const bbs_maps* maps = nullptr;
    std::vector<float> scan;
    bbs_ranges ranges{};
    bool has_ranges = false;
    bbs_opts opts{};
    double t_submit = 0;
    size_t est_bytes = 0;
};

struct Finished {
    bbs_result res{};
    double t_submit = 0, t_done = 0;
};

}  // namespace

}  // namespace bbs

struct bbs_server {
    int device = 0;
    cudaStream_t st = nullptr;
    bbs::Engine* engine = nullptr;
    size_t budget = 0;
    size_t in_use = 0;
    int max_active = 32;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<bbs::Request> queue;
    std::unordered_map<uint64_t, bbs::Finished> done;
    std::unordered_map<uint64_t, int> running;        // ticket -> engine slot
    std::unordered_map<int, bbs::Request> slot_req;    // engine slot -> request (worker thread only)
    std::unordered_set<uint64_t> cancels;
    std::unordered_set<uint64_t> uncollected;         // submitted tickets whose result has not been polled
    std::vector<double> latencies;
    uint64_t next_ticket = 1;
    int64_t submitted = 0, rejected = 0, peak_active = 0;
    double t_first = -1, t_last = 0;
    double probes = 0;
    int fatal = 0;
    char fatal_msg[512] = {0};
    bool stop = false;
    std::thread worker;
};

namespace bbs {

namespace {

// host-side d_max and grid of a request, to estimate its device memory
size_t estimate_request(bbs_server* S, const Request& q)
{
    double dm = 0.0;
    const int64_t k = (int64_t)(q.scan.size() / 3);
    for (int64_t i = 0; i < k; ++i) {
        const double x = q.scan[3 * i], y = q.scan[3 * i + 1], z = q.scan[3 * i + 2];
        dm = std::max(dm, std::sqrt((x * x + y * y) + z * z));
    }
    if (q.opts.d_max > 0.0) dm = q.opts.d_max;
    bbs_ranges rg;
    if (q.has_ranges) rg = q.ranges;
    else default_ranges(q.maps, &rg);
    HostGrid g;
    if (grid_build((double)q.maps->r, q.maps->levels, dm, &rg, q.opts.flags, &g) < 0) return 0;   // rejected by add()
    return S->engine->estimate_bytes(k, g);
}

void worker_main(bbs_server* S)
{
    cudaSetDevice(S->device);
    std::vector<int> fin;
    for (;;) {
        std::vector<Request> admit;
        std::vector<std::pair<int, uint64_t>> to_cancel;
        {
            std::unique_lock<std::mutex> lock(S->mu);
            S->cv_work.wait(lock, [&] { return S->stop || !S->queue.empty() || S->engine->used_count() > 0; });
            if (S->stop) break;
            // arrivals and cancels after this point wake the device loop again
            *S->engine->wake_flag() = 0;
            for (uint64_t t : S->cancels) {
                auto it = S->running.find(t);
                if (it != S->running.end()) to_cancel.push_back({it->second, t});
            }
            S->cancels.clear();
            // admission in arrival order while a slot and the memory budget allow
            const int used = S->engine->used_count();
            while (!S->queue.empty() && used + (int)admit.size() < S->max_active) {
                Request& q = S->queue.front();
                if (S->in_use + q.est_bytes > S->budget) break;   // wait until memory frees up
                S->in_use += q.est_bytes;
                admit.push_back(std::move(q));
                S->queue.pop_front();
            }
        }
        for (auto& c : to_cancel) {
            bbs_result r;
            S->engine->cancel(c.first, BBS_ECANCELED, &r);
            std::lock_guard<std::mutex> lock(S->mu);
            Request& q = S->slot_req[c.first];
            S->in_use -= q.est_bytes;
            Finished f;
            f.res = r;
            f.t_submit = q.t_submit;
            f.t_done = now_ms();
            S->done[c.second] = f;
            S->running.erase(c.second);
            S->slot_req.erase(c.first);
            S->cv_done.notify_all();
        }
        for (auto& q : admit) {
            int slot = -1;
            const int rc = S->engine->add(q.maps, q.scan.data(), (int64_t)(q.scan.size() / 3), 0,
                                          q.has_ranges ? &q.ranges : nullptr, &q.opts, q.ticket, &slot);
            std::lock_guard<std::mutex> lock(S->mu);
            if (rc < 0) {
                Finished f;
                f.res.status = rc;
                f.res.num_points = (int32_t)(q.scan.size() / 3);
                f.t_submit = q.t_submit;
                f.t_done = now_ms();
                S->in_use -= q.est_bytes;
                S->done[q.ticket] = f;
                S->cv_done.notify_all();
                continue;
            }
            S->running[q.ticket] = slot;
            S->slot_req[slot] = std::move(q);
        }
        {
            std::lock_guard<std::mutex> lock(S->mu);
            S->peak_active = std::max<int64_t>(S->peak_active, (int64_t)S->running.size());
        }
        int rc = S->engine->start();
        fin.clear();
        // the device loop runs until a search finishes or fails, or a request
        // arrives or is cancelled (the wake flag): then admission again
        if (rc >= 0) rc = S->engine->iterate(1 << 20, &fin);
        if (rc < 0) {
            std::lock_guard<std::mutex> lock(S->mu);
            S->fatal = rc;
            std::snprintf(S->fatal_msg, sizeof(S->fatal_msg), "%s", bbs_last_error());
            S->stop = true;
            S->cv_done.notify_all();
            break;
        }
        for (int slot : fin) {
            bbs_result r;
            S->engine->finalize(slot, &r);
            std::lock_guard<std::mutex> lock(S->mu);
            Request& q = S->slot_req[slot];
            S->in_use -= q.est_bytes;
            Finished f;
            f.res = r;
            f.t_submit = q.t_submit;
            f.t_done = now_ms();
            S->latencies.push_back(f.t_done - f.t_submit);
            S->t_last = std::max(S->t_last, f.t_done);
            S->probes += (double)r.probes;
            S->done[q.ticket] = f;
            S->running.erase(q.ticket);
            S->slot_req.erase(slot);
            S->cv_done.notify_all();
        }
    }
}

}  // namespace

}  // namespace bbs

using namespace bbs;

extern "C" {

int bbs_server_create(const bbs_server_opts* o, bbs_server** out)
{
    clear_error();
    if (!out) return set_error(BBS_EINVAL, "server_create: out is NULL");
    *out = nullptr;
    bbs_server* S = new bbs_server;
    cudaGetDevice(&S->device);
    S->budget = (o && o->mem_budget) ? o->mem_budget : ((size_t)8 << 30);
    S->max_active = (o && o->max_active > 0) ? o->max_active : 32;
    if (S->max_active > MAX_SLOTS) {
        delete S;
        return set_error(BBS_EINVAL, "server_create: max_active above %d", MAX_SLOTS);
    }
    const int64_t pool = (o && o->max_frontier > 0) ? o->max_frontier : ((int64_t)1 << 24);
    if (cudaStreamCreateWithFlags(&S->st, cudaStreamNonBlocking) != cudaSuccess) {
        delete S;
        return set_error(BBS_ECUDA, "server_create: cannot create a stream");
    }
    S->engine = new Engine(S->st, S->max_active, pool, false);
    int rc = S->engine->init();
    if (rc == BBS_OK && S->engine->fixed_bytes() > S->budget)
        rc = set_error(BBS_ENOMEM, "server_create: the frontier pool needs %zu bytes, budget %zu",
                       S->engine->fixed_bytes(), S->budget);
    if (rc == BBS_OK) rc = S->engine->set_exit_on_finish(true);
    if (rc == BBS_OK && cudaStreamSynchronize(S->st) != cudaSuccess) rc = set_error(BBS_ECUDA, "server_create: init");
    if (rc < 0) {
        delete S->engine;
        cudaStreamDestroy(S->st);
        delete S;
        return rc;
    }
    S->in_use = S->engine->fixed_bytes();
    S->worker = std::thread(worker_main, S);
    *out = S;
    return BBS_OK;
}

int bbs_server_submit(bbs_server* S, const bbs_maps* maps, const float* scan_xyz, int64_t k,
                      const bbs_ranges* ranges, const bbs_opts* opts, uint64_t* ticket)
{
    clear_error();
    if (!S || !maps || !ticket || k < 0 || (k > 0 && !scan_xyz)) return set_error(BBS_EINVAL, "server_submit: bad arguments");
    if (maps->device != S->device) return set_error(BBS_EINVAL, "server_submit: maps live on another device");
    Request q;
    q.maps = maps;
    q.scan.assign(scan_xyz, scan_xyz + 3 * k);
    if (ranges) {
        q.ranges = *ranges;
        q.has_ranges = true;
    }
    if (opts) q.opts = *opts;
    q.opts.cuda_stream = nullptr;
    q.opts.flags &= ~BBS_TIME_KERNELS;
    q.t_submit = now_ms();
    std::lock_guard<std::mutex> lock(S->mu);
    if (S->fatal) return set_error(S->fatal, "server: %s", S->fatal_msg);
    q.ticket = S->next_ticket++;
    *ticket = q.ticket;
    S->uncollected.insert(q.ticket);
    S->submitted++;
    if (S->t_first < 0) S->t_first = q.t_submit;
    q.est_bytes = estimate_request(S, q);
    if (q.est_bytes + S->engine->fixed_bytes() > S->budget) {
        // can never fit: fails now instead of waiting forever
        Finished f;
        f.res.status = BBS_ENOMEM;
        f.res.num_points = (int32_t)k;
        f.t_submit = f.t_done = q.t_submit;
        S->done[q.ticket] = f;
        S->rejected++;
        S->cv_done.notify_all();
        return BBS_OK;
    }
    S->queue.push_back(std::move(q));
    *S->engine->wake_flag() = 1;   // a running device loop ends after its current iteration
    S->cv_work.notify_one();
    return BBS_OK;
}

int bbs_server_poll(bbs_server* S, uint64_t ticket, int wait_ms, bbs_result* out)
{
    clear_error();
    if (!S || !out) return set_error(BBS_EINVAL, "server_poll: bad arguments");
    std::unique_lock<std::mutex> lock(S->mu);
    // a ticket never issued, or whose result was already returned, would never be ready
    if (!S->uncollected.count(ticket))
        return set_error(BBS_EINVAL, "server_poll: ticket %llu is unknown or already collected",
                         (unsigned long long)ticket);
    auto ready = [&] { return S->done.count(ticket) > 0 || S->fatal != 0; };
    if (!ready() && wait_ms != 0) {
        if (wait_ms < 0) S->cv_done.wait(lock, ready);
        else S->cv_done.wait_for(lock, std::chrono::milliseconds(wait_ms), ready);
    }
    auto it = S->done.find(ticket);
    if (it == S->done.end()) {
        if (S->fatal) return set_error(S->fatal, "server: %s", S->fatal_msg);
        return BBS_PENDING;
    }
    *out = it->second.res;
    out->ms_total = it->second.t_done - it->second.t_submit;   // submission to result
    const int st = out->status;
    S->done.erase(it);
    S->uncollected.erase(ticket);
    if (st < 0) set_error(st, "server: request %llu failed", (unsigned long long)ticket);
    return st;
}

int bbs_server_cancel(bbs_server* S, uint64_t ticket)
{
    clear_error();
    if (!S) return set_error(BBS_EINVAL, "server_cancel: NULL server");
    std::lock_guard<std::mutex> lock(S->mu);
    for (auto it = S->queue.begin(); it != S->queue.end(); ++it)
        if (it->ticket == ticket) {
            Finished f;
            f.res.status = BBS_ECANCELED;
            f.res.num_points = (int32_t)(it->scan.size() / 3);
            f.t_submit = it->t_submit;
            f.t_done = now_ms();
            S->done[ticket] = f;
            S->queue.erase(it);
            S->cv_done.notify_all();
            return BBS_OK;
        }
    if (S->running.count(ticket)) {
        S->cancels.insert(ticket);
        *S->engine->wake_flag() = 1;   // the device loop returns so that the cancel takes effect
        S->cv_work.notify_one();
        return BBS_OK;
    }
    return set_error(BBS_EINVAL, "server_cancel: ticket %llu is not queued or running", (unsigned long long)ticket);
}

int bbs_server_stats(bbs_server* S, bbs_server_counters* out)
{
    clear_error();
    if (!S || !out) return set_error(BBS_EINVAL, "server_stats: bad arguments");
    std::lock_guard<std::mutex> lock(S->mu);
    std::memset(out, 0, sizeof(*out));
    out->submitted = S->submitted;
    out->completed = (int64_t)S->latencies.size();
    out->active = (int64_t)S->running.size();
    out->queued = (int64_t)S->queue.size();
    out->rejected = S->rejected;
    out->peak_active = S->peak_active;
    std::vector<double> l = S->latencies;
    if (!l.empty()) {
        std::sort(l.begin(), l.end());
        auto pct = [&](double p) {
            const size_t i = (size_t)std::min<double>((double)l.size() - 1, std::floor(p * (double)(l.size() - 1) + 0.5));
            return l[i];
        };
        out->p50_ms = pct(0.50);
        out->p99_ms = pct(0.99);
        double sum = 0;
        for (double v : l) sum += v;
        out->mean_ms = sum / (double)l.size();
        const double span = S->t_last - S->t_first;
        out->throughput_rps = span > 0 ? (double)l.size() / (span / 1e3) : 0.0;
        out->probes_per_s = span > 0 ? S->probes / (span / 1e3) : 0.0;
    }
    out->mem_in_use = S->in_use;
    out->mem_budget = S->budget;
    return BBS_OK;
}

void bbs_server_destroy(bbs_server* S)
{
    if (!S) return;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->worker.joinable()) S->worker.join();
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(S->device);
    delete S->engine;
    cudaStreamSynchronize(S->st);
    cudaStreamDestroy(S->st);
    if (prev >= 0) cudaSetDevice(prev);
    delete S;
}

}  // extern "C"
