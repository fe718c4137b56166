// Continuous-batching query server over one resident index.
//
// The index (data set, projections, leaf layout) stays on the device.  A
// client submits a request (query rows on the host, Algorithm 2 options) and
// gets a ticket at once.  `slots` worker threads, each with its own CUDA
// stream and scratch buffers, take the oldest waiting request plus every
// later waiting request with identical options, up to `max_batch_queries`
// rows and within the device-memory budget, and run them as one batch; a
// request that arrives while batches run joins the next free slot, so the
// device works on several batches at once.  Every request's results equal
// those of pmlsh_knn on that request alone (each query's computation does
// not depend on the batch it rides in).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <string>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "pmlsh_impl.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket = 0;
    int64_t nq = 0;
    pmlsh_knn_opts opts{};
    std::vector<float> Q;          // [nq][d] host copy
    std::vector<int64_t> ids;      // [nq][k]
    std::vector<float> dists;      // [nq][k]
    std::vector<float> err;        // [nq][k] |returned - FP64 distance|
    pmlsh_status status = PMLSH_OK;
    std::string error;
    bool done = false;
    Clock::time_point t_submit, t_done;
};

bool same_opts(const pmlsh_knn_opts &a, const pmlsh_knn_opts &b)
{
    return a.k == b.k && a.c == b.c && a.alpha1 == b.alpha1 && a.beta == b.beta && a.r_min == b.r_min &&
           a.precision == b.precision && a.t == b.t && a.stop_rule == b.stop_rule;
}

}  // namespace

struct pmlsh_server {
    pmlsh_index *ix = nullptr;
    pmlsh_serve_opts opts{};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Request>> queue;
    std::map<uint64_t, std::shared_ptr<Request>> tickets;
    uint64_t next_ticket = 1;
    bool stopping = false;
    // device memory of the slots' workspaces: what each holds now, and the
    // growth charged at admission to the batches still running
    std::vector<int64_t> resident;
    int64_t reserved = 0;
    int inflight = 0;
    uint64_t trim_epoch = 0;   // idle slots release their workspaces when it moves
    int64_t peak_bytes = 0;
    // statistics
    int64_t submitted = 0, completed = 0, queries = 0, batches = 0, deferred = 0, canceled = 0;
    std::vector<double> lat_ms;
    Clock::time_point t_first{}, t_last{};
    bool any_done = false;
    std::vector<std::thread> workers;

    int64_t held() const
    {
        int64_t b = reserved;
        for (int64_t r : resident) b += r;
        return b;
    }

    // Memory admission: a batch is admitted when the slots' resident
    // workspaces, the growth already charged to running batches and this
    // batch's own growth of its slot's workspace (pm_knn_work_growth) fit
    // mem_budget_bytes.  When nothing runs and a batch does not fit, the idle
    // slots release their workspaces first; a batch that does not fit even
    // then runs alone.  A slot whose batch left the total above the budget
    // releases its workspace afterwards.
    void worker(int slot)
    {
        cudaSetDevice(device);
        cudaStream_t st = nullptr;
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        KnnWork work;
        uint64_t seen_epoch = 0;
        for (;;) {
            std::vector<std::shared_ptr<Request>> batch;
            int64_t growth = 0;
            {
                std::unique_lock<std::mutex> lk(mu);
                for (;;) {
                    if (trim_epoch != seen_epoch) {
                        // a batch waits for the memory this idle slot holds
                        seen_epoch = trim_epoch;
                        if (resident[slot] > 0) {
                            lk.unlock();
                            pm_release_work(work);
                            lk.lock();
                            resident[slot] = 0;
                            cv_work.notify_all();
                        }
                        continue;
                    }
                    if (stopping && queue.empty()) break;
                    if (!queue.empty()) {
                        // the oldest request and the later ones with the same options
                        const pmlsh_knn_opts o = queue.front()->opts;
                        int64_t rows = 0;
                        std::vector<size_t> pick;
                        for (size_t i = 0; i < queue.size(); i++) {
                            const Request &r = *queue[i];
                            // the oldest request always rides (whatever its options)
                            if (i > 0 && !same_opts(r.opts, o)) continue;
                            if (!pick.empty() && rows + r.nq > opts.max_batch_queries) break;
                            pick.push_back(i);
                            rows += r.nq;
                        }
                        const int64_t g = pm_knn_work_growth(ix, rows, o.k, o.precision, work);
                        bool admit = held() + g <= opts.mem_budget_bytes;
                        if (!admit && inflight == 0) {
                            if (held() - resident[slot] > 0) {
                                seen_epoch = ++trim_epoch;
                                cv_work.notify_all();
                                cv_work.wait(lk);
                                continue;
                            }
                            admit = true;   // alone, above the budget if it must
                        }
                        if (admit) {
                            for (size_t j = pick.size(); j-- > 0;) {
                                batch.push_back(queue[pick[j]]);
                                queue.erase(queue.begin() + (long)pick[j]);
                            }
                            std::reverse(batch.begin(), batch.end());
                            growth = g;
                            reserved += g;
                            inflight++;
                            peak_bytes = std::max(peak_bytes, held());
                            break;
                        }
                        deferred++;   // waits for memory held by other slots
                    }
                    cv_work.wait(lk);
                }
                if (batch.empty()) break;
            }
            // one launch for the whole batch
            const pmlsh_knn_opts o = batch[0]->opts;
            int64_t rows = 0;
            for (auto &r : batch) rows += r->nq;
            std::vector<float> Q((size_t)rows * ix->d);
            int64_t at = 0;
            for (auto &r : batch) {
                std::memcpy(Q.data() + at * ix->d, r->Q.data(), r->Q.size() * sizeof(float));
                at += r->nq;
            }
            std::vector<int64_t> ids((size_t)rows * o.k);
            std::vector<float> dd((size_t)rows * o.k), ee((size_t)rows * o.k);
            pmlsh_status s = pm_knn(ix, Q.data(), rows, &o, ids.data(), dd.data(), ee.data(), nullptr, st, &work);
            std::string err = s == PMLSH_OK ? "" : pmlsh_last_error();
            bool trim = false;
            {
                std::lock_guard<std::mutex> lk(mu);
                at = 0;
                const auto now = Clock::now();
                for (auto &r : batch) {
                    r->status = s;
                    r->error = err;
                    if (s == PMLSH_OK) {
                        r->ids.assign(ids.begin() + at * o.k, ids.begin() + (at + r->nq) * o.k);
                        r->dists.assign(dd.begin() + at * o.k, dd.begin() + (at + r->nq) * o.k);
                        r->err.assign(ee.begin() + at * o.k, ee.begin() + (at + r->nq) * o.k);
                    }
                    at += r->nq;
                    r->done = true;
                    r->t_done = now;
                    completed++;
                    queries += r->nq;
                    lat_ms.push_back(std::chrono::duration<double, std::milli>(now - r->t_submit).count());
                    if (!any_done) { t_first = r->t_submit; any_done = true; }
                    t_last = now;
                }
                batches++;
                reserved -= growth;
                inflight--;
                resident[slot] = pm_work_resident(work);
                peak_bytes = std::max(peak_bytes, held());
                trim = held() > opts.mem_budget_bytes;
            }
            if (trim) {
                pm_release_work(work);
                std::lock_guard<std::mutex> lk(mu);
                resident[slot] = 0;
            }
            cv_done.notify_all();
            cv_work.notify_all();
        }
        pm_release_work(work);
        {
            std::lock_guard<std::mutex> lk(mu);
            resident[slot] = 0;
        }
        cudaStreamDestroy(st);
    }
};

extern "C" {

void pmlsh_serve_opts_default(pmlsh_serve_opts *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->slots = 3;
    o->max_batch_queries = 16384;
    o->mem_budget_bytes = (int64_t)8 << 30;
}

pmlsh_status pmlsh_serve_create(pmlsh_index *ix, const pmlsh_serve_opts *opts, pmlsh_server **out)
{
    if (!ix || !out) {
        pm_set_error("NULL argument");
        return PMLSH_EINVAL;
    }
    pmlsh_serve_opts o;
    if (opts) o = *opts;
    else pmlsh_serve_opts_default(&o);
    if (o.slots < 1 || o.slots > 64 || o.max_batch_queries < 1 || o.mem_budget_bytes < 1) {
        pm_set_error("slots must be in 1..64, max_batch_queries and mem_budget_bytes >= 1");
        return PMLSH_EINVAL;
    }
    auto *s = new (std::nothrow) pmlsh_server();
    if (!s) {
        pm_set_error("host allocation failed");
        return PMLSH_ENOMEM;
    }
    s->ix = ix;
    s->opts = o;
    s->resident.assign(o.slots, 0);
    cudaGetDevice(&s->device);
    for (int i = 0; i < o.slots; i++) s->workers.emplace_back(&pmlsh_server::worker, s, i);
    *out = s;
    return PMLSH_OK;
}

pmlsh_status pmlsh_serve_submit(pmlsh_server *s, const float *Q, int64_t nq, const pmlsh_knn_opts *opts,
                                uint64_t *ticket)
{
    if (!s || !Q || !opts || !ticket || nq < 1) {
        pm_set_error("NULL argument or nq < 1");
        return PMLSH_EINVAL;
    }
    const pmlsh_knn_opts &o = *opts;
    if (o.k < 1 || o.k > PM_MAX_K || o.k > s->ix->n || !(o.c > 1.0) || !std::isfinite(o.c) ||
        !(o.beta > 0.0 && o.beta <= 1.0) || !(o.alpha1 > 0.0 && o.alpha1 < 1.0) || !std::isfinite(o.r_min) ||
        !std::isfinite(o.t) ||
        o.precision < 0 || o.precision > PMLSH_BF16_RERANK ||
        (o.precision != PMLSH_FP32_PLAIN && !(s->ix->Bsplit && s->ix->Xr)) ||
        (o.stop_rule != PMLSH_STOP_LITERAL && o.stop_rule != PMLSH_STOP_BC_CONSISTENT)) {
        pm_set_error("invalid query options");
        return PMLSH_EINVAL;
    }
    if (pm_is_device_ptr(Q)) {
        pm_set_error("serving takes query rows in host memory");
        return PMLSH_EINVAL;
    }
    auto r = std::make_shared<Request>();
    r->nq = nq;
    r->opts = o;
    try {
        r->Q.assign(Q, Q + nq * s->ix->d);
    } catch (...) {
        pm_set_error("host allocation failed");
        return PMLSH_ENOMEM;
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stopping) {
            pm_set_error("server is stopping");
            return PMLSH_ECANCELED;
        }
        r->ticket = s->next_ticket++;
        r->t_submit = Clock::now();
        s->tickets[r->ticket] = r;
        s->queue.push_back(r);
        s->submitted++;
        *ticket = r->ticket;
    }
    s->cv_work.notify_one();
    return PMLSH_OK;
}

pmlsh_status pmlsh_serve_wait(pmlsh_server *s, uint64_t ticket, int64_t *ids, float *dists, float *err,
                              int timeout_ms)
{
    if (!s || !ids || !dists) {
        pm_set_error("NULL argument");
        return PMLSH_EINVAL;
    }
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) {
        pm_set_error("unknown ticket %llu", (unsigned long long)ticket);
        return PMLSH_EINVAL;
    }
    std::shared_ptr<Request> r = it->second;
    const auto pred = [&] { return r->done; };
    if (timeout_ms < 0) s->cv_done.wait(lk, pred);
    else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred)) {
        pm_set_error("request %llu not complete after %d ms", (unsigned long long)ticket, timeout_ms);
        return PMLSH_ETIMEOUT;
    }
    s->tickets.erase(ticket);
    if (r->status != PMLSH_OK) {
        pm_set_error("%s", r->error.c_str());
        return r->status;
    }
    std::memcpy(ids, r->ids.data(), r->ids.size() * sizeof(int64_t));
    std::memcpy(dists, r->dists.data(), r->dists.size() * sizeof(float));
    if (err) std::memcpy(err, r->err.data(), r->err.size() * sizeof(float));
    return PMLSH_OK;
}

pmlsh_status pmlsh_serve_stop(pmlsh_server *s)
{
    if (!s) {
        pm_set_error("NULL argument");
        return PMLSH_EINVAL;
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;
        // requests not started yet are cancelled; running batches finish
        for (auto &r : s->queue) {
            r->status = PMLSH_ECANCELED;
            r->error = "cancelled: server stopped";
            r->done = true;
            s->canceled++;
        }
        s->queue.clear();
    }
    s->cv_work.notify_all();
    s->cv_done.notify_all();
    for (auto &t : s->workers)
        if (t.joinable()) t.join();
    s->workers.clear();
    return PMLSH_OK;
}

pmlsh_status pmlsh_serve_stats(pmlsh_server *s, pmlsh_server_stats *out)
{
    if (!s || !out) {
        pm_set_error("NULL argument");
        return PMLSH_EINVAL;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(out, 0, sizeof(*out));
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->queries = s->queries;
    out->batches = s->batches;
    out->deferred = s->deferred;
    out->canceled = s->canceled;
    out->queue_depth = (int64_t)s->queue.size();
    out->resident_bytes = s->held();
    out->peak_bytes = s->peak_bytes;
    if (!s->lat_ms.empty()) {
        std::vector<double> v(s->lat_ms);
        std::sort(v.begin(), v.end());
        auto pct = [&v](double p) {
            size_t i = (size_t)std::ceil(p * (double)v.size()) - 1;
            return v[std::min(v.size() - 1, i)];
        };
        out->p50_ms = pct(0.50);
        out->p99_ms = pct(0.99);
        double sum = 0.0;
        for (double x : v) sum += x;
        out->mean_ms = sum / (double)v.size();
        const double span = std::chrono::duration<double>(s->t_last - s->t_first).count();
        out->qps = span > 0 ? (double)s->queries / span : 0.0;
    }
    return PMLSH_OK;
}

pmlsh_status pmlsh_serve_destroy(pmlsh_server *s)
{
    if (!s) return PMLSH_OK;
    pmlsh_serve_stop(s);
    delete s;
    return PMLSH_OK;
}

}  // extern "C"
