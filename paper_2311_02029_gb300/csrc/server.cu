// Continuous-batching request loop over one resident index.
//
// Requests (host read batches) enter a FIFO queue. `max_slots` worker threads, each with its
// own CUDA stream, take requests as they free up, so a request that arrives while others run
// is admitted as soon as a slot and memory free up, and the device overlaps the work of all
// admitted requests. Each slot owns two plans (preallocated workspaces replayed from captured
// CUDA graphs, grids sized to their capacity) for batches of up to SMALL_READS and SLOT_READS
// reads of <= SLOT_READ_LEN bases; they are charged once against the HBM budget when the
// server starts (a plan that does not fit is not made). A request runs on the smallest of its
// slot's plans that holds it; any other request is
// admitted only while its own workspace fits in the budget still free (charged at admission,
// released at completion). A request larger than the whole budget fails with MT_ENOMEM instead
// of blocking the queue. Completion is observed by polling with a bounded wait; latency is
// measured from submit to results on the host.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t id = 0;
    const uint8_t *reads = nullptr;
    uint64_t n_bases = 0;
    const uint64_t *offsets = nullptr;
    uint64_t n_reads = 0;
    int32_t *taxon = nullptr;
    uint8_t *nloc = nullptr;
    mt_loc *locs = nullptr;
    uint64_t *genome_hits = nullptr;
    double *abundance = nullptr;
    uint64_t ws_bytes = 0;
    uint64_t max_len = 0;
    int status = MT_EBUSY;
    bool done = false;
    bool cancelled = false;
    bool running = false;
    Clock::time_point t_submit, t_done;
};

}  // namespace

static constexpr uint64_t SLOT_READS = 1ull << 20;
static constexpr uint64_t SMALL_READS = 1ull << 16;
static constexpr uint32_t SLOT_READ_LEN = 256;

struct mt_server {
    const mt_index *ix = nullptr;
    mt_classify_params params{};
    uint64_t budget = 0, in_use = 0;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Request>> queue;
    std::map<uint64_t, std::shared_ptr<Request>> all;
    std::vector<std::thread> workers;
    uint64_t next_id = 1;
    bool stop = false;

    static bool fits(const Request &r, uint64_t cap) {
        return r.n_reads <= cap && r.n_bases <= cap * SLOT_READ_LEN && r.max_len <= SLOT_READ_LEN;
    }

    mt_plan *make_plan(uint64_t cap) {   // called with mu held
        uint64_t need = mt::classify_ws_bytes(ix, cap * SLOT_READ_LEN, cap, &params, SLOT_READ_LEN, true);
        mt_plan *pl = nullptr;
        if (need && need <= budget - in_use &&
            mt_plan_create(ix, &params, cap, cap * SLOT_READ_LEN, SLOT_READ_LEN, &pl) == MT_OK) {
            in_use += mt_plan_device_bytes(pl);
            return pl;
        }
        return nullptr;
    }

    void worker_main(int slot) {
        cudaSetDevice(device);
        cudaStream_t s;
        cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        mt_plan *small = nullptr, *large = nullptr;
        {
            std::lock_guard<std::mutex> lk(mu);
            small = make_plan(SMALL_READS);
            large = make_plan(SLOT_READS);
            plan_slots += (small != nullptr) + (large != nullptr);
            ready++;
            cv_done.notify_all();
        }
        auto plan_for = [&](const Request &r) -> mt_plan * {
            if (small && fits(r, SMALL_READS)) return small;
            if (large && fits(r, SLOT_READS)) return large;
            return nullptr;
        };
        std::unique_lock<std::mutex> lk(mu);
        while (true) {
            std::shared_ptr<Request> job;
            mt_plan *on_plan = nullptr;
            auto runnable = [&](const Request &r) {
                return plan_for(r) != nullptr || r.ws_bytes <= budget - in_use || r.ws_bytes > budget;
            };
            cv_work.wait(lk, [&] {
                if (stop) return true;
                for (auto &r : queue)
                    if (runnable(*r)) return true;
                return false;
            });
            if (stop) break;
            for (auto it = queue.begin(); it != queue.end(); ++it) {
                auto &r = *it;
                if ((on_plan = plan_for(*r)) != nullptr) {
                    job = r;
                    queue.erase(it);
                    break;
                }
                if (r->ws_bytes > budget) {   // can never fit: fail it
                    r->status = MT_ENOMEM;
                    r->done = true;
                    r->t_done = Clock::now();
                    queue.erase(it);
                    cv_done.notify_all();
                    break;
                }
                if (r->ws_bytes <= budget - in_use) {
                    job = r;
                    queue.erase(it);
                    break;
                }
            }
            if (!job) continue;
            if (!on_plan) in_use += job->ws_bytes;
            job->running = true;
            lk.unlock();
            int rc = on_plan
                ? mt_plan_classify(on_plan, job->reads, job->n_bases, job->offsets, job->n_reads, 0, s, job->taxon,
                                   job->nloc, job->locs, job->genome_hits, job->abundance, nullptr)
                : mt_classify(ix, job->reads, job->n_bases, job->offsets, job->n_reads, &params, 0, s, job->taxon,
                              job->nloc, job->locs, job->genome_hits, job->abundance, nullptr);
            lk.lock();
            if (!on_plan) in_use -= job->ws_bytes;
            job->running = false;
            job->status = rc;
            job->done = true;
            job->t_done = Clock::now();
            cv_done.notify_all();
            cv_work.notify_all();
        }
        for (mt_plan *pl : {small, large}) {
            if (!pl) continue;
            in_use -= mt_plan_device_bytes(pl);
            mt_plan_destroy(pl);
        }
        lk.unlock();
        cudaStreamDestroy(s);
        (void)slot;
    }
    int plan_slots = 0, ready = 0;
};

extern "C" int mt_server_create(const mt_index *ix, uint64_t hbm_budget, int max_slots,
                                const mt_classify_params *params, mt_server **out) {
    if (!out) return MT_EINVAL;
    *out = nullptr;
    if (!ix || !params || max_slots < 1 || max_slots > 64 || hbm_budget == 0) return MT_EINVAL;
    if (mt_classify_workspace_bytes(ix, 1024, 1, 0, params) == 0) return MT_EINVAL;
    mt_server *s = new mt_server();
    s->ix = ix;
    s->params = *params;
    s->budget = hbm_budget;
    cudaGetDevice(&s->device);
    for (int i = 0; i < max_slots; i++) s->workers.emplace_back([s, i] { s->worker_main(i); });
    {   // wait until every slot has (or has not) set up its plan
        std::unique_lock<std::mutex> lk(s->mu);
        s->cv_done.wait(lk, [&] { return s->ready == max_slots; });
    }
    *out = s;
    return MT_OK;
}

extern "C" int mt_server_submit(mt_server *s, const uint8_t *reads, uint64_t n_bases, const uint64_t *offsets,
                                uint64_t n_reads, int32_t *taxon, uint8_t *nloc, mt_loc *locs,
                                uint64_t *genome_hits, double *abundance, uint64_t *req_id) {
    if (!s || !offsets || !taxon || !req_id || (!reads && n_bases)) return MT_EINVAL;
    auto r = std::make_shared<Request>();
    r->reads = reads; r->n_bases = n_bases; r->offsets = offsets; r->n_reads = n_reads;
    r->taxon = taxon; r->nloc = nloc; r->locs = locs; r->genome_hits = genome_hits; r->abundance = abundance;
    // the longest read bounds the slow-path scratch; account for it exactly
    uint64_t maxn = 0;
    for (uint64_t i = 0; i < n_reads; i++) maxn = std::max<uint64_t>(maxn, offsets[i + 1] - offsets[i]);
    r->ws_bytes = mt::classify_ws_bytes(s->ix, n_bases, n_reads, &s->params,
                                        (uint32_t)std::min<uint64_t>(maxn, MT_MAX_READ_LEN), true);
    r->max_len = maxn;
    r->t_submit = Clock::now();
    std::lock_guard<std::mutex> lk(s->mu);
    r->id = s->next_id++;
    s->all[r->id] = r;
    s->queue.push_back(r);
    *req_id = r->id;
    s->cv_work.notify_all();
    return MT_OK;
}

extern "C" int mt_server_poll(mt_server *s, uint64_t req_id, int timeout_ms, double *latency_s) {
    if (!s) return MT_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(req_id);
    if (it == s->all.end()) return MT_EINVAL;
    auto r = it->second;
    if (!r->done && timeout_ms > 0)
        s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return r->done; });
    if (!r->done) return timeout_ms > 0 ? MT_ETIMEDOUT : MT_EBUSY;
    if (latency_s) latency_s[0] = std::chrono::duration<double>(r->t_done - r->t_submit).count();
    s->all.erase(req_id);   // reported: released (a long-running loop keeps no finished requests)
    return r->status;
}

extern "C" int mt_server_cancel(mt_server *s, uint64_t req_id) {
    if (!s) return MT_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(req_id);
    if (it == s->all.end()) return MT_EINVAL;
    auto r = it->second;
    if (r->done || r->running) return MT_EBUSY;
    for (auto q = s->queue.begin(); q != s->queue.end(); ++q)
        if ((*q)->id == req_id) { s->queue.erase(q); break; }
    r->cancelled = true;
    r->status = MT_ECANCELED;
    r->done = true;
    r->t_done = std::chrono::steady_clock::now();
    s->cv_done.notify_all();
    return MT_OK;
}

extern "C" void mt_server_destroy(mt_server *s) {
    if (!s) return;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        // let admitted work finish, drop what is still queued
        for (auto &r : s->queue) {
            r->status = MT_ECANCELED;
            r->done = true;
        }
        s->queue.clear();
        s->stop = true;
        s->cv_work.notify_all();
        s->cv_done.notify_all();
    }
    for (auto &t : s->workers) t.join();
    delete s;
}

extern "C" const char *mt_strerror(int status) {
    switch (status) {
        case MT_OK: return "ok";
        case MT_EINVAL: return "invalid argument or input";
        case MT_ENOMEM: return "out of memory or over the HBM budget";
        case MT_ETIMEDOUT: return "timed out";
        case MT_ECUDA: return "CUDA runtime error";
        case MT_ECANCELED: return "cancelled";
        case MT_EBUSY: return "still in flight";
        case MT_EXCHANGE: return "the allreduce of a sharded batch failed";
        case MT_EIO: return "file I/O failed or not a saved index";
        default: return "unknown status";
    }
}

extern "C" int mt_version(void) { return 1; }
