// Native drivers of the serving path; see include/ssj_serve.h.
//
// ssj_serve_replay is an open-loop load generator: requests arrive at given
// times whatever the state of the server, wait on the client side while the
// library has no free slot or budget, and their latency runs from arrival to
// collected results.  ssj_serve_coprocess is the H0/H1/H2 scheme of
// Section 3.2: the filtering thread builds chunks and hands them over, the
// device verifies them on per-slot streams, a collector thread gathers the
// results.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <functional>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/ssj_feeder.h"
#include "../../include/ssj_serve.h"

namespace {

using Clock = std::chrono::steady_clock;

double seconds_since(Clock::time_point t0, Clock::time_point t) {
    return std::chrono::duration<double>(t - t0).count();
}

void wait_until(Clock::time_point t) {
    // sleep while far ahead, then spin for precision
    for (;;) {
        const auto now = Clock::now();
        if (now >= t) return;
        const auto left = t - now;
        if (left > std::chrono::microseconds(300)) std::this_thread::sleep_for(left - std::chrono::microseconds(200));
        else std::this_thread::yield();
    }
}

struct Admitted {
    uint64_t ticket;
    uint32_t idx;
    Clock::time_point submitted;
};

// Collector shared by both drivers: polls admitted tickets, collects results.
struct Collector {
    ssj_ctx* ctx;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Admitted> pending;
    bool closed = false;           // no more submissions will come
    std::atomic<uint32_t> inflight{0};
    std::atomic<uint64_t> results{0};
    ssj_status first_err = SSJ_OK;
    std::vector<ssj_triple> buf;

    // called for each collected request: (idx, submitted time, done time)
    std::function<void(uint32_t, Clock::time_point, Clock::time_point)> on_done;

    void add(const Admitted& a) {
        {
            std::lock_guard<std::mutex> lk(mu);
            pending.push_back(a);
        }
        inflight++;
        cv.notify_one();
    }
    void close() {
        {
            std::lock_guard<std::mutex> lk(mu);
            closed = true;
        }
        cv.notify_one();
    }
    void run() {
        std::vector<Admitted> local;
        for (;;) {
            {
                std::unique_lock<std::mutex> lk(mu);
                cv.wait_for(lk, std::chrono::microseconds(50), [&] { return closed || !pending.empty(); });
                while (!pending.empty()) {
                    local.push_back(pending.front());
                    pending.pop_front();
                }
                if (closed && local.empty() && pending.empty()) return;
            }
            bool progressed = false;
            for (size_t i = 0; i < local.size();) {
                int done = 0;
                ssj_status st = ssj_poll(ctx, local[i].ticket, 0, &done);
                if (st == SSJ_ETIMEDOUT || (st == SSJ_OK && !done)) {
                    ++i;
                    continue;
                }
                uint64_t n = 0;
                if (st == SSJ_OK) st = ssj_results(ctx, local[i].ticket, nullptr, 0, &n);
                if (st == SSJ_OK) {
                    if (buf.size() < std::max<uint64_t>(n, 1)) buf.resize(std::max<uint64_t>(n, 1));
                    st = ssj_results(ctx, local[i].ticket, buf.data(), n, &n);
                }
                const auto t_done = Clock::now();
                if (st != SSJ_OK) {
                    if (first_err == SSJ_OK) first_err = st;
                    uint64_t dummy;
                    ssj_results(ctx, local[i].ticket, buf.data(), 0, &dummy);  // release if possible
                } else {
                    results += n;
                }
                if (on_done) on_done(local[i].idx, local[i].submitted, t_done);
                inflight--;
                local[i] = local.back();
                local.pop_back();
                progressed = true;
            }
            if (!progressed && !local.empty()) std::this_thread::sleep_for(std::chrono::microseconds(10));
        }
    }
};

// Submit, retrying while the library answers SSJ_EAGAIN.
ssj_status submit_retry(ssj_ctx* ctx, const ssj_batch* b, uint64_t* ticket, uint32_t* eagain) {
    for (;;) {
        ssj_status st = ssj_submit(ctx, b, ticket);
        if (st != SSJ_EAGAIN) return st;
        ++*eagain;
        std::this_thread::sleep_for(std::chrono::microseconds(5));
    }
}

}  // namespace

extern "C" ssj_status ssj_serve_replay(ssj_ctx* ctx, const ssj_request* reqs, uint32_t n, double* latency_s,
                                       ssj_serve_stats* stats) {
    if (!ctx || (n && (!reqs || !latency_s))) return SSJ_EINVAL;
    Collector col;
    col.ctx = ctx;
    const auto t0 = Clock::now();
    Clock::time_point last_done = t0;
    std::mutex done_mu;
    col.on_done = [&](uint32_t idx, Clock::time_point, Clock::time_point t_done) {
        latency_s[idx] = seconds_since(t0, t_done) - reqs[idx].arrival_s;
        std::lock_guard<std::mutex> lk(done_mu);
        if (t_done > last_done) last_done = t_done;
    };
    std::thread collector([&] { col.run(); });
    uint32_t eagain = 0, max_inflight = 0;
    uint64_t pairs = 0;
    ssj_status err = SSJ_OK;
    for (uint32_t i = 0; i < n; ++i) {
        wait_until(t0 + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(reqs[i].arrival_s)));
        uint64_t ticket = 0;
        ssj_status st = submit_retry(ctx, &reqs[i].batch, &ticket, &eagain);
        if (st != SSJ_OK) {
            err = st;
            latency_s[i] = -1.0;
            continue;
        }
        const uint64_t nc = reqs[i].batch.n_cands ? reqs[i].batch.n_cands
                                                  : (reqs[i].batch.cand_offsets ? reqs[i].batch.cand_offsets[reqs[i].batch.n_probes] : 0);
        pairs += nc;
        col.add(Admitted{ticket, i, Clock::now()});
        max_inflight = std::max<uint32_t>(max_inflight, col.inflight.load());
    }
    col.close();
    collector.join();
    if (stats) {
        stats->wall_s = seconds_since(t0 + std::chrono::duration_cast<Clock::duration>(
                                               std::chrono::duration<double>(n ? reqs[0].arrival_s : 0.0)),
                                      last_done);
        stats->pairs = pairs;
        stats->results = col.results.load();
        stats->eagain = eagain;
        stats->max_inflight = max_inflight;
    }
    if (err != SSJ_OK) return err;
    return col.first_err;
}

extern "C" ssj_status ssj_serve_coprocess(ssj_ctx* ctx, ssj_coll coll, const uint64_t* offsets,
                                          const uint32_t* tokens, uint32_t n_sets, uint32_t p, uint32_t q,
                                          uint32_t n_threads, uint64_t chunk_cands, ssj_coprocess_stats* stats) {
    if (!ctx || !offsets || !stats || chunk_cands == 0) return SSJ_EINVAL;
    memset(stats, 0, sizeof(*stats));
    const uint32_t max_probes = std::max<uint32_t>(n_sets, 1);
    std::vector<uint32_t> probe(max_probes), cands(chunk_cands);
    std::vector<uint64_t> offs((size_t)max_probes + 1);

    // 1. the filter alone
    {
        ssj_feeder* f = nullptr;
        ssj_status st = ssj_feeder_create(offsets, tokens, n_sets, p, q, n_threads, &f);
        if (st != SSJ_OK) return st;
        const auto t0 = Clock::now();
        int done = 0;
        while (!done) {
            uint32_t np = 0;
            uint64_t nc = 0;
            st = ssj_feeder_next(f, max_probes, chunk_cands, probe.data(), offs.data(), cands.data(), &np, &nc, &done);
            if (st != SSJ_OK) break;
        }
        stats->filter_only_s = seconds_since(t0, Clock::now());
        ssj_feeder_destroy(f);
        if (st != SSJ_OK) return st;
    }

    // 2. filter and verification overlapped
    ssj_feeder* f = nullptr;
    ssj_status st = ssj_feeder_create(offsets, tokens, n_sets, p, q, n_threads, &f);
    if (st != SSJ_OK) return st;
    Collector col;
    col.ctx = ctx;
    std::mutex busy_mu;
    double busy = 0;
    Clock::time_point last_done;
    col.on_done = [&](uint32_t, Clock::time_point sub, Clock::time_point done_t) {
        std::lock_guard<std::mutex> lk(busy_mu);
        busy += std::chrono::duration<double>(done_t - sub).count();
        last_done = done_t;
    };
    const auto t0 = Clock::now();
    last_done = t0;
    std::thread collector([&] { col.run(); });
    uint32_t eagain = 0, chunks = 0;
    uint64_t cand_total = 0;
    int done = 0;
    while (!done && st == SSJ_OK) {
        uint32_t np = 0;
        uint64_t nc = 0;
        st = ssj_feeder_next(f, max_probes, chunk_cands, probe.data(), offs.data(), cands.data(), &np, &nc, &done);
        if (st != SSJ_OK || nc == 0) break;
        ssj_batch b;
        memset(&b, 0, sizeof(b));
        b.R = coll;
        b.S = coll;
        b.p = p;
        b.q = q;
        b.n_probes = np;
        b.probe_ids = probe.data();
        b.cand_offsets = offs.data();
        b.cand_ids = cands.data();
        b.n_cands = nc;
        uint64_t ticket = 0;
        st = submit_retry(ctx, &b, &ticket, &eagain);  // inputs are copied before this returns
        if (st != SSJ_OK) break;
        col.add(Admitted{ticket, chunks, Clock::now()});
        ++chunks;
        cand_total += nc;
    }
    col.close();
    collector.join();
    ssj_feeder_destroy(f);
    stats->join_s = seconds_since(t0, std::max(last_done, t0));
    stats->gpu_busy_s = busy;
    stats->candidates = cand_total;
    stats->results = col.results.load();
    stats->chunks = chunks;
    if (st != SSJ_OK) return st;
    return col.first_err;
}
