// CPU candidate feeder: algorithm ALL (Section 3.1) as an index nested loop
// join (Section 2.2.4) over a collection preprocessed as in Section 2.2.1.
// See include/ssj_feeder.h for the contract.
//
// The incremental self-join probes set r against the index of every set
// before it in (size, lexicographic) order.  Because that order is fixed in
// advance, the index of all prefixes can be built once with posting lists
// sorted by position; probe r then reads only the entries whose position
// lies in [first position whose size passes the length filter, position of
// r).  That makes probes independent, so worker threads generate the
// candidates of consecutive blocks of probes in parallel while the consumer
// emits them in order (the H0 role of Section 3.2, parallelised).
#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/ssj_feeder.h"
#include "filters.h"

namespace ssj {
void renumber_by_frequency(const uint64_t* offsets, const uint32_t* tokens, uint32_t n, std::vector<uint32_t>& out);
}

namespace {

struct Block {
    std::vector<uint32_t> probe;   // original ids
    std::vector<uint64_t> offs;    // probe.size()+1, relative
    std::vector<uint32_t> cands;   // original ids
};

constexpr uint32_t kPruned = 0xFFFFFFFFu;

// Sort ids by (size, lexicographic renumbered tokens, id) (Section 2.2.1).
void order_sets(const uint64_t* of, const uint32_t* tk, uint32_t n, std::vector<uint32_t>& order) {
    order.resize(n);
    for (uint32_t i = 0; i < n; ++i) order[i] = i;
    std::sort(order.begin(), order.end(), [of, tk](uint32_t a, uint32_t b) {
        const uint64_t na = of[a + 1] - of[a], nb = of[b + 1] - of[b];
        if (na != nb) return na < nb;
        for (uint64_t i = 0; i < na; ++i)
            if (tk[of[a] + i] != tk[of[b] + i]) return tk[of[a] + i] < tk[of[b] + i];
        return a < b;
    });
}

ssj_status check_sets(const uint64_t* offsets, const uint32_t* tokens, uint32_t n) {
    if (!offsets || (offsets[n] && !tokens)) return SSJ_EINVAL;
    if (offsets[0] != 0) return SSJ_EINVAL;
    for (uint32_t i = 0; i < n; ++i) {
        if (offsets[i + 1] < offsets[i] || offsets[i + 1] - offsets[i] >= (1ull << 31)) return SSJ_EINVAL;
        for (uint64_t t = offsets[i] + 1; t < offsets[i + 1]; ++t)
            if (tokens[t - 1] >= tokens[t]) return SSJ_EINVAL;
    }
    return SSJ_OK;
}

}  // namespace

struct ssj_feeder {
    uint32_t n = 0, p = 1, q = 1, sim = 0;  // n: probe sets
    bool rs = false;                         // R x S (probes of R against the index of S)
    bool ppjoin = false;
    // probe side (R; the collection itself for a self-join)
    std::vector<uint64_t> offs;      // by original id
    std::vector<uint32_t> toks;      // renumbered, each set ascending
    // index side (S; for a self-join these stay empty and the probe side's
    // arrays are indexed)
    uint32_t n_s = 0;
    std::vector<uint64_t> s_offs;
    std::vector<uint32_t> s_toks;
    std::vector<uint32_t> order;     // index position -> original id (size order)
    std::vector<uint32_t> size_at;   // index position -> size (nondecreasing)
    std::vector<uint64_t> post_off;  // token -> range in post
    std::vector<uint32_t> post;      // index positions, ascending per token
    std::vector<uint32_t> post_j;    // position of the token in its set (PPJoin)

    uint32_t block_size = 2048;
    uint32_t n_blocks = 0;
    uint32_t max_ahead = 8;

    std::mutex mu;
    std::condition_variable cv_prod, cv_cons;
    std::map<uint32_t, std::unique_ptr<Block>> ready;
    uint32_t next_produce = 0;  // guarded by mu
    uint32_t next_emit = 0;     // block being emitted
    bool stop = false;
    std::vector<std::thread> workers;

    std::unique_ptr<Block> cur;  // block being emitted
    size_t cur_probe = 0;
    uint64_t cur_cand = 0;       // candidates of cur_probe already emitted
    uint64_t emitted = 0;
    uint32_t probed = 0;

    ssj::Filters flt;  // prefix and length filters of the function and threshold

    uint64_t min_overlap(uint64_t len) const { return flt.min_overlap(len); }
    uint32_t max_partner(uint64_t len) const { return flt.max_partner(len); }
    uint32_t required(uint32_t nr, uint32_t ns) const { return flt.required(nr, ns); }
    uint32_t prefix_len(uint32_t len) const { return flt.prefix_len(len); }

    // Candidates of one probe: index entries in positions [lo, hi) sharing a
    // prefix token with r, deduplicated (stamp) or, with PPJoin, counted
    // (acc) and dropped once the positional bound A + 1 + min(|r|-i-1,
    // |s|-j-1) falls below the pair's equivalent overlap.
    void probe_one(uint32_t key, const uint32_t* rt, uint32_t L, uint32_t lo, uint32_t hi, Block& out,
                   std::vector<uint32_t>& stamp, std::vector<uint32_t>& acc, std::vector<uint32_t>& touched) const {
        const uint32_t pl = prefix_len(L);
        if (!ppjoin) {
            for (uint32_t a = 0; a < pl; ++a) {
                const uint32_t* lb = post.data() + post_off[rt[a]];
                const uint32_t* le = post.data() + post_off[rt[a] + 1];
                for (const uint32_t* it = std::lower_bound(lb, le, lo); it != le && *it < hi; ++it) {
                    const uint32_t e = *it;
                    if (stamp[e] == key) continue;
                    stamp[e] = key;
                    out.cands.push_back(order[e]);
                }
            }
            return;
        }
        touched.clear();
        for (uint32_t a = 0; a < pl; ++a) {
            const uint64_t b0 = post_off[rt[a]], b1 = post_off[rt[a] + 1];
            const uint32_t* lb = post.data() + b0;
            const uint32_t* le = post.data() + b1;
            for (const uint32_t* it = std::lower_bound(lb, le, lo); it != le && *it < hi; ++it) {
                const uint32_t e = *it;
                uint32_t& A = acc[e];
                if (A == kPruned) continue;
                const uint32_t ns = size_at[e], j = post_j[it - post.data()];
                const uint32_t ub = 1 + std::min(L - a - 1, ns - j - 1);
                if (A == 0) touched.push_back(e);
                if ((uint64_t)A + ub >= required(L, ns)) ++A; else A = kPruned;
            }
        }
        for (uint32_t e : touched) {
            if (acc[e] != kPruned) out.cands.push_back(order[e]);
            acc[e] = 0;
        }
    }

    void generate(uint32_t b, Block& out, std::vector<uint32_t>& stamp, std::vector<uint32_t>& acc,
                  std::vector<uint32_t>& touched) const {
        const uint32_t i0 = b * block_size;
        const uint32_t i1 = std::min<uint32_t>(n, i0 + block_size);
        out.offs.push_back(0);
        for (uint32_t i = i0; i < i1; ++i) {
            // self-join: probe i is index position i (incremental index of
            // the sets before it); R x S: probe i is set i of R
            const uint32_t r = rs ? i : order[i];
            const uint32_t L = (uint32_t)(offs[r + 1] - offs[r]);
            const uint64_t start = out.cands.size();
            if (L > 0) {
                const uint64_t min_size = min_overlap(L);  // length filter (for Jaccard q|s| >= p|r|)
                const uint32_t lo = (uint32_t)(std::lower_bound(size_at.begin(), size_at.begin() + (rs ? n_s : i),
                                                                (uint32_t)std::min<uint64_t>(min_size, 0xFFFFFFFFu)) -
                                               size_at.begin());
                uint32_t hi = i;
                if (rs) {
                    const uint32_t mx = max_partner(L);
                    hi = (uint32_t)(std::upper_bound(size_at.begin(), size_at.end(), mx) - size_at.begin());
                }
                if (lo < hi) probe_one(i, toks.data() + offs[r], L, lo, hi, out, stamp, acc, touched);
            }
            if (out.cands.size() > start) {
                out.probe.push_back(r);
                out.offs.push_back(out.cands.size());
            }
        }
    }

    void worker() {
        std::vector<uint32_t> stamp(ppjoin ? 0 : n_s, 0xFFFFFFFFu);
        std::vector<uint32_t> acc(ppjoin ? n_s : 0, 0u), touched;
        for (;;) {
            uint32_t b;
            {
                std::unique_lock<std::mutex> lk(mu);
                cv_prod.wait(lk, [&] { return stop || next_produce < n_blocks && next_produce < next_emit + max_ahead; });
                if (stop || next_produce >= n_blocks) return;
                b = next_produce++;
            }
            std::unique_ptr<Block> blk(new Block());
            generate(b, *blk, stamp, acc, touched);
            {
                std::unique_lock<std::mutex> lk(mu);
                ready[b] = std::move(blk);
            }
            cv_cons.notify_all();
        }
    }

    // Index of every prefix of the index side, posting lists sorted by position.
    void build_index() {
        const uint64_t* of = rs ? s_offs.data() : offs.data();
        const uint32_t* tk = rs ? s_toks.data() : toks.data();
        order_sets(of, tk, n_s, order);
        size_at.resize(n_s);
        for (uint32_t pos = 0; pos < n_s; ++pos) size_at[pos] = (uint32_t)(of[order[pos] + 1] - of[order[pos]]);
        uint32_t vocab = 0;
        for (uint32_t t : toks) vocab = std::max(vocab, t + 1);
        for (uint32_t t : s_toks) vocab = std::max(vocab, t + 1);
        post_off.assign((size_t)vocab + 1, 0);
        for (uint32_t pos = 0; pos < n_s; ++pos) {
            const uint32_t r = order[pos];
            const uint32_t pl = prefix_len(size_at[pos]);
            for (uint32_t a = 0; a < pl; ++a) post_off[tk[of[r] + a] + 1]++;
        }
        for (size_t t = 0; t < vocab; ++t) post_off[t + 1] += post_off[t];
        post.resize(post_off[vocab]);
        if (ppjoin) post_j.resize(post_off[vocab]);
        std::vector<uint64_t> fill(post_off.begin(), post_off.end() - 1);
        for (uint32_t pos = 0; pos < n_s; ++pos) {
            const uint32_t r = order[pos];
            const uint32_t pl = prefix_len(size_at[pos]);
            for (uint32_t a = 0; a < pl; ++a) {
                const uint64_t k = fill[tk[of[r] + a]]++;
                post[k] = pos;
                if (ppjoin) post_j[k] = a;
            }
        }
    }
};

extern "C" ssj_status ssj_feeder_create_ex(const uint64_t* r_offsets, const uint32_t* r_tokens, uint32_t n_r,
                                           const uint64_t* s_offsets, const uint32_t* s_tokens, uint32_t n_s,
                                           const ssj_feeder_opts* opts, ssj_feeder** out) {
    if (!opts || !out) return SSJ_EINVAL;
    const uint32_t sim = opts->sim, p = opts->p, q = opts->q;
    if (!ssj::Filters::valid(sim, p, q) || (opts->flags & ~SSJ_FEEDER_PPJOIN)) return SSJ_EINVAL;
    if (check_sets(r_offsets, r_tokens, n_r) != SSJ_OK) return SSJ_EINVAL;
    const bool rs = s_offsets != nullptr;
    if (rs && check_sets(s_offsets, s_tokens, n_s) != SSJ_OK) return SSJ_EINVAL;
    std::unique_ptr<ssj_feeder> f(new ssj_feeder());
    try {
        f->n = n_r;
        f->p = p;
        f->q = q;
        f->sim = sim;
        f->flt.sim = sim;
        f->flt.p = p;
        f->flt.q = q;
        f->rs = rs;
        f->ppjoin = (opts->flags & SSJ_FEEDER_PPJOIN) != 0;
        if (!rs) {
            f->offs.assign(r_offsets, r_offsets + n_r + 1);
            ssj::renumber_by_frequency(r_offsets, r_tokens, n_r, f->toks);
            f->n_s = n_r;
        } else {
            // one token order for both sides: renumber R and S together
            std::vector<uint64_t> cat_offs((size_t)n_r + n_s + 1);
            std::vector<uint32_t> cat_toks;
            cat_toks.reserve(r_offsets[n_r] + s_offsets[n_s]);
            cat_toks.insert(cat_toks.end(), r_tokens, r_tokens + r_offsets[n_r]);
            cat_toks.insert(cat_toks.end(), s_tokens, s_tokens + s_offsets[n_s]);
            for (uint32_t i = 0; i <= n_r; ++i) cat_offs[i] = r_offsets[i];
            for (uint32_t i = 1; i <= n_s; ++i) cat_offs[n_r + i] = r_offsets[n_r] + s_offsets[i];
            std::vector<uint32_t> renum;
            ssj::renumber_by_frequency(cat_offs.data(), cat_toks.data(), n_r + n_s, renum);
            f->offs.assign(r_offsets, r_offsets + n_r + 1);
            f->toks.assign(renum.begin(), renum.begin() + r_offsets[n_r]);
            f->n_s = n_s;
            f->s_offs.assign(s_offsets, s_offsets + n_s + 1);
            f->s_toks.assign(renum.begin() + r_offsets[n_r], renum.end());
        }
        f->build_index();
    } catch (const std::bad_alloc&) {
        return SSJ_ENOMEM;
    }
    f->n_blocks = (n_r + f->block_size - 1) / f->block_size;
    const uint32_t nt = std::max<uint32_t>(1, std::min<uint32_t>(opts->n_threads, 256));
    f->max_ahead = std::max<uint32_t>(8, 2 * nt);
    ssj_feeder* raw = f.release();
    for (uint32_t i = 0; i < nt; ++i) raw->workers.emplace_back(&ssj_feeder::worker, raw);
    *out = raw;
    return SSJ_OK;
}

extern "C" ssj_status ssj_feeder_create_sim(const uint64_t* offsets, const uint32_t* tokens, uint32_t n_sets,
                                            uint32_t sim, uint32_t p, uint32_t q, uint32_t n_threads,
                                            ssj_feeder** out) {
    ssj_feeder_opts o;
    o.sim = sim;
    o.p = p;
    o.q = q;
    o.flags = 0;
    o.n_threads = n_threads;
    return ssj_feeder_create_ex(offsets, tokens, n_sets, nullptr, nullptr, 0, &o, out);
}

extern "C" ssj_status ssj_feeder_create(const uint64_t* offsets, const uint32_t* tokens, uint32_t n_sets, uint32_t p,
                                        uint32_t q, uint32_t n_threads, ssj_feeder** out) {
    return ssj_feeder_create_sim(offsets, tokens, n_sets, 0, p, q, n_threads, out);
}

extern "C" ssj_status ssj_feeder_next(ssj_feeder* f, uint32_t max_probes, uint64_t max_cands, uint32_t* probe_ids,
                                      uint64_t* cand_offsets, uint32_t* cand_ids, uint32_t* n_probes,
                                      uint64_t* n_cands, int* done) {
    if (!f || !probe_ids || !cand_offsets || !cand_ids || !n_probes || !n_cands || !done) return SSJ_EINVAL;
    if (max_probes == 0 || max_cands == 0) return SSJ_EINVAL;
    uint32_t np = 0;
    uint64_t nc = 0;
    cand_offsets[0] = 0;
    *done = 0;
    for (;;) {
        if (f->cur && f->cur_probe >= f->cur->probe.size()) {  // block fully emitted
            {
                std::unique_lock<std::mutex> lk(f->mu);
                f->probed = std::min<uint32_t>(f->n, (f->next_emit + 1) * f->block_size);
                f->next_emit++;
            }
            f->cv_prod.notify_all();
            f->cur.reset();
        }
        if (np >= max_probes || nc >= max_cands) break;
        if (!f->cur) {
            if (f->next_emit >= f->n_blocks) break;
            std::unique_lock<std::mutex> lk(f->mu);
            f->cv_cons.wait(lk, [&] { return f->ready.count(f->next_emit) > 0; });
            f->cur = std::move(f->ready[f->next_emit]);
            f->ready.erase(f->next_emit);
            f->cur_probe = 0;
            f->cur_cand = 0;
            continue;
        }
        Block& b = *f->cur;
        const uint64_t beg = b.offs[f->cur_probe] + f->cur_cand;
        const uint64_t end = b.offs[f->cur_probe + 1];
        const uint64_t take = std::min<uint64_t>(end - beg, max_cands - nc);
        memcpy(cand_ids + nc, b.cands.data() + beg, sizeof(uint32_t) * take);
        probe_ids[np] = b.probe[f->cur_probe];
        nc += take;
        ++np;
        cand_offsets[np] = nc;
        if (beg + take == end) {
            f->cur_probe++;
            f->cur_cand = 0;
        } else {
            f->cur_cand += take;
        }
    }
    f->emitted += nc;
    *n_probes = np;
    *n_cands = nc;
    *done = (!f->cur && f->next_emit >= f->n_blocks) ? 1 : 0;
    return SSJ_OK;
}

extern "C" ssj_status ssj_feeder_progress(ssj_feeder* f, uint64_t* n_cands, uint32_t* probed, uint32_t* n_sets) {
    if (!f) return SSJ_EINVAL;
    if (n_cands) *n_cands = f->emitted;
    if (probed) *probed = f->probed;
    if (n_sets) *n_sets = f->n;
    return SSJ_OK;
}

extern "C" void ssj_feeder_destroy(ssj_feeder* f) {
    if (!f) return;
    {
        std::unique_lock<std::mutex> lk(f->mu);
        f->stop = true;
    }
    f->cv_prod.notify_all();
    for (auto& t : f->workers) t.join();
    delete f;
}
