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

namespace ssj {
void renumber_by_frequency(const uint64_t* offsets, const uint32_t* tokens, uint32_t n, std::vector<uint32_t>& out);
}

namespace {

struct Block {
    std::vector<uint32_t> probe;   // original ids
    std::vector<uint64_t> offs;    // probe.size()+1, relative
    std::vector<uint32_t> cands;   // original ids
};

// ceil(p*x/q) with 128-bit intermediate
inline uint64_t ceil_mul_div(uint64_t x, uint64_t p, uint64_t q) {
    return (uint64_t)(((unsigned __int128)p * x + q - 1) / q);
}

}  // namespace

struct ssj_feeder {
    uint32_t n = 0, p = 1, q = 1;
    std::vector<uint64_t> offs;      // by original id
    std::vector<uint32_t> toks;      // renumbered, each set ascending
    std::vector<uint32_t> order;     // position -> original id
    std::vector<uint32_t> size_at;   // position -> size (nondecreasing)
    std::vector<uint64_t> post_off;  // token -> range in post
    std::vector<uint32_t> post;      // positions, ascending per token

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

    uint32_t prefix_len(uint32_t len) const {
        if (len == 0) return 0;
        const uint64_t need = ceil_mul_div(len, p, q);
        const uint64_t pl = (uint64_t)len + 1 - need;
        return pl > len ? len : (uint32_t)pl;
    }

    void generate(uint32_t b, Block& out, std::vector<uint32_t>& stamp) const {
        const uint32_t pos0 = b * block_size;
        const uint32_t pos1 = std::min<uint32_t>(n, pos0 + block_size);
        out.offs.push_back(0);
        for (uint32_t pos = pos0; pos < pos1; ++pos) {
            const uint32_t r = order[pos];
            const uint32_t L = size_at[pos];
            const uint64_t start = out.cands.size();
            if (L > 0) {
                const uint64_t min_size = ceil_mul_div(L, p, q);  // length filter: q|s| >= p|r|
                const uint32_t lo_pos =
                    (uint32_t)(std::lower_bound(size_at.begin(), size_at.begin() + pos, (uint32_t)std::min<uint64_t>(min_size, 0xFFFFFFFFu)) -
                               size_at.begin());
                const uint32_t* rt = toks.data() + offs[r];
                const uint32_t pl = prefix_len(L);
                for (uint32_t a = 0; a < pl; ++a) {
                    const uint32_t* lb = post.data() + post_off[rt[a]];
                    const uint32_t* le = post.data() + post_off[rt[a] + 1];
                    const uint32_t* it = std::lower_bound(lb, le, lo_pos);
                    for (; it != le && *it < pos; ++it) {
                        const uint32_t e = *it;
                        if (stamp[e] == pos) continue;
                        stamp[e] = pos;
                        out.cands.push_back(order[e]);
                    }
                }
            }
            if (out.cands.size() > start) {
                out.probe.push_back(r);
                out.offs.push_back(out.cands.size());
            }
        }
    }

    void worker() {
        std::vector<uint32_t> stamp(n, 0xFFFFFFFFu);
        for (;;) {
            uint32_t b;
            {
                std::unique_lock<std::mutex> lk(mu);
                cv_prod.wait(lk, [&] { return stop || next_produce < n_blocks && next_produce < next_emit + max_ahead; });
                if (stop || next_produce >= n_blocks) return;
                b = next_produce++;
            }
            std::unique_ptr<Block> blk(new Block());
            generate(b, *blk, stamp);
            {
                std::unique_lock<std::mutex> lk(mu);
                ready[b] = std::move(blk);
            }
            cv_cons.notify_all();
        }
    }
};

extern "C" ssj_status ssj_feeder_create(const uint64_t* offsets, const uint32_t* tokens, uint32_t n_sets, uint32_t p,
                                        uint32_t q, uint32_t n_threads, ssj_feeder** out) {
    if (!offsets || !out || (offsets[n_sets] && !tokens)) return SSJ_EINVAL;
    if (p == 0 || p > q || q >= (1u << 31)) return SSJ_EINVAL;
    if (offsets[0] != 0) return SSJ_EINVAL;
    for (uint32_t i = 0; i < n_sets; ++i) {
        if (offsets[i + 1] < offsets[i] || offsets[i + 1] - offsets[i] >= (1ull << 31)) return SSJ_EINVAL;
        for (uint64_t t = offsets[i] + 1; t < offsets[i + 1]; ++t)
            if (tokens[t - 1] >= tokens[t]) return SSJ_EINVAL;
    }
    std::unique_ptr<ssj_feeder> f(new ssj_feeder());
    try {
        f->n = n_sets;
        f->p = p;
        f->q = q;
        f->offs.assign(offsets, offsets + n_sets + 1);
        ssj::renumber_by_frequency(offsets, tokens, n_sets, f->toks);
        // order by (size, lexicographic, id)
        f->order.resize(n_sets);
        for (uint32_t i = 0; i < n_sets; ++i) f->order[i] = i;
        const uint64_t* of = f->offs.data();
        const uint32_t* tk = f->toks.data();
        std::sort(f->order.begin(), f->order.end(), [of, tk](uint32_t a, uint32_t b) {
            const uint64_t na = of[a + 1] - of[a], nb = of[b + 1] - of[b];
            if (na != nb) return na < nb;
            for (uint64_t i = 0; i < na; ++i)
                if (tk[of[a] + i] != tk[of[b] + i]) return tk[of[a] + i] < tk[of[b] + i];
            return a < b;
        });
        f->size_at.resize(n_sets);
        for (uint32_t pos = 0; pos < n_sets; ++pos) {
            const uint32_t r = f->order[pos];
            f->size_at[pos] = (uint32_t)(of[r + 1] - of[r]);
        }
        // index of every prefix, posting lists sorted by position
        uint32_t vocab = 0;
        for (uint32_t t : f->toks) vocab = std::max(vocab, t + 1);
        f->post_off.assign((size_t)vocab + 1, 0);
        for (uint32_t pos = 0; pos < n_sets; ++pos) {
            const uint32_t r = f->order[pos];
            const uint32_t pl = f->prefix_len(f->size_at[pos]);
            for (uint32_t a = 0; a < pl; ++a) f->post_off[tk[of[r] + a] + 1]++;
        }
        for (size_t t = 0; t < vocab; ++t) f->post_off[t + 1] += f->post_off[t];
        f->post.resize(f->post_off[vocab]);
        std::vector<uint64_t> fill(f->post_off.begin(), f->post_off.end() - 1);
        for (uint32_t pos = 0; pos < n_sets; ++pos) {
            const uint32_t r = f->order[pos];
            const uint32_t pl = f->prefix_len(f->size_at[pos]);
            for (uint32_t a = 0; a < pl; ++a) f->post[fill[tk[of[r] + a]]++] = pos;
        }
    } catch (const std::bad_alloc&) {
        return SSJ_ENOMEM;
    }
    f->n_blocks = (n_sets + f->block_size - 1) / f->block_size;
    const uint32_t nt = std::max<uint32_t>(1, std::min<uint32_t>(n_threads, 256));
    f->max_ahead = std::max<uint32_t>(8, 2 * nt);
    ssj_feeder* raw = f.release();
    for (uint32_t i = 0; i < nt; ++i) raw->workers.emplace_back(&ssj_feeder::worker, raw);
    *out = raw;
    return SSJ_OK;
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
