// GroupJoin candidate generation (the GRP algorithm the paper evaluates,
// Sections 2.2.4 and 4.1.3): sets that have the same size and the same
// prefix form a group; the prefix filter, the length filter and the
// inverted index work on groups, and each candidate group pair stands for
// every pair of their members.  Expanding the groups (done on the device by
// ssj_verify_groups) gives exactly the candidates of algorithm ALL.
// See include/ssj_feeder.h for the contract.
#include <algorithm>
#include <cstdint>
#include <memory>
#include <new>
#include <vector>

#include "../../include/ssj_feeder.h"
#include "filters.h"

namespace ssj {
void renumber_by_frequency(const uint64_t* offsets, const uint32_t* tokens, uint32_t n, std::vector<uint32_t>& out);
}

struct ssj_groups {
    std::vector<uint64_t> group_offsets;  // n_groups + 1, into members
    std::vector<uint32_t> members;        // set ids, grouped
    std::vector<uint32_t> probe_groups;   // groups with candidate groups
    std::vector<uint64_t> cand_offsets;   // n_probe_groups + 1
    std::vector<uint32_t> cand_groups;
    uint64_t n_pairs = 0;                 // member pairs the groups stand for
};

extern "C" ssj_status ssj_groups_create(const uint64_t* offsets, const uint32_t* tokens, uint32_t n_sets,
                                        const ssj_feeder_opts* opts, ssj_groups** out) {
    if (!offsets || !opts || !out || (offsets[n_sets] && !tokens) || offsets[0] != 0) return SSJ_EINVAL;
    if (!ssj::Filters::valid(opts->sim, opts->p, opts->q) || opts->flags) return SSJ_EINVAL;
    for (uint32_t i = 0; i < n_sets; ++i) {
        if (offsets[i + 1] < offsets[i] || offsets[i + 1] - offsets[i] >= (1ull << 31)) return SSJ_EINVAL;
        for (uint64_t t = offsets[i] + 1; t < offsets[i + 1]; ++t)
            if (tokens[t - 1] >= tokens[t]) return SSJ_EINVAL;
    }
    ssj::Filters flt;
    flt.sim = opts->sim;
    flt.p = opts->p;
    flt.q = opts->q;
    std::unique_ptr<ssj_groups> g(new ssj_groups());
    try {
        // preprocessing of Section 2.2.1: renumber, order by (size, lexicographic, id)
        std::vector<uint32_t> tk;
        ssj::renumber_by_frequency(offsets, tokens, n_sets, tk);
        std::vector<uint32_t> order(n_sets);
        for (uint32_t i = 0; i < n_sets; ++i) order[i] = i;
        const uint64_t* of = offsets;
        std::sort(order.begin(), order.end(), [of, &tk](uint32_t a, uint32_t b) {
            const uint64_t na = of[a + 1] - of[a], nb = of[b + 1] - of[b];
            if (na != nb) return na < nb;
            for (uint64_t i = 0; i < na; ++i)
                if (tk[of[a] + i] != tk[of[b] + i]) return tk[of[a] + i] < tk[of[b] + i];
            return a < b;
        });
        // groups: consecutive sets of equal size and equal prefix
        std::vector<uint32_t> gsize, gpl, grep;  // per group: set size, prefix length, representative
        g->group_offsets.push_back(0);
        for (uint32_t pos = 0; pos < n_sets; ++pos) {
            const uint32_t s = order[pos];
            const uint32_t len = (uint32_t)(of[s + 1] - of[s]);
            const uint32_t pl = flt.prefix_len(len);
            bool same = !grep.empty() && gsize.back() == len;
            if (same) {
                const uint32_t r = grep.back();
                for (uint32_t a = 0; a < pl && same; ++a) same = tk[of[r] + a] == tk[of[s] + a];
            }
            if (!same) {
                if (!grep.empty()) g->group_offsets.push_back(g->members.size());
                gsize.push_back(len);
                gpl.push_back(pl);
                grep.push_back(s);
            }
            g->members.push_back(s);
        }
        if (!grep.empty()) g->group_offsets.push_back(g->members.size());
        const uint32_t n_groups = (uint32_t)grep.size();
        // pairs inside a group: members share a non-empty prefix and their size
        for (uint32_t k = 0; k < n_groups; ++k) {
            const uint64_t m = g->group_offsets[k + 1] - g->group_offsets[k];
            if (gpl[k] > 0) g->n_pairs += m * (m - 1) / 2;
        }
        // inverted index over the groups' prefixes (positions ascending per token)
        uint32_t vocab = 0;
        for (uint32_t t : tk) vocab = std::max(vocab, t + 1);
        std::vector<uint64_t> post_off((size_t)vocab + 1, 0);
        for (uint32_t k = 0; k < n_groups; ++k)
            for (uint32_t a = 0; a < gpl[k]; ++a) post_off[tk[of[grep[k]] + a] + 1]++;
        for (size_t t = 0; t < vocab; ++t) post_off[t + 1] += post_off[t];
        std::vector<uint32_t> post(post_off[vocab]);
        std::vector<uint64_t> fill(post_off.begin(), post_off.end() - 1);
        for (uint32_t k = 0; k < n_groups; ++k)
            for (uint32_t a = 0; a < gpl[k]; ++a) post[fill[tk[of[grep[k]] + a]]++] = k;
        // probe each group against the groups before it (incremental index,
        // Section 2.2.4), with the length filter on the group size
        std::vector<uint32_t> stamp(n_groups, 0xFFFFFFFFu);
        g->cand_offsets.push_back(0);
        for (uint32_t k = 0; k < n_groups; ++k) {
            const uint32_t len = gsize[k];
            if (len == 0) continue;
            const uint64_t min_size = flt.min_overlap(len);
            const uint32_t lo = (uint32_t)(std::lower_bound(gsize.begin(), gsize.begin() + k,
                                                            (uint32_t)std::min<uint64_t>(min_size, 0xFFFFFFFFu)) -
                                           gsize.begin());
            const uint64_t start = g->cand_groups.size();
            const uint64_t mk = g->group_offsets[k + 1] - g->group_offsets[k];
            for (uint32_t a = 0; a < gpl[k]; ++a) {
                const uint32_t t = tk[of[grep[k]] + a];
                const uint32_t* lb = post.data() + post_off[t];
                const uint32_t* le = post.data() + post_off[t + 1];
                for (const uint32_t* it = std::lower_bound(lb, le, lo); it != le && *it < k; ++it) {
                    if (stamp[*it] == k) continue;
                    stamp[*it] = k;
                    g->cand_groups.push_back(*it);
                    g->n_pairs += mk * (g->group_offsets[*it + 1] - g->group_offsets[*it]);
                }
            }
            if (g->cand_groups.size() > start) {
                g->probe_groups.push_back(k);
                g->cand_offsets.push_back(g->cand_groups.size());
            }
        }
    } catch (const std::bad_alloc&) {
        return SSJ_ENOMEM;
    }
    *out = g.release();
    return SSJ_OK;
}

extern "C" ssj_status ssj_groups_info(ssj_groups* g, uint32_t* n_groups, uint32_t* n_probe_groups,
                                      uint64_t* n_cand_groups, uint64_t* n_pairs) {
    if (!g) return SSJ_EINVAL;
    if (n_groups) *n_groups = (uint32_t)(g->group_offsets.size() - 1);
    if (n_probe_groups) *n_probe_groups = (uint32_t)g->probe_groups.size();
    if (n_cand_groups) *n_cand_groups = g->cand_groups.size();
    if (n_pairs) *n_pairs = g->n_pairs;
    return SSJ_OK;
}

extern "C" ssj_status ssj_groups_copy(ssj_groups* g, uint64_t* group_offsets, uint32_t* members,
                                      uint32_t* probe_groups, uint64_t* cand_offsets, uint32_t* cand_groups) {
    if (!g || !group_offsets || !members || !probe_groups || !cand_offsets || !cand_groups) return SSJ_EINVAL;
    std::copy(g->group_offsets.begin(), g->group_offsets.end(), group_offsets);
    std::copy(g->members.begin(), g->members.end(), members);
    std::copy(g->probe_groups.begin(), g->probe_groups.end(), probe_groups);
    std::copy(g->cand_offsets.begin(), g->cand_offsets.end(), cand_offsets);
    std::copy(g->cand_groups.begin(), g->cand_groups.end(), cand_groups);
    return SSJ_OK;
}

extern "C" void ssj_groups_destroy(ssj_groups* g) { delete g; }
