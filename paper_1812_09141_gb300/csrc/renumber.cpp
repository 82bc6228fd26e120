// Token renumbering by ascending global frequency (Section 2.2.1): each
// token is replaced by its rank when the distinct tokens are ordered by
// (number of sets containing it, token value), so infrequent tokens come
// first in every set; each set is then re-sorted.  Used by the collection
// loader (SSJ_RENUMBER_BY_FREQ) and by the candidate feeder.
#include <algorithm>
#include <cstdint>
#include <utility>
#include <vector>

namespace ssj {

void renumber_by_frequency(const uint64_t* offsets, const uint32_t* tokens, uint32_t n, std::vector<uint32_t>& out) {
    const uint64_t total = offsets[n];
    std::vector<uint32_t> sorted(tokens, tokens + total);
    std::sort(sorted.begin(), sorted.end());
    std::vector<uint32_t> distinct;
    std::vector<std::pair<uint32_t, uint32_t>> by_freq;  // (count, token)
    for (uint64_t i = 0; i < total;) {
        uint64_t j = i;
        while (j < total && sorted[j] == sorted[i]) ++j;
        distinct.push_back(sorted[i]);
        by_freq.emplace_back((uint32_t)(j - i), sorted[i]);
        i = j;
    }
    std::vector<uint32_t>().swap(sorted);
    std::sort(by_freq.begin(), by_freq.end());
    std::vector<uint32_t> rank(distinct.size());
    for (size_t k = 0; k < by_freq.size(); ++k) {
        const size_t pos = std::lower_bound(distinct.begin(), distinct.end(), by_freq[k].second) - distinct.begin();
        rank[pos] = (uint32_t)k;
    }
    out.resize(total);
    for (uint64_t t = 0; t < total; ++t)
        out[t] = rank[std::lower_bound(distinct.begin(), distinct.end(), tokens[t]) - distinct.begin()];
    for (uint32_t s = 0; s < n; ++s) std::sort(out.begin() + offsets[s], out.begin() + offsets[s + 1]);
}

}  // namespace ssj
