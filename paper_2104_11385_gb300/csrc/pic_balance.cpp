// pic_balance.cpp -- the load-balancing routine of arXiv 2104.11385 Sec. 2.2,
// host C++: load-balance efficiency (Eq. 1), the knapsack and Morton
// space-filling-curve policies, the improvement threshold, the Sec. 4 speedup
// model, and the cutting of boxes into work units for the persistent kernel.
#include "pic_balance.h"

#include <algorithm>
#include <cmath>
#include <numeric>

namespace pic {

double lb_efficiency(const double* costs, const int32_t* assign, int64_t nboxes, int n_workers) {
    std::vector<double> load(n_workers, 0.0);
    for (int64_t b = 0; b < nboxes; ++b) load[assign[b]] += costs[b];
    double total = 0.0, mx = 0.0;
    for (int w = 0; w < n_workers; ++w) {
        total += load[w];
        mx = std::max(mx, load[w]);
    }
    if (mx == 0.0) return 1.0;
    return (total / (double)n_workers) / mx;
}

// Greedy longest-processing-time-first with a cap on boxes per worker.
void knapsack(const double* costs, int64_t nboxes, int n_workers, double cap_factor,
              int32_t* assign) {
    std::vector<int64_t> order(nboxes);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int64_t a, int64_t b) { return costs[a] > costs[b]; });
    const int64_t cap_ceil = (nboxes + n_workers - 1) / n_workers;
    const int64_t cap_f = (int64_t)std::floor(cap_factor * (double)nboxes / (double)n_workers);
    const int64_t cap = std::max(cap_ceil, cap_f);
    // min-heap keyed by (load, worker id) over workers below the cap; a worker
    // that reaches the cap leaves the heap
    using Entry = std::pair<double, int>;
    auto cmp = [](const Entry& a, const Entry& b) {
        return a.first > b.first || (a.first == b.first && a.second > b.second);
    };
    std::vector<Entry> heap;
    heap.reserve(n_workers);
    for (int w = 0; w < n_workers; ++w) heap.push_back({0.0, w});
    std::make_heap(heap.begin(), heap.end(), cmp);
    std::vector<int64_t> cnt(n_workers, 0);
    for (int64_t b : order) {
        std::pop_heap(heap.begin(), heap.end(), cmp);
        Entry e = heap.back();
        heap.pop_back();
        assign[b] = e.second;
        e.first += costs[b];
        if (++cnt[e.second] < cap) {
            heap.push_back(e);
            std::push_heap(heap.begin(), heap.end(), cmp);
        }
    }
}

uint64_t morton_key(int dim, int64_t bx, int64_t by, int64_t bz) {
    // spread the bits of each coordinate with shift-and-mask steps
    auto spread3 = [](uint64_t v) {
        v &= 0x1fffffull;
        v = (v | (v << 32)) & 0x1f00000000ffffull;
        v = (v | (v << 16)) & 0x1f0000ff0000ffull;
        v = (v | (v << 8)) & 0x100f00f00f00f00full;
        v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
        v = (v | (v << 2)) & 0x1249249249249249ull;
        return v;
    };
    auto spread2 = [](uint64_t v) {
        v &= 0xffffffffull;
        v = (v | (v << 16)) & 0x0000ffff0000ffffull;
        v = (v | (v << 8)) & 0x00ff00ff00ff00ffull;
        v = (v | (v << 4)) & 0x0f0f0f0f0f0f0f0full;
        v = (v | (v << 2)) & 0x3333333333333333ull;
        v = (v | (v << 1)) & 0x5555555555555555ull;
        return v;
    };
    if (dim == 3)
        return spread3((uint64_t)bx) | (spread3((uint64_t)by) << 1) | (spread3((uint64_t)bz) << 2);
    return spread2((uint64_t)bx) | (spread2((uint64_t)bz) << 1);
}

void sfc(const double* costs, const int32_t* ijk, int64_t nboxes, int dim, int n_workers,
         int32_t* assign) {
    std::vector<std::pair<uint64_t, int64_t>> keyed(nboxes);
    for (int64_t b = 0; b < nboxes; ++b)
        keyed[b] = {morton_key(dim, ijk[3 * b], ijk[3 * b + 1], ijk[3 * b + 2]), b};
    std::sort(keyed.begin(), keyed.end());
    double total = 0.0;
    for (const auto& kb : keyed) total += costs[kb.second];
    double prefix = 0.0;
    int w = 0;
    for (const auto& kb : keyed) {
        assign[kb.second] = w;
        prefix += costs[kb.second];
        if (w < n_workers - 1 && prefix * (double)n_workers >= (double)(w + 1) * total) ++w;
    }
}

bool adopt(double e_old, double e_new, double theta) { return e_new >= (1.0 + theta) * e_old; }

double predicted_speedup(double e0, double x) { return std::pow(1.0 / e0, x); }

// Cuts boxes into units: a box of cost c gets ceil(c / target) units (at most
// one per min_particles particles, at least one), target = total /
// (n_workers * split).  Unit cost = box cost / units.
std::vector<Unit> make_units(const double* costs, const int64_t* np, int64_t nboxes, int n_workers,
                             int split, int64_t min_particles, bool allow_split) {
    double total = 0.0;
    for (int64_t b = 0; b < nboxes; ++b) total += costs[b];
    const double target = total / ((double)n_workers * (double)std::max(1, split));
    std::vector<Unit> units;
    units.reserve(nboxes);
    for (int64_t b = 0; b < nboxes; ++b) {
        int64_t k = 1;
        if (allow_split && target > 0.0 && costs[b] > target) {
            k = (int64_t)std::ceil(costs[b] / target);
            int64_t kmax = std::max<int64_t>(1, np[b] / std::max<int64_t>(1, min_particles));
            k = std::min(k, kmax);
            k = std::min<int64_t>(k, 1 << 20);
        }
        for (int64_t c = 0; c < k; ++c) units.push_back(Unit{(int32_t)b, (int32_t)c, (int32_t)k, costs[b] / (double)k});
    }
    return units;
}

}  // namespace pic
