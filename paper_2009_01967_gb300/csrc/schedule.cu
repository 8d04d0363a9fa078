// Host-side lane schedule of the Y-build in the linewidth kernel.
//
// The first-index contraction Y_s(b, c) = sum over the fc3 blocks of the
// (j, k) atom pair of (b, c) is irregular: for a pair potential the diagonal
// pairs (j, j) collect a block from every neighbour (about 80) while the
// others hold one to six.  The schedule gives each of the 256 threads a
// near-equal number of blocks:
//   * heavy groups (more than H blocks) are cut into R slices on R aligned
//     lanes (R a power of two), whose partial sums a warp shuffle adds
//     (fixed order, so the result does not depend on timing);
//   * light groups are packed onto lanes by longest-processing-time first.

#include <algorithm>
#include <queue>

#include "kald_internal.h"

namespace kald {

void plan_ybuild(const HostSystem &h, YSchedule &ys) {
    const int lanes = kLwThreads;
    const int n_groups = (int)h.pair3_j.size();
    ys.group_jk.resize(2 * (size_t)n_groups);
    long long total = 0;
    int maxc = 0;
    for (int g = 0; g < n_groups; ++g) {
        ys.group_jk[2 * g] = h.pair3_j[g];
        ys.group_jk[2 * g + 1] = h.pair3_k[g];
        const int c = h.pair3_start[g + 1] - h.pair3_start[g];
        total += c;
        maxc = std::max(maxc, c);
    }
    const int target = (int)std::max<long long>(1, (total + lanes - 1) / lanes);
    const int H = std::max(8, target);
    int R = 1;
    while (R < 32 && (maxc + R - 1) / R > H) R *= 2;
    std::vector<int> heavy, light;
    for (int g = 0; g < n_groups; ++g) {
        const int c = h.pair3_start[g + 1] - h.pair3_start[g];
        if (R > 1 && c > H) heavy.push_back(g); else light.push_back(g);
    }
    ys.segs.clear();
    ys.sched.clear();
    int rounds = 0;
    // heavy rounds: R aligned lanes per heavy group, one segment per lane
    const int per_round = lanes / R;
    for (size_t h0 = 0; h0 < heavy.size(); h0 += per_round) {
        for (int t = 0; t < lanes; ++t) {
            ys.sched.push_back((int)ys.segs.size());
            const size_t hi = h0 + t / R;
            if (hi < heavy.size()) {
                const int g = heavy[hi];
                const int b0 = h.pair3_start[g], n = h.pair3_start[g + 1] - b0;
                const int sl = t % R;
                const int s0 = b0 + (int)((long long)n * sl / R);
                const int s1 = b0 + (int)((long long)n * (sl + 1) / R);
                ys.segs.push_back(make_int4(g, s0, s1, R));
            } else {
                ys.segs.push_back(make_int4(-1, 0, 0, R));
            }
        }
        ++rounds;
    }
    // one light round: longest-processing-time packing onto the lanes
    if (!light.empty()) {
        std::stable_sort(light.begin(), light.end(), [&](int a, int b) {
            return (h.pair3_start[a + 1] - h.pair3_start[a]) > (h.pair3_start[b + 1] - h.pair3_start[b]);
        });
        std::vector<std::vector<int>> lane_groups(lanes);
        using Item = std::pair<long long, int>;     // (load, lane)
        std::priority_queue<Item, std::vector<Item>, std::greater<Item>> pq;
        for (int t = 0; t < lanes; ++t) pq.push({0, t});
        for (int g : light) {
            Item it = pq.top();
            pq.pop();
            lane_groups[it.second].push_back(g);
            it.first += h.pair3_start[g + 1] - h.pair3_start[g];
            pq.push(it);
        }
        for (int t = 0; t < lanes; ++t) {
            ys.sched.push_back((int)ys.segs.size());
            for (int g : lane_groups[t])
                ys.segs.push_back(make_int4(g, h.pair3_start[g], h.pair3_start[g + 1], 0));
        }
        ++rounds;
    }
    ys.sched.push_back((int)ys.segs.size());
    if (ys.segs.empty()) ys.segs.push_back(make_int4(-1, 0, 0, 0));
    ys.n_rounds = rounds;
}

}  // namespace kald
