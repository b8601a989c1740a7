// sifter.cpp -- candidate sifting after the single-pulse search (arXiv
// 2606.27262, Sec. 3.2.1): DBSCAN clustering of a beam's candidates in the
// DM-time plane (neighbourhood radius eps, at least min_points points within
// eps of a core point, the point itself included), the highest-S/N member of
// each cluster kept, then thresholds on S/N, DM and width.  Points that
// belong to no cluster are dropped.
//
// Coordinates: DM in pc cm^-3 and arrival time in seconds (sample index x
// sampling time), Euclidean distance, a neighbour when the distance is at
// most eps.  Points are visited in (dm_idx, t) order and clusters grow
// breadth first from the first unvisited core point, so the assignment of
// border points (reachable from two clusters) is deterministic: the cluster
// that reaches them first keeps them.
//
// Host code: a uniform grid of eps-sized cells finds neighbours in the 3x3
// cells around a point.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <unordered_map>
#include <vector>

#include "sp_internal.h"

namespace {

struct Pt {
    double x, y;   // DM, time (s)
    int64_t src;   // index in the caller's array
};

inline int64_t cell_key(int64_t ix, int64_t iy) { return (ix << 32) ^ (iy & 0xffffffffLL); }

}  // namespace

extern "C" int sp_sift(const sp_cand *h_cands, int64_t n, const double *h_dms, int32_t ndm, const int32_t *h_widths,
                       int32_t nw, double tsamp_s, const sp_sift_params *params, sp_cand *h_out, int64_t cap,
                       int64_t *n_out, int32_t *h_labels) {
    if (n < 0 || !n_out || !params || !h_dms || ndm <= 0 || !h_widths || nw <= 0 || !(tsamp_s > 0.0) ||
        (n > 0 && !h_cands) || cap < 0 || (cap > 0 && !h_out))
        return SP_EINVAL;
    const sp_sift_params &P = *params;
    if (!(P.eps > 0.0f) || P.min_points < 1) return SP_EINVAL;
    *n_out = 0;
    for (int64_t i = 0; i < n; ++i) {
        const sp_cand &c = h_cands[i];
        if (c.dm_idx < 0 || c.dm_idx >= ndm || c.width_idx < 0 || c.width_idx >= nw || c.t < 0) return SP_EINVAL;
    }
    // Canonical visiting order.
    std::vector<int64_t> order((size_t)n);
    for (int64_t i = 0; i < n; ++i) order[(size_t)i] = i;
    std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
        const sp_cand &p = h_cands[a], &q = h_cands[b];
        if (p.dm_idx != q.dm_idx) return p.dm_idx < q.dm_idx;
        if (p.t != q.t) return p.t < q.t;
        return a < b;
    });
    std::vector<Pt> pts((size_t)n);
    const double eps = (double)P.eps, eps2 = eps * eps;
    std::unordered_map<int64_t, std::vector<int32_t>> grid;
    grid.reserve((size_t)n);
    for (int64_t k = 0; k < n; ++k) {
        const sp_cand &c = h_cands[order[(size_t)k]];
        pts[(size_t)k] = {h_dms[c.dm_idx], (double)c.t * tsamp_s, order[(size_t)k]};
        const int64_t ix = (int64_t)std::floor(pts[(size_t)k].x / eps), iy = (int64_t)std::floor(pts[(size_t)k].y / eps);
        grid[cell_key(ix, iy)].push_back((int32_t)k);
    }
    auto neighbours = [&](int64_t k, std::vector<int32_t> &out) {
        out.clear();
        const Pt &p = pts[(size_t)k];
        const int64_t ix = (int64_t)std::floor(p.x / eps), iy = (int64_t)std::floor(p.y / eps);
        for (int64_t dx = -1; dx <= 1; ++dx)
            for (int64_t dy = -1; dy <= 1; ++dy) {
                auto it = grid.find(cell_key(ix + dx, iy + dy));
                if (it == grid.end()) continue;
                for (int32_t j : it->second) {
                    const double ddx = pts[(size_t)j].x - p.x, ddy = pts[(size_t)j].y - p.y;
                    if (ddx * ddx + ddy * ddy <= eps2) out.push_back(j);
                }
            }
        std::sort(out.begin(), out.end());  // expansion order independent of the hash layout
    };
    // DBSCAN: label -2 unvisited, -1 noise, >= 0 cluster.
    std::vector<int32_t> label((size_t)n, -2);
    std::vector<int32_t> nb, nb2, queue;
    int32_t nclusters = 0;
    for (int64_t k = 0; k < n; ++k) {
        if (label[(size_t)k] != -2) continue;
        neighbours(k, nb);
        if ((int64_t)nb.size() < P.min_points) {
            label[(size_t)k] = -1;
            continue;
        }
        const int32_t c = nclusters++;
        label[(size_t)k] = c;
        queue.assign(nb.begin(), nb.end());
        for (size_t q = 0; q < queue.size(); ++q) {
            const int32_t j = queue[q];
            if (label[(size_t)j] == -1) label[(size_t)j] = c;  // border point
            if (label[(size_t)j] != -2) continue;
            label[(size_t)j] = c;
            neighbours(j, nb2);
            if ((int64_t)nb2.size() >= P.min_points) queue.insert(queue.end(), nb2.begin(), nb2.end());
        }
    }
    if (h_labels)
        for (int64_t k = 0; k < n; ++k) h_labels[pts[(size_t)k].src] = label[(size_t)k];
    // Peak of each cluster: highest S/N, ties to the first in visiting order.
    std::vector<int64_t> best((size_t)nclusters, -1);
    for (int64_t k = 0; k < n; ++k) {
        const int32_t c = label[(size_t)k];
        if (c < 0) continue;
        const int64_t b = best[(size_t)c];
        if (b < 0 || h_cands[pts[(size_t)k].src].snr > h_cands[pts[(size_t)b].src].snr) best[(size_t)c] = k;
    }
    // Thresholds (Sec. 3.2.1), then output in (dm_idx, t) order.
    std::vector<int64_t> keep;
    for (int32_t c = 0; c < nclusters; ++c) {
        const sp_cand &p = h_cands[pts[(size_t)best[(size_t)c]].src];
        const double width_s = (double)h_widths[p.width_idx] * tsamp_s;
        if (p.snr < P.snr_min || h_dms[p.dm_idx] < (double)P.dm_min || width_s > (double)P.width_max_s) continue;
        keep.push_back(best[(size_t)c]);
    }
    std::sort(keep.begin(), keep.end());  // visiting order = (dm_idx, t)
    *n_out = (int64_t)keep.size();
    const int64_t m = std::min<int64_t>(cap, (int64_t)keep.size());
    for (int64_t i = 0; i < m; ++i) h_out[i] = h_cands[pts[(size_t)keep[(size_t)i]].src];
    return (int64_t)keep.size() > cap ? SP_EOVERFLOW : SP_OK;
}
