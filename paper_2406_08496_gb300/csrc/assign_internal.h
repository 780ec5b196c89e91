// Internal state of the assignment engine (include/lpsim_assign.h keeps it
// opaque), shared by the host engine (assign.cpp) and its GPU searches
// (assign_gpu.cu).
#pragma once
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "host_par.h"

struct AssignGpu;  // device copy of the graph and search workspaces (assign_gpu.cu)
void assign_gpu_free(AssignGpu *g);

struct lpsim_assign {
    uint32_t n_nodes = 0, n_edges = 0;
    std::vector<uint32_t> src, dst, lanes;
    std::vector<float> len, vmax;
    std::vector<uint32_t> out_off, out_edge;  // CSR of out-edges by source node
    // trips
    uint64_t n = 0;
    std::vector<uint32_t> orig, dest, dep;    // depart step
    std::vector<std::vector<uint32_t>> route, cand;
    std::vector<float> tsp;                   // shortest time under the last tt (s)
    std::vector<float> excess;                // current route's time minus tsp (s), from a simulation or a prediction
    float dt = 0.5f;
    uint64_t seed = 0;
    AssignGpu *gpu = nullptr;
    ~lpsim_assign() { assign_gpu_free(gpu); }
};

namespace lpsim_assign_detail {

// A link time in whole milliseconds: nearest, at least 1 ms.  Integer times
// make every path time an exact sum, whatever order it is added in.
inline uint32_t cost_ms(float seconds) {
    const long long m = std::llround((double)seconds * 1000.0);
    return (uint32_t)std::min<long long>(std::max<long long>(m, 1), 0x7FFFFFFFll);
}

inline uint64_t to_ms(double seconds) { return (uint64_t)std::llround(seconds * 1000.0); }

// Time-dependent link times in whole milliseconds.  The table gives a time
// per (edge, entry bin); entering edge e at time t (ms) in bin b (the last
// bin beyond the table) arrives at
//     arrive(e, t) = min(t + c[b][e], M[b][e]),
//     M[b][e] = min over later bins b' of (start of b' + c[b'][e]),
// i.e. a vehicle may hold back its entry to a later bin when that gets it
// out earlier.  This makes the arrival non-decreasing in the entry time (the
// FIFO property), without which a time-dependent label-setting search is not
// exact and the piecewise-constant bin table would let an earlier entry
// arrive later.  Times are rounded to the nearest millisecond (at least 1 ms)
// so every path time is an exact integer sum, independent of the order it is
// added in: the host searches and the GPU searches reach the same arrival
// times and, with ties to the lower edge id, the same paths.  The table is
// kept bin-major (n_bins x n_edges, {c, M} pairs): a search or a route walk
// stays within a few bins, so the values it reads sit in a few contiguous
// rows.
struct LinkTime {
    uint32_t c;  // link time when entered in this bin (ms)
    uint32_t m;  // earliest arrival by entering in a later bin (ms; 0xFFFFFFFF: none)
};

// bin length (ms) of a link-time table with bins of bin_steps steps
inline uint64_t table_bin_ms(const lpsim_assign *a, uint32_t bin_steps) {
    return std::max<uint64_t>(1, to_ms((double)bin_steps * a->dt));
}

// The link-time table, bin-major (n_bins x n_edges): each (edge, bin)'s time in
// ms and the earliest arrival entering a later bin, on the host's threads.
inline void fill_link_times(const lpsim_assign *a, const float *tt, uint32_t n_bins, uint64_t bin_ms, LinkTime *tbm) {
    const uint32_t ne = a->n_edges;
    lpsim::parallel_pieces(ne, [&](uint64_t e0, uint64_t e1, uint64_t) {
        for (uint64_t e = e0; e < e1; e++) {
            uint64_t m = 0xFFFFFFFFull;
            for (uint32_t b = n_bins; b-- > 0;) {
                const uint32_t c = cost_ms(tt[e * n_bins + b]);
                tbm[(size_t)b * ne + e] = LinkTime{c, (uint32_t)m};
                m = std::min<uint64_t>(m, (uint64_t)b * bin_ms + c);
            }
        }
    });
}

struct TD {
    const lpsim_assign *a;
    std::vector<LinkTime> tbm;  // n_bins x n_edges
    uint32_t n_bins;
    uint64_t bin_ms;

    TD(const lpsim_assign *a_, const float *tt, uint32_t n_bins_, uint32_t bin_steps)
        : a(a_), tbm((size_t)n_bins_ * a_->n_edges), n_bins(n_bins_), bin_ms(table_bin_ms(a_, bin_steps)) {
        fill_link_times(a, tt, n_bins, bin_ms, tbm.data());
    }

    uint32_t bin(uint64_t t) const { return (uint32_t)std::min<uint64_t>(t / bin_ms, n_bins - 1); }
    uint64_t arrive(uint32_t e, uint64_t t) const {
        const LinkTime lt = tbm[(size_t)bin(t) * a->n_edges + e];
        return std::min<uint64_t>(t + lt.c, lt.m);
    }
};

// Trips grouped by (origin, departure period): order[] lists trip indices
// group by group (groups ascending by origin, then period; trips ascending
// within a group), gstart[] the first position of each group plus the end.
inline void group_trips(const lpsim_assign *a, uint32_t period_steps, std::vector<uint64_t> &order,
                        std::vector<uint64_t> &gstart) {
    order.resize(a->n);
    for (uint64_t j = 0; j < a->n; j++) order[j] = j;
    auto key = [&](uint64_t j) { return ((uint64_t)a->orig[j] << 32) | (a->dep[j] / period_steps); };
    std::sort(order.begin(), order.end(), [&](uint64_t x, uint64_t y) {
        const uint64_t kx = key(x), ky = key(y);
        return kx != ky ? kx < ky : x < y;
    });
    gstart.clear();
    for (uint64_t i = 0; i < a->n; i++)
        if (i == 0 || key(order[i]) != key(order[i - 1])) gstart.push_back(i);
    gstart.push_back(a->n);
}

// Root time of a group's tree: the middle of its departure period (ms).
inline uint64_t period_root_ms(const lpsim_assign *a, uint32_t period, uint32_t period_steps) {
    return to_ms(((double)period + 0.5) * period_steps * a->dt);
}

}  // namespace lpsim_assign_detail
